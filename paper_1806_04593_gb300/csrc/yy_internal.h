// Internal declarations shared by the translation units of libyy.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "yy.h"

#define YY_LMAX_CAP 80
#define YY_GL_WEIGHT_NODES 32

// Device error word bits (set with atomicOr, read by yy_last_device_status).
#define YY_DEVERR_CHECK 1
#define YY_DEVERR_TIMEOUT 2

// Operand tables of one reduced-precision form (tensor-core path).
struct yy_tc_tables;

struct yy_grid {
  int device;
  int n_r, n_theta, n_phi, n_ang, lmax, n_lm;
  double delta_theta, delta_phi, G;
  double th0, ph0, dth, dph;

  // float64 tables (device)
  double *r_edges;     // [n_r + 1]
  double *w;           // [n_theta][n_phi]        overlap weights
  double *tbar;        // [n_theta][n_lm]         K_lm T_j^(lm)
  double *ban;         // [n_lm][n_ang]           analysis operand (K-major)
  double *ysyn;        // [n_ang][n_lm]           synthesis operand (own frame)
  double *ysyn_t;      // [n_ang][n_lm]           d/dtheta
  double *ysyn_p;      // [n_ang][n_lm]           (1/sin) d/dphi
  double *rot;         // [sum_l (2l+1)^2]        D^l, other-frame harmonics in own-frame ones
  float *rot32;        // same, rounded to float32
  double *scan;        // [n_r][lmax+1][8]        a_in, b_in, e_out, f_out, output factors
  double *scan_maps;   // [2][chunks][n_lm] x 4   per-chunk affine maps of the scans
  double *gl_nodes;    // GL nodes / weights on [0, 1] for the weight integrals

  // workspace (device)
  double *A;           // [2 n_r][n_lm]           moments of each patch's own cells
  double *Atot;        // [2 n_r][n_lm]           both patches' moments in each patch's frame
  double *part;        // split-K partials [split][2 n_r][n_lm]
  int split_k;
  double *cin;         // [2 n_r][n_lm] inner scan values
  double *Q;           // [3][2 n_r][n_lm]    Phi, g_r and g_angle coefficients
  int *err;            // device error word

  // float32 form
  float *ban32, *ysyn32, *ysyn_t32, *ysyn_p32;   // same layouts as float64
  float *rho32;        // [2 n_r][n_ang]
  float *Q32;          // [3][2 n_r][n_lm]

  // tensor-core forms
  yy_tc_tables *tc[5];

  // kernels launched by the last yy_potential call
  int launches;

  // stage timing
  int profiling;
  cudaEvent_t ev[YY_STAGE_COUNT + 1];

  // host-buffer staging (yy_potential_host)
  double *stage_rho, *stage_phi, *stage_grad;
};

namespace yy {

// allocation with the test hook (see yy_debug.h)
cudaError_t dmalloc(void **p, size_t bytes);

// tables (yy_tables.cu)
cudaError_t build_tables(yy_grid *g, const double *gl_host, int n_gl);
// entries of the rotation table: sum_{l <= lmax} (2l+1)^2
inline int rotation_table_size(int lmax) { return (lmax + 1) * (4 * (lmax + 1) * (lmax + 1) - 1) / 3; }

// float64 / float32 CUDA-core contractions (yy_gemm_simt.cu)
cudaError_t analysis_simt(yy_grid *g, const double *rho_yin, const double *rho_yang,
                          bool fp32, cudaStream_t s);
// Phi, and the three gradient components when grad_yin != NULL
cudaError_t synthesis_simt(yy_grid *g, double *phi_yin, double *phi_yang,
                           double *grad_yin, double *grad_yang, bool fp32, cudaStream_t s);
cudaError_t convert_tables_f32(yy_grid *g);

// Atot = A + D^T A(other patch), float32 products unless fp64 (yy_scan.cu)
cudaError_t rotate_moments(yy_grid *g, bool fp64, cudaStream_t s);
// radial scans (yy_scan.cu): Atot -> Q (and Q32 if want_f32); f64_out: output
// factors applied in float64 (else in fp32, for the reduced-precision forms)
void scan_geometry(const yy_grid *g, int *nc, int *ch);
cudaError_t radial_scan(yy_grid *g, bool want_f32, bool f64_out, cudaStream_t s);

// tensor-core path (yy_tc.cu)
yy_status tc_prepare(yy_grid *g, yy_precision prec);
void tc_free(yy_grid *g);
cudaError_t tc_analysis(yy_grid *g, yy_precision prec, const double *rho_yin,
                        const double *rho_yang, cudaStream_t s);
cudaError_t tc_pack_coefficients(yy_grid *g, yy_precision prec, cudaStream_t s);
cudaError_t tc_synthesis(yy_grid *g, yy_precision prec, double *phi_yin,
                         double *phi_yang, double *grad_yin, double *grad_yang, cudaStream_t s);

}  // namespace yy
