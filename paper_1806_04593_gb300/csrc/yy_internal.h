// Internal declarations shared by the translation units of libyy.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "yy.h"

#define YY_LMAX_CAP 80
#define YY_GL_WEIGHT_NODES 32
#define YY_MAX_KERNEL_EVENTS 32

// Device error word bits (set with atomicOr, read by yy_last_device_status).
#define YY_DEVERR_CHECK 1
#define YY_DEVERR_TIMEOUT 2

// Operand tables of one reduced-precision form (tensor-core path).
struct yy_tc_tables;
struct yy_oz_tables;

struct yy_grid {
  int device;
  int n_patch;          // 2: Yin-Yang; 1: full spherical polar grid (rows of every stage: n_patch n_r)
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
  // (row counts below are for the Yin-Yang grid; a polar grid has n_r rows)
  double *A;           // [2 n_r][n_lm]           moments of each patch's own cells
  double *Atot;        // [2 n_r][n_lm]           both patches' moments in each patch's frame
  double *part;        // K-segment partials [segment][2 n_r][n_lm]
  int split_k;         // K segments of the dense CUDA-core analysis (fixed by the sizes)
  int seg_k;           // K per segment (a multiple of the contraction's K step)
  int simt_splits;     // blocks along K, each taking whole segments (1 .. split_k)
  double *cin;         // [2 n_r][n_lm] inner scan values
  double *Q;           // [3][2 n_r][n_lm]    Phi, g_r and g_angle coefficients
  int *err;            // device error word

  // separable analysis (yy_separable.cu)
  int analysis_method;  // yy_analysis
  int last_sep_synthesis;   // the last solve's synthesis ran in separable form
  int last_separable;   // the last solve used the separable analysis
  int sep_nt_pad;       // 2 l_max + 1 azimuthal functions, padded to a multiple of 4
  int sep_ok;           // the grid fits the separable kernels' shared memory: bit 0 fp32, bit 1 float64
  int sep_jc[2];        // rows per item of the azimuthal stage (fp32, float64)
  int sep_phi_blocks[2];  // persistent blocks of the azimuthal stage (fp32, float64)
  double *sep_az;       // [n_phi][sep_nt_pad] cell integrals of the azimuthal functions
  float *sep_az32, *sep_w32, *sep_tb32;   // fp32 copies of sep_az, w, tbar
  double *sep_F;        // [2 n_r][n_theta][sep_nt_pad] azimuthal stage (float64 or fp32)
  double *sep_F0;       // [2 n_r][n_theta] m = 0 row sums as fp32 pairs (fp32 form)
  float2 *sep_tb0;      // [n_theta][l_max + 1] K_l0 T_j^(l0) d_phi as fp32 pairs
  double *sep_P, *sep_dP, *sep_Qs;   // [n_theta][n_lm] Legendre factors at the cell colatitudes
  double *sep_tr;                    // [2 l_max + 1][n_phi] 1, cos, sin at the cell longitudes
  float *sep_P32, *sep_dP32, *sep_Qs32, *sep_tr32;   // fp32 copies
  int sep_syn_ok;                    // the grid fits the separable synthesis's shared memory: bit 0 fp32, bit 1 float64
  int sep_syn_rows[2];               // rows of G per chunk (fp32, float64)
  size_t sep_syn_smem[2];            // its shared memory (fp32, float64)
  int sep_syn_blocks[2];             // its persistent blocks (fp32, float64)

  // float32 form
  float *ban32, *ysyn32, *ysyn_t32, *ysyn_p32;   // same layouts as float64
  float *rho32;        // [2 n_r][n_ang]
  float *Q32;          // [3][2 n_r][n_lm]

  // tensor-core forms
  yy_tc_tables *tc[5];
  // float64 by the Ozaki scheme (YY_FP64_OZAKI): slices of G and of the trig table
  yy_oz_tables *oz;

  // kernels launched by the last yy_potential call
  int launches;
  // per-kernel timing while profiling: an event recorded after each launch of
  // the solve, and the kernel's name
  cudaEvent_t kev[YY_MAX_KERNEL_EVENTS];
  const char *kname[YY_MAX_KERNEL_EVENTS];
  // the last analysis also formed Atot (the combined moments): the separate
  // combination is skipped
  int atot_done;

  // stage timing
  int profiling;
  cudaEvent_t ev[YY_STAGE_COUNT + 1];

  // host-buffer staging (yy_potential_host)
  double *stage_rho, *stage_phi, *stage_grad;
  // pipelined host-buffer solves (yy_potential_host_async): two staging sets,
  // copies in and out on their own streams, ordered by events
  double *pipe_rho[2], *pipe_phi[2], *pipe_grad[2];
  cudaStream_t pipe_in, pipe_out;
  cudaEvent_t pipe_ev_in[2], pipe_ev_done[2], pipe_ev_out[2];
  int pipe_used[2], pipe_next;
};

namespace yy {

// Count a kernel launch of the current solve; while profiling, also record an
// event after it on the launching stream (yy_grid_kernel_ms reads them).
inline void note_launch(yy_grid *g, const char *name, cudaStream_t s) {
  if (g->profiling && g->launches < YY_MAX_KERNEL_EVENTS) {
    cudaEventRecord(g->kev[g->launches], s);
    g->kname[g->launches] = name;
  }
  g->launches++;
}

// allocation with the test hook (see yy_debug.h)
cudaError_t dmalloc(void **p, size_t bytes);

// tables (yy_tables.cu)
cudaError_t build_tables(yy_grid *g, const double *gl_host, int n_gl);
// entries of the rotation table: sum_{l <= lmax} (2l+1)^2
inline int rotation_table_size(int lmax) { return (lmax + 1) * (4 * (lmax + 1) * (lmax + 1) - 1) / 3; }
// rows of the stacked per-patch arrays (moments, coefficients, outputs)
inline int grid_rows(const yy_grid *g) { return g->n_patch * g->n_r; }
// the moments the radial scans read: both patches combined (Yin-Yang) or A itself (polar)
inline const double *moments_total(const yy_grid *g) { return g->n_patch == 2 ? g->Atot : g->A; }

#ifdef __CUDACC__
// The rotation M (x, y, z) -> (-x, z, y) commutes with the reflection
// x -> -x, under which a real harmonic of order m is even or odd: cos(m phi)
// with the sign (-1)^m, sin(m phi) with (-1)^(m + 1).  So D^l_ij vanishes
// unless modes i and j have the same parity, and the sum over i runs over
// j's class only (half the products): local index 0 (m = 0) and 4k + 2,
// 4k + 3 are even, 1 and 4k, 4k + 1 (k >= 1) odd.  The table's entries
// across the classes are quadrature rounding (below 1e-16 of the others).
__device__ __forceinline__ bool rot_even(int i) { return i == 0 || (i & 3) >= 2; }

template <typename T>
__device__ __forceinline__ void rot_class_dot(const T *__restrict__ D, int w, int jj, const T *x0, const T *x1, T &s0,
                                              T &s1) {
  const bool even = rot_even(jj);
  // first index of the class, then steps alternating +1 and +3
  int i = even ? 0 : 1;
  if (even) {
    const T d = D[0];
    s0 = fma(d, x1[0], s0);
    s1 = fma(d, x0[0], s1);
    i = 2;
  } else {
    const T d = D[(size_t)w];
    s0 = fma(d, x1[1], s0);
    s1 = fma(d, x0[1], s1);
    i = 4;
  }
#pragma unroll 2
  for (; i < w; i += 4) {
    const T d = D[(size_t)i * w];
    s0 = fma(d, x1[i], s0);
    s1 = fma(d, x0[i], s1);
    if (i + 1 < w) {
      const T e = D[(size_t)(i + 1) * w];
      s0 = fma(e, x1[i + 1], s0);
      s1 = fma(e, x0[i + 1], s1);
    }
  }
}
#endif


// float64 / float32 CUDA-core contractions (yy_gemm_simt.cu)
cudaError_t analysis_simt(yy_grid *g, const double *rho_yin, const double *rho_yang,
                          bool fp32, cudaStream_t s);
// Phi, and the three gradient components when grad_yin != NULL
cudaError_t synthesis_simt(yy_grid *g, double *phi_yin, double *phi_yang,
                           double *grad_yin, double *grad_yang, bool fp32, cudaStream_t s);
cudaError_t convert_tables_f32(yy_grid *g);

// separable analysis (yy_separable.cu): tables once per grid, then per solve
cudaError_t separable_prepare(yy_grid *g);
cudaError_t analysis_separable(yy_grid *g, const double *rho_yin, const double *rho_yang, bool fp64,
                               cudaStream_t s);
cudaError_t synthesis_separable(yy_grid *g, double *phi_yin, double *phi_yang, double *grad_yin,
                                double *grad_yang, bool fp64, cudaStream_t s);
// the float64 polar stage alone: A from the azimuthal sums in sep_F
cudaError_t separable_theta_f64(yy_grid *g, cudaStream_t s);

// Atot = A + D^T A(other patch), float32 products unless fp64 (yy_scan.cu)
cudaError_t rotate_moments(yy_grid *g, bool fp64, cudaStream_t s);
// radial scans (yy_scan.cu): Atot -> Q (and Q32 if want_f32); f64_out: output
// factors applied in float64 (else in fp32, for the reduced-precision forms)
void scan_geometry(const yy_grid *g, int *nc, int *ch);
cudaError_t radial_scan(yy_grid *g, bool want_f32, bool f64_out, cudaStream_t s);

// Grouped solves (yy_tc.cu): every field solved densely in a tensor-core form,
// one launch per stage over all of them; NOT_SUPPORTED when a field does not
// fit the grouped kernels (then each field is solved on its own).
struct TcGroup;
yy_status tc_group_create(yy_grid *const *grids, int n, yy_precision prec, const double *const *rho_yin,
                          const double *const *rho_yang, double *const *phi_yin, double *const *phi_yang,
                          double *const *grad_yin, double *const *grad_yang, TcGroup **out);
cudaError_t tc_group_run(const TcGroup *grp, cudaStream_t s);
int tc_group_launches(const TcGroup *grp);
void tc_group_destroy(TcGroup *grp);

// Grouped radial scans (one launch for many fields, yy_scan.cu): a field's
// arguments when its scan takes the one-pass warp form (n_r <= 768), the
// 128-thread blocks it takes, and the launch over a device table of fields
// with a block map (per block: field << 24 | the field's own block).
struct ScanGroupField {
  int n_patch, n_r, lmax, n_lm, ch;   // ch: radii per lane, 8, 12, 18 or 24
  const double *A, *coef;
  double *Q;
  float *Q32;
};
bool scan_group_field(yy_grid *g, bool want_f32, ScanGroupField *f);
int scan_group_blocks(const ScanGroupField &f);
cudaError_t scan_group_launch(const ScanGroupField *fields, const uint32_t *block_map, int blocks, bool f64_out,
                              cudaStream_t s);

// tensor-core path (yy_tc.cu)
yy_status tc_prepare(yy_grid *g, yy_precision prec);
void tc_free(yy_grid *g);
cudaError_t tc_analysis(yy_grid *g, yy_precision prec, const double *rho_yin,
                        const double *rho_yang, cudaStream_t s);
cudaError_t tc_pack_coefficients(yy_grid *g, yy_precision prec, cudaStream_t s);
// polar stage of the separable analysis from the raw sums of the tensor-core
// azimuthal stage (yy_separable.cu; the launcher fills the tables, A and the
// sizes from the grid)
struct SepThetaPartials {
  int n_theta, n_lm, lmax1, nt_pad, nt;
  const float *part;            // [t][part_ld]: raw fp32 sums per row (shell, j)
  size_t part_ld;
  const float *row_scale;       // per row: undoes the row's power-of-two scaling
  const double *mean;           // per row: the centring value
  const float *t_scale;         // per slot t: undoes the table row's scaling
  const float *colsum;          // per slot t: sum over k of the table row
  const double *F0;             // per row: sum over k of rho w (slot 0, times d_phi in tb0)
  const float *tb;
  const float2 *tb0;
  double *A;
};
cudaError_t separable_theta_partials(yy_grid *g, SepThetaPartials a, cudaStream_t s);
size_t separable_theta_partials_smem(const yy_grid *g, int nt_pad);

// separable synthesis on the tensor cores: polar stage (G operands), then the
// azimuthal contraction; available once the form is prepared, when it fits
bool tc_separable_synthesis_ready(const yy_grid *g, yy_precision prec);
// tables of both separable tensor-core paths: built for a prepared form while
// YY_ANALYSIS_SEPARABLE is selected (never during stream capture), released
// by the batch tuner for fields that do not use them
yy_status tc_build_separable(yy_grid *g, yy_precision prec);
void tc_release_separable(yy_grid *g, yy_precision prec);
// separable analysis with its azimuthal stage on the tensor cores
bool tc_separable_analysis_ready(const yy_grid *g, yy_precision prec);
cudaError_t tc_separable_analysis(yy_grid *g, yy_precision prec, const double *rho_yin, const double *rho_yang,
                                  cudaStream_t s);
// K split of the dense tensor-core analysis: current count (0 when the form is
// not prepared), the rule's count and the largest the partial buffer holds
int tc_analysis_splits(const yy_grid *g, yy_precision prec, int *rule, int *cap);
yy_status tc_set_analysis_splits(yy_grid *g, yy_precision prec, int splits);
cudaError_t tc_theta(yy_grid *g, yy_precision prec, bool grad, cudaStream_t s);
cudaError_t tc_separable_synthesis(yy_grid *g, yy_precision prec, double *phi_yin, double *phi_yang,
                                   double *grad_yin, double *grad_yang, cudaStream_t s);
cudaError_t tc_synthesis(yy_grid *g, yy_precision prec, double *phi_yin,
                         double *phi_yang, double *grad_yin, double *grad_yang, cudaStream_t s);

// float64 synthesis with its azimuthal stage on the tensor cores by the Ozaki
// scheme (yy_tc.cu): tables once (2 l_max + 1 <= 64), then per solve
yy_status ozaki_prepare(yy_grid *g);
void ozaki_free(yy_grid *g);
bool ozaki_ready(const yy_grid *g);
// the separable analysis with its azimuthal stage by the same scheme (n_phi <= 640)
bool ozaki_analysis_ready(const yy_grid *g);
// the other patch's moments in each frame, float-float arithmetic (k_rotate_ff)
cudaError_t ozaki_rotate(yy_grid *g, cudaStream_t s);
cudaError_t ozaki_analysis(yy_grid *g, const double *rho_yin, const double *rho_yang, cudaStream_t s);
cudaError_t ozaki_synthesis(yy_grid *g, double *phi_yin, double *phi_yang, double *grad_yin, double *grad_yang,
                            cudaStream_t s);

}  // namespace yy
