// C ABI of libyy: handle life cycle, argument checks and the solve pipeline.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <vector>

#include "yy_debug.h"
#include "yy_internal.h"

namespace yy {

static int g_fail_alloc_countdown = -1;   // test hook: < 0 disabled

cudaError_t dmalloc(void **p, size_t bytes) {
  *p = nullptr;
  if (g_fail_alloc_countdown == 0) return cudaErrorMemoryAllocation;
  if (g_fail_alloc_countdown > 0) --g_fail_alloc_countdown;
  return cudaMalloc(p, bytes == 0 ? 16 : bytes);
}

void simt_segments(int M, int N, int K, int *seg, int *n_seg);

// Gauss-Legendre nodes and weights on [0, 1] (weights sum to 1), by Newton
// iteration on P_n with the three-term recurrence.
static void gauss_legendre01(int n, double *x, double *w) {
  const double pi = 3.141592653589793238462643383279502884;
  for (int i = 0; i < n; ++i) {
    double z = cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = 0.0;
      for (int k = 1; k <= n; ++k) {
        const double p2 = p1;
        p1 = p0;
        p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
      }
      dp = n * (z * p0 - p1) / (z * z - 1.0);
      const double dz = p0 / dp;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

static yy_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return YY_OK;
  if (e == cudaErrorMemoryAllocation) return YY_ERR_OOM;
  return YY_ERR_CUDA;
}

static void free_all(yy_grid *g) {
  if (!g) return;
  double *dbufs[] = {g->r_edges, g->w,      g->tbar,      g->ban,       g->ysyn,  g->ysyn_t,
                     g->ysyn_p,  g->rot,    g->scan,      g->scan_maps, g->gl_nodes, g->A,
                     g->Atot,    g->part,   g->cin,       g->Q,         g->stage_rho, g->stage_phi,
                     g->stage_grad};
  for (double *p : dbufs)
    if (p) cudaFree(p);
  float *fbufs[] = {g->rot32, g->ban32, g->ysyn32, g->ysyn_t32, g->ysyn_p32, g->rho32, g->Q32,
                    g->sep_az32, g->sep_w32, g->sep_tb32};
  double *sbufs[] = {g->sep_az, g->sep_F, g->sep_F0, g->sep_P, g->sep_dP, g->sep_Qs, g->sep_tr};
  float *sfbufs[] = {g->sep_P32, g->sep_dP32, g->sep_Qs32, g->sep_tr32};
  for (float *p : sfbufs)
    if (p) cudaFree(p);
  for (double *p : sbufs)
    if (p) cudaFree(p);
  if (g->sep_tb0) cudaFree(g->sep_tb0);
  for (float *p : fbufs)
    if (p) cudaFree(p);
  if (g->err) cudaFree(g->err);
  for (int k = 0; k < 2; ++k) {
    double *pb[] = {g->pipe_rho[k], g->pipe_phi[k], g->pipe_grad[k]};
    for (double *p : pb)
      if (p) cudaFree(p);
    if (g->pipe_ev_in[k]) cudaEventDestroy(g->pipe_ev_in[k]);
    if (g->pipe_ev_done[k]) cudaEventDestroy(g->pipe_ev_done[k]);
    if (g->pipe_ev_out[k]) cudaEventDestroy(g->pipe_ev_out[k]);
  }
  if (g->pipe_in) cudaStreamDestroy(g->pipe_in);
  if (g->pipe_out) cudaStreamDestroy(g->pipe_out);
  tc_free(g);
  ozaki_free(g);
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace yy

using namespace yy;

extern "C" {

void yy_debug_fail_alloc_after(int n) { g_fail_alloc_countdown = n; }

const char *yy_status_string(yy_status s) {
  switch (s) {
    case YY_OK: return "ok";
    case YY_ERR_INVALID_ARG: return "invalid argument";
    case YY_ERR_OOM: return "device memory allocation failed";
    case YY_ERR_CUDA: return "CUDA error";
    case YY_ERR_NOT_SUPPORTED: return "not supported (precision not prepared or device lacks it)";
    case YY_ERR_TIMEOUT: return "device-side wait timed out";
    case YY_ERR_DEVICE_CHECK: return "device-side check failed";
  }
  return "unknown status";
}

static constexpr double kQuarterPi = 0.78539816339744830962;

// checks shared by both grid kinds
static bool valid_shape(const double *r_edges, int n_r, int n_theta, int n_phi, int l_max, double G) {
  if (r_edges == nullptr || n_r < 1 || n_r > (1 << 20) || n_theta < 1 || n_phi < 1 ||
      (long long)n_theta * n_phi > (1 << 24) || l_max < 0 || l_max > YY_LMAX_CAP)
    return false;
  if (!isfinite(G)) return false;
  if (!(r_edges[0] >= 0.0) || !isfinite(r_edges[0])) return false;
  for (int i = 0; i < n_r; ++i)
    if (!(r_edges[i + 1] > r_edges[i]) || !isfinite(r_edges[i + 1])) return false;
  return true;
}

static yy_status create_grid(const double *r_edges, int n_r, int n_theta, int n_phi, double delta_theta,
                             double delta_phi, int l_max, double G, bool polar, yy_grid **out) {
  const double quarter_pi = kQuarterPi;
  yy_grid *g = new (std::nothrow) yy_grid();
  if (!g) return YY_ERR_OOM;
  memset((void *)g, 0, sizeof(yy_grid));
  cudaGetDevice(&g->device);
  g->n_patch = polar ? 1 : 2;
  g->n_r = n_r;
  g->n_theta = n_theta;
  g->n_phi = n_phi;
  g->n_ang = n_theta * n_phi;
  g->lmax = l_max;
  g->n_lm = (l_max + 1) * (l_max + 1);
  g->delta_theta = delta_theta;
  g->delta_phi = delta_phi;
  g->G = G;
  if (polar) {   // theta in [0, pi], phi in [0, 2 pi)
    g->th0 = 0.0;
    g->ph0 = 0.0;
    g->dth = 4.0 * quarter_pi / n_theta;
    g->dph = 8.0 * quarter_pi / n_phi;
  } else {
    g->th0 = quarter_pi - delta_theta;
    g->ph0 = -3.0 * quarter_pi - delta_phi;
    g->dth = (2.0 * quarter_pi + 2.0 * delta_theta) / n_theta;
    g->dph = (6.0 * quarter_pi + 2.0 * delta_phi) / n_phi;
  }

  const size_t n_ang = g->n_ang, n_lm = g->n_lm, M = (size_t)grid_rows(g);
  simt_segments((int)M, (int)n_lm, (int)n_ang, &g->seg_k, &g->split_k);
  g->simt_splits = g->split_k;
  cudaError_t e = cudaSuccess;
  auto A = [&](void **p, size_t bytes) {
    if (e == cudaSuccess) e = dmalloc(p, bytes);
  };
  A((void **)&g->r_edges, (n_r + 1) * sizeof(double));
  A((void **)&g->w, n_ang * sizeof(double));
  A((void **)&g->tbar, (size_t)n_theta * n_lm * sizeof(double));
  A((void **)&g->ban, n_lm * n_ang * sizeof(double));
  A((void **)&g->ysyn, n_ang * n_lm * sizeof(double));
  A((void **)&g->ysyn_t, n_ang * n_lm * sizeof(double));
  A((void **)&g->ysyn_p, n_ang * n_lm * sizeof(double));
  if (!polar) A((void **)&g->rot, rotation_table_size(l_max) * sizeof(double));
  A((void **)&g->sep_P, (size_t)n_theta * n_lm * sizeof(double));
  A((void **)&g->sep_dP, (size_t)n_theta * n_lm * sizeof(double));
  A((void **)&g->sep_Qs, (size_t)n_theta * n_lm * sizeof(double));
  A((void **)&g->sep_tr, (size_t)(2 * l_max + 1) * n_phi * sizeof(double));
  if (!polar) A((void **)&g->rot32, rotation_table_size(l_max) * sizeof(float));
  A((void **)&g->scan, (size_t)n_r * (l_max + 1) * 8 * sizeof(double));
  {
    int nc = 1, ch = 1;
    scan_geometry(g, &nc, &ch);
    A((void **)&g->scan_maps, (size_t)g->n_patch * nc * n_lm * 4 * sizeof(double));
  }
  A((void **)&g->A, M * n_lm * sizeof(double));
  A((void **)&g->Atot, M * n_lm * sizeof(double));
  if (g->split_k > 1) A((void **)&g->part, (size_t)g->split_k * M * n_lm * sizeof(double));
  A((void **)&g->cin, M * n_lm * sizeof(double));
  A((void **)&g->Q, 3 * M * n_lm * sizeof(double));
  A((void **)&g->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(g->r_edges, r_edges, (n_r + 1) * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(g->err, 0, sizeof(int));
  if (e == cudaSuccess) {
    const int n_gl = l_max + 32, n_mu = l_max + 1;
    std::vector<double> gl(2 * YY_GL_WEIGHT_NODES + 2 * n_gl + 2 * n_mu);
    gauss_legendre01(YY_GL_WEIGHT_NODES, gl.data(), gl.data() + YY_GL_WEIGHT_NODES);
    double *tg = gl.data() + 2 * YY_GL_WEIGHT_NODES;
    gauss_legendre01(n_gl, tg, tg + n_gl);
    gauss_legendre01(n_mu, tg + 2 * n_gl, tg + 2 * n_gl + n_mu);
    e = build_tables(g, gl.data(), n_gl);
  }
  if (e == cudaSuccess) e = separable_prepare(g);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    const yy_status st = from_cuda(e);
    cudaGetLastError();
    free_all(g);
    delete g;
    return st;
  }
  *out = g;
  return YY_OK;
}

yy_status yy_grid_create(const double *r_edges, int n_r, int n_theta, int n_phi, double delta_theta,
                         double delta_phi, int l_max, double G, yy_grid **out) {
  if (out == nullptr) return YY_ERR_INVALID_ARG;
  *out = nullptr;
  if (!valid_shape(r_edges, n_r, n_theta, n_phi, l_max, G)) return YY_ERR_INVALID_ARG;
  if (!(delta_theta >= 0.0 && delta_theta < kQuarterPi) || !(delta_phi >= 0.0 && delta_phi < kQuarterPi))
    return YY_ERR_INVALID_ARG;
  return create_grid(r_edges, n_r, n_theta, n_phi, delta_theta, delta_phi, l_max, G, false, out);
}

yy_status yy_polar_grid_create(const double *r_edges, int n_r, int n_theta, int n_phi, int l_max, double G,
                               yy_grid **out) {
  if (out == nullptr) return YY_ERR_INVALID_ARG;
  *out = nullptr;
  if (!valid_shape(r_edges, n_r, n_theta, n_phi, l_max, G)) return YY_ERR_INVALID_ARG;
  return create_grid(r_edges, n_r, n_theta, n_phi, 0.0, 0.0, l_max, G, true, out);
}

yy_status yy_grid_set_analysis(yy_grid *g, yy_analysis method) {
  if (!g || (method != YY_ANALYSIS_AUTO && method != YY_ANALYSIS_SEPARABLE && method != YY_ANALYSIS_DENSE))
    return YY_ERR_INVALID_ARG;
  g->analysis_method = (int)method;
  if (method == YY_ANALYSIS_SEPARABLE)   // the separable tensor-core tables of the prepared forms
    for (yy_precision p : {YY_TF32, YY_BF16X3, YY_FP16X2}) {
      const yy_status st = tc_build_separable(g, p);
      if (st != YY_OK) return st;
    }
  return YY_OK;
}

int yy_grid_analysis_splits(const yy_grid *g, yy_precision prec, int *rule, int *max_splits) {
  if (!g) return -1;
  switch (prec) {
    case YY_FP64:
    case YY_FP32:
    case YY_FP64_OZAKI:
      if (rule) *rule = g->split_k;
      if (max_splits) *max_splits = g->split_k;
      return g->simt_splits;
    case YY_TF32:
    case YY_BF16X3:
    case YY_FP16X2: return tc_analysis_splits(g, prec, rule, max_splits);
  }
  return -1;
}

yy_status yy_grid_set_analysis_splits(yy_grid *g, yy_precision prec, int splits) {
  if (!g || splits < 0) return YY_ERR_INVALID_ARG;
  switch (prec) {
    case YY_FP64:
    case YY_FP32:
    case YY_FP64_OZAKI:
      if (splits > g->split_k) return YY_ERR_INVALID_ARG;
      g->simt_splits = splits == 0 ? g->split_k : splits;
      return YY_OK;
    case YY_TF32:
    case YY_BF16X3:
    case YY_FP16X2: {
      int rule = 0;
      if (tc_analysis_splits(g, prec, &rule, nullptr) == 0) return YY_ERR_NOT_SUPPORTED;
      return tc_set_analysis_splits(g, prec, splits == 0 ? rule : splits);
    }
  }
  return YY_ERR_INVALID_ARG;
}

yy_status yy_grid_prepare(yy_grid *g, yy_precision prec) {
  if (!g) return YY_ERR_INVALID_ARG;
  switch (prec) {
    case YY_FP64: return YY_OK;
    case YY_FP32: {
      if (g->ban32) return YY_OK;
      cudaError_t e = convert_tables_f32(g);
      if (e == cudaSuccess) e = cudaDeviceSynchronize();
      return from_cuda(e);
    }
    case YY_TF32:
    case YY_BF16X3:
    case YY_FP16X2: return tc_prepare(g, prec);
    case YY_FP64_OZAKI: {
      const yy_status st = ozaki_prepare(g);
      return st == YY_OK ? from_cuda(cudaDeviceSynchronize()) : st;
    }
  }
  return YY_ERR_INVALID_ARG;
}

static yy_status check_solve_args(yy_grid *g, const double *rho_yin, const double *rho_yang,
                                  double *phi_yin, double *phi_yang, double *grad_yin,
                                  double *grad_yang, yy_precision prec) {
  if (!g || !rho_yin || !phi_yin) return YY_ERR_INVALID_ARG;
  if (g->n_patch == 1) {   // polar grid: one patch, the Yang arguments stay NULL
    if (rho_yang || phi_yang || grad_yang) return YY_ERR_INVALID_ARG;
  } else {
    if (!rho_yang || !phi_yang) return YY_ERR_INVALID_ARG;
    if ((grad_yin == nullptr) != (grad_yang == nullptr)) return YY_ERR_INVALID_ARG;
  }
  const void *ptrs[] = {rho_yin, rho_yang, phi_yin, phi_yang, grad_yin, grad_yang};
  for (const void *p : ptrs)
    if (p && !aligned16(p)) return YY_ERR_INVALID_ARG;
  if ((int)prec < 0 || (int)prec > (int)YY_FP64_OZAKI) return YY_ERR_INVALID_ARG;
  if (prec == YY_FP32 && !g->ban32) return YY_ERR_NOT_SUPPORTED;
  if (prec == YY_FP64_OZAKI && !ozaki_ready(g)) return YY_ERR_NOT_SUPPORTED;
  if ((prec == YY_TF32 || prec == YY_BF16X3 || prec == YY_FP16X2) && !g->tc[prec]) return YY_ERR_NOT_SUPPORTED;
  return YY_OK;
}

yy_status yy_potential(yy_grid *g, const double *rho_yin, const double *rho_yang, double *phi_yin,
                       double *phi_yang, double *grad_yin, double *grad_yang, yy_precision prec,
                       void *cuda_stream) {
  yy_status st = check_solve_args(g, rho_yin, rho_yang, phi_yin, phi_yang, grad_yin, grad_yang, prec);
  if (st != YY_OK) return st;
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != g->device) return YY_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const bool prof = g->profiling != 0;
  cudaError_t e = cudaSuccess;
  auto mark = [&](int i) {
    if (prof && e == cudaSuccess) e = cudaEventRecord(g->ev[i], s);
  };
  // YY_FP64_OZAKI: the analysis and the scans of YY_FP64, the synthesis by the Ozaki scheme
  const bool ozaki = prec == YY_FP64_OZAKI;
  if (ozaki) prec = YY_FP64;
  const bool simt = (prec == YY_FP64 || prec == YY_FP32);
  const bool f32 = (prec == YY_FP32);
  g->launches = 0;
  g->atot_done = 0;
  mark(0);
  if (e == cudaSuccess) {
    const bool separable = g->analysis_method == YY_ANALYSIS_SEPARABLE ||
                           (g->analysis_method == YY_ANALYSIS_AUTO && simt);
    const bool tc_sep = separable && !simt && tc_separable_analysis_ready(g, prec);
    const bool oz_an = ozaki && separable && ozaki_analysis_ready(g);
    g->last_separable = tc_sep || oz_an || (separable && (g->sep_ok & (prec == YY_FP64 ? 2 : 1)));
    if (oz_an)
      e = ozaki_analysis(g, rho_yin, rho_yang, s);
    else if (tc_sep)
      e = tc_separable_analysis(g, prec, rho_yin, rho_yang, s);
    else if (g->last_separable)
      e = analysis_separable(g, rho_yin, rho_yang, prec == YY_FP64, s);
    else
      e = simt ? analysis_simt(g, rho_yin, rho_yang, f32, s) : tc_analysis(g, prec, rho_yin, rho_yang, s);
  }
  mark(1);
  // synthesis evaluation: on the CUDA-core forms separable unless
  // YY_ANALYSIS_DENSE is set; on the tensor-core forms dense unless
  // YY_ANALYSIS_SEPARABLE is set (there the dense contraction is faster);
  // dense wherever the grid does not fit the separable kernels
  const bool sep_synth = ozaki || (simt ? (g->analysis_method != YY_ANALYSIS_DENSE && (g->sep_syn_ok & (f32 ? 1 : 2)) != 0)
                                        : (g->analysis_method == YY_ANALYSIS_SEPARABLE && tc_separable_synthesis_ready(g, prec)));
  g->last_sep_synthesis = sep_synth ? 1 : 0;
  if (e == cudaSuccess && !g->atot_done) e = ozaki ? ozaki_rotate(g, s) : rotate_moments(g, prec == YY_FP64, s);
  // the separable tensor-core synthesis reads the coefficients in fp32 (the scan's copy)
  if (e == cudaSuccess) e = radial_scan(g, f32 || (sep_synth && !simt && !ozaki), true, s);
  if (e == cudaSuccess && !simt)
    e = sep_synth ? tc_theta(g, prec, grad_yin != nullptr, s) : tc_pack_coefficients(g, prec, s);
  mark(2);
  if (e == cudaSuccess) {
    if (ozaki)
      e = ozaki_synthesis(g, phi_yin, phi_yang, grad_yin, grad_yang, s);
    else if (simt)
      e = sep_synth ? synthesis_separable(g, phi_yin, phi_yang, grad_yin, grad_yang, !f32, s)
                    : synthesis_simt(g, phi_yin, phi_yang, grad_yin, grad_yang, f32, s);
    else
      e = sep_synth ? tc_separable_synthesis(g, prec, phi_yin, phi_yang, grad_yin, grad_yang, s)
                    : tc_synthesis(g, prec, phi_yin, phi_yang, grad_yin, grad_yang, s);
  }
  mark(3);
  return from_cuda(e);
}

yy_status yy_potential_host(yy_grid *g, const double *rho_yin, const double *rho_yang, double *phi_yin,
                            double *phi_yang, double *grad_yin, double *grad_yang, yy_precision prec,
                            void *cuda_stream) {
  if (!g || !rho_yin || !phi_yin) return YY_ERR_INVALID_ARG;
  const bool two = g->n_patch == 2;
  if (two ? (!rho_yang || !phi_yang || (grad_yin == nullptr) != (grad_yang == nullptr))
          : (rho_yang || phi_yang || grad_yang))
    return YY_ERR_INVALID_ARG;
  const size_t field = (size_t)g->n_r * g->n_ang, np = (size_t)g->n_patch;
  cudaError_t e = cudaSuccess;
  if (!g->stage_rho) e = dmalloc((void **)&g->stage_rho, np * field * sizeof(double));
  if (e == cudaSuccess && !g->stage_phi) e = dmalloc((void **)&g->stage_phi, np * field * sizeof(double));
  if (e == cudaSuccess && grad_yin && !g->stage_grad)
    e = dmalloc((void **)&g->stage_grad, 3 * np * field * sizeof(double));
  if (e != cudaSuccess) return from_cuda(e);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t bytes = field * sizeof(double);
  e = cudaMemcpyAsync(g->stage_rho, rho_yin, bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && two) e = cudaMemcpyAsync(g->stage_rho + field, rho_yang, bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return from_cuda(e);
  double *gy = grad_yin ? g->stage_grad : nullptr;
  double *gg = (grad_yin && two) ? g->stage_grad + 3 * field : nullptr;
  yy_status st = yy_potential(g, g->stage_rho, two ? g->stage_rho + field : nullptr, g->stage_phi,
                              two ? g->stage_phi + field : nullptr, gy, gg, prec, cuda_stream);
  if (st != YY_OK) return st;
  e = cudaMemcpyAsync(phi_yin, g->stage_phi, bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && two) e = cudaMemcpyAsync(phi_yang, g->stage_phi + field, bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && grad_yin) e = cudaMemcpyAsync(grad_yin, gy, 3 * bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && gg) e = cudaMemcpyAsync(grad_yang, gg, 3 * bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return from_cuda(e);
}

// Pipelined host-buffer solve.  Staging set k alternates between calls; the
// copy in (stream pipe_in) waits until the last solve that read set k is
// done, the solve (cuda_stream) waits for its copy in and for the last copy
// out of set k, and the copy out (stream pipe_out) waits for the solve.  So
// the copy out of one call runs beside the copy in and the solve of the next.
yy_status yy_potential_host_async(yy_grid *g, const double *rho_yin, const double *rho_yang, double *phi_yin,
                                  double *phi_yang, double *grad_yin, double *grad_yang, yy_precision prec,
                                  void *cuda_stream) {
  if (!g || !rho_yin || !phi_yin) return YY_ERR_INVALID_ARG;
  const bool two = g->n_patch == 2;
  if (two ? (!rho_yang || !phi_yang || (grad_yin == nullptr) != (grad_yang == nullptr))
          : (rho_yang || phi_yang || grad_yang))
    return YY_ERR_INVALID_ARG;
  const size_t field = (size_t)g->n_r * g->n_ang, np = (size_t)g->n_patch;
  cudaError_t e = cudaSuccess;
  if (!g->pipe_in) e = cudaStreamCreateWithFlags(&g->pipe_in, cudaStreamNonBlocking);
  if (e == cudaSuccess && !g->pipe_out) e = cudaStreamCreateWithFlags(&g->pipe_out, cudaStreamNonBlocking);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    if (!g->pipe_ev_in[k]) e = cudaEventCreateWithFlags(&g->pipe_ev_in[k], cudaEventDisableTiming);
    if (e == cudaSuccess && !g->pipe_ev_done[k]) e = cudaEventCreateWithFlags(&g->pipe_ev_done[k], cudaEventDisableTiming);
    if (e == cudaSuccess && !g->pipe_ev_out[k]) e = cudaEventCreateWithFlags(&g->pipe_ev_out[k], cudaEventDisableTiming);
  }
  const int k = g->pipe_next;
  if (e == cudaSuccess && !g->pipe_rho[k]) e = dmalloc((void **)&g->pipe_rho[k], np * field * sizeof(double));
  if (e == cudaSuccess && !g->pipe_phi[k]) e = dmalloc((void **)&g->pipe_phi[k], np * field * sizeof(double));
  if (e == cudaSuccess && grad_yin && !g->pipe_grad[k])
    e = dmalloc((void **)&g->pipe_grad[k], 3 * np * field * sizeof(double));
  if (e != cudaSuccess) return from_cuda(e);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t bytes = field * sizeof(double);
  double *rho = g->pipe_rho[k], *phi = g->pipe_phi[k], *grad = grad_yin ? g->pipe_grad[k] : nullptr;
  // copy in, once the last solve on this set has read it
  if (g->pipe_used[k]) e = cudaStreamWaitEvent(g->pipe_in, g->pipe_ev_done[k], 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(rho, rho_yin, bytes, cudaMemcpyHostToDevice, g->pipe_in);
  if (e == cudaSuccess && two) e = cudaMemcpyAsync(rho + field, rho_yang, bytes, cudaMemcpyHostToDevice, g->pipe_in);
  if (e == cudaSuccess) e = cudaEventRecord(g->pipe_ev_in[k], g->pipe_in);
  // solve, once the data is in and the last copy out of this set has finished
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, g->pipe_ev_in[k], 0);
  if (e == cudaSuccess && g->pipe_used[k]) e = cudaStreamWaitEvent(s, g->pipe_ev_out[k], 0);
  if (e != cudaSuccess) return from_cuda(e);
  yy_status st = yy_potential(g, rho, two ? rho + field : nullptr, phi, two ? phi + field : nullptr, grad,
                              (grad && two) ? grad + 3 * field : nullptr, prec, cuda_stream);
  if (st != YY_OK) return st;
  e = cudaEventRecord(g->pipe_ev_done[k], s);
  // copy out
  if (e == cudaSuccess) e = cudaStreamWaitEvent(g->pipe_out, g->pipe_ev_done[k], 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(phi_yin, phi, bytes, cudaMemcpyDeviceToHost, g->pipe_out);
  if (e == cudaSuccess && two) e = cudaMemcpyAsync(phi_yang, phi + field, bytes, cudaMemcpyDeviceToHost, g->pipe_out);
  if (e == cudaSuccess && grad) e = cudaMemcpyAsync(grad_yin, grad, 3 * bytes, cudaMemcpyDeviceToHost, g->pipe_out);
  if (e == cudaSuccess && grad && two)
    e = cudaMemcpyAsync(grad_yang, grad + 3 * field, 3 * bytes, cudaMemcpyDeviceToHost, g->pipe_out);
  if (e == cudaSuccess) e = cudaEventRecord(g->pipe_ev_out[k], g->pipe_out);
  if (e != cudaSuccess) return from_cuda(e);
  g->pipe_used[k] = 1;
  g->pipe_next = k ^ 1;
  return YY_OK;
}

yy_status yy_potential_host_wait(yy_grid *g) {
  if (!g) return YY_ERR_INVALID_ARG;
  cudaError_t e = cudaSuccess;
  if (g->pipe_out) e = cudaStreamSynchronize(g->pipe_out);
  if (e == cudaSuccess && g->pipe_in) e = cudaStreamSynchronize(g->pipe_in);
  return from_cuda(e);
}

yy_status yy_grid_copy_table(yy_grid *g, yy_table which, double *host_dst, size_t *count) {
  if (!g || !count) return YY_ERR_INVALID_ARG;
  const size_t n_ang = g->n_ang, n_lm = g->n_lm, M = (size_t)grid_rows(g);
  const double *src = nullptr;
  size_t n = 0;
  switch (which) {
    case YY_TABLE_WEIGHTS: src = g->w; n = n_ang; break;
    case YY_TABLE_TBAR: src = g->tbar; n = (size_t)g->n_theta * n_lm; break;
    case YY_TABLE_ANALYSIS: src = g->ban; n = n_lm * n_ang; break;
    case YY_TABLE_SYNTH: src = g->ysyn; n = n_ang * n_lm; break;
    case YY_TABLE_SYNTH_T: src = g->ysyn_t; n = n_ang * n_lm; break;
    case YY_TABLE_SYNTH_P: src = g->ysyn_p; n = n_ang * n_lm; break;
    case YY_TABLE_MOMENTS: src = g->A; n = M * n_lm; break;
    case YY_TABLE_COEFF: src = g->Q; n = 3 * M * n_lm; break;
    case YY_TABLE_ROTATION:
      if (g->n_patch != 2) return YY_ERR_NOT_SUPPORTED;   // a polar grid has no second patch
      src = g->rot;
      n = (size_t)rotation_table_size(g->lmax);
      break;
    case YY_TABLE_MOMENTS_TOTAL: src = moments_total(g); n = M * n_lm; break;
    default: return YY_ERR_INVALID_ARG;
  }
  if (host_dst == nullptr) {
    *count = n;
    return YY_OK;
  }
  if (*count != n) return YY_ERR_INVALID_ARG;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(host_dst, src, n * sizeof(double), cudaMemcpyDeviceToHost);
  return from_cuda(e);
}

yy_status yy_last_device_status(yy_grid *g) {
  if (!g) return YY_ERR_INVALID_ARG;
  int h = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&h, g->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(g->err, 0, sizeof(int));
  if (e != cudaSuccess) return from_cuda(e);
  if (h & YY_DEVERR_TIMEOUT) return YY_ERR_TIMEOUT;
  if (h & YY_DEVERR_CHECK) return YY_ERR_DEVICE_CHECK;
  return YY_OK;
}

void yy_destroy(yy_grid *g) {
  if (!g) return;
  cudaDeviceSynchronize();
  if (g->profiling) yy_grid_set_profiling(g, 0);
  free_all(g);
  delete g;
}

yy_status yy_grid_set_profiling(yy_grid *g, int enable) {
  if (!g) return YY_ERR_INVALID_ARG;
  if (enable && !g->profiling) {
    for (int i = 0; i <= YY_STAGE_COUNT; ++i) {
      cudaError_t e = cudaEventCreate(&g->ev[i]);
      if (e != cudaSuccess) return from_cuda(e);
    }
    for (int i = 0; i < YY_MAX_KERNEL_EVENTS; ++i) {
      cudaError_t e = cudaEventCreate(&g->kev[i]);
      if (e != cudaSuccess) return from_cuda(e);
      g->kname[i] = nullptr;
    }
  } else if (!enable && g->profiling) {
    cudaDeviceSynchronize();
    for (int i = 0; i <= YY_STAGE_COUNT; ++i) cudaEventDestroy(g->ev[i]);
    for (int i = 0; i < YY_MAX_KERNEL_EVENTS; ++i) cudaEventDestroy(g->kev[i]);
  }
  g->profiling = enable ? 1 : 0;
  return YY_OK;
}

yy_status yy_grid_stage_ms(yy_grid *g, double *ms) {
  if (!g || !ms || !g->profiling) return YY_ERR_INVALID_ARG;
  cudaError_t e = cudaEventSynchronize(g->ev[YY_STAGE_COUNT]);
  float t[YY_STAGE_COUNT] = {};
  for (int i = 0; i < YY_STAGE_COUNT && e == cudaSuccess; ++i)
    e = cudaEventElapsedTime(&t[i], g->ev[i], g->ev[i + 1]);
  if (e != cudaSuccess) return from_cuda(e);
  for (int i = 0; i < YY_STAGE_COUNT; ++i) ms[i] = t[i];
  return YY_OK;
}

yy_status yy_grid_kernel_ms(yy_grid *g, int index, double *ms, const char **name) {
  if (!g || !ms || !g->profiling || index < 0 || index >= g->launches || index >= YY_MAX_KERNEL_EVENTS ||
      !g->kname[index])
    return YY_ERR_INVALID_ARG;
  cudaError_t e = cudaEventSynchronize(g->kev[index]);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, index == 0 ? g->ev[0] : g->kev[index - 1], g->kev[index]);
  if (e != cudaSuccess) return from_cuda(e);
  *ms = t;
  if (name) *name = g->kname[index];
  return YY_OK;
}

int yy_last_launch_count(const yy_grid *g) { return g ? g->launches : -1; }

double yy_solve_flops(const yy_grid *g, int with_gradient) {
  if (!g) return 0.0;
  const double M = (double)grid_rows(g), K_an = g->n_ang, N_an = g->n_lm;
  const int nt = 2 * g->lmax + 1;
  const double analysis = g->last_separable
                              ? 2.0 * M * K_an * nt + 2.0 * M * g->n_theta * N_an
                              : 2.0 * M * N_an * K_an;
  const double synth = g->last_sep_synthesis ? 2.0 * M * g->n_theta * N_an + 2.0 * M * K_an * nt
                                             : 2.0 * M * g->n_lm * g->n_ang;
  double rotation = 0.0;
  for (int l = 0; l <= g->lmax && g->n_patch == 2; ++l) rotation += 2.0 * M * (2.0 * l + 1.0) * (2.0 * l + 1.0);
  return analysis + rotation + (with_gradient ? 4.0 : 1.0) * synth;
}

}  // extern "C"
