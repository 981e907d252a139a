// Radial inner / outer sums of the solver (§3 Eqs. phiin / phiout) as
// float64 affine scans over r, one warp per (patch, mode).
//
// For output radius r_{n+1} (outer interface of zone n):
//   c_n = r_{n+1}^-(l+1) sum_{i<=n} R_in,i A_i  = a_n c_{n-1} + b_n A_n
//   d_n = r_{n+1}^l      sum_{i>n}  R_out,i A_i = e_n d_{n+1} + f_n A_{n+1}
// with the per-zone factors built once per grid.  Each lane folds a
// contiguous chunk of zones into one affine map x -> alpha x + beta, the warp
// combines the maps with shuffles (prefix for c, suffix for d), and each lane
// replays its chunk from the combined start value.  All factors are <= 1 in
// magnitude for the homogeneous part, so the scans are contracting.
//
// Outputs, in the layout the synthesis contraction reads ("cat" rows: the
// row of patch p holds [coefficients of p | coefficients of the other patch]):
//   Q   = -G 4 pi/(2l+1) (c_n + d_n)                         -> Phi
//   Q_r =  G 4 pi/(2l+1) (-(l+1) c_n + l d_n) / r_{n+1}      -> g_r
//   Q_t =  G 4 pi/(2l+1) (c_n + d_n) / r_{n+1}               -> g_theta, g_phi
#include "yy_internal.h"

namespace yy {
namespace {

constexpr double kFourPi = 12.566370614359172953850573533118;

__global__ void __launch_bounds__(256)
k_radial_scan(int n_r, int lmax, int n_lm, double G, const double *__restrict__ A,
              const double *__restrict__ coef, const double *__restrict__ r_edges,
              double *__restrict__ cin, double *__restrict__ Q, float *__restrict__ Q32) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= 2 * n_lm) return;
  const int p = warp / n_lm, idx = warp % n_lm;
  int l = (int)sqrt((double)idx);
  while (l * l > idx) --l;
  while ((l + 1) * (l + 1) <= idx) ++l;
  const int L1 = lmax + 1;
  const int CH = (n_r + 31) / 32;
  const int n0 = min(n_r, lane * CH), n1 = min(n_r, n0 + CH);
  const double *Ap = A + (size_t)p * n_r * n_lm + idx;
  double *Cp = cin + (size_t)p * n_r * n_lm + idx;

  // ---- inner (prefix) scan
  double al = 1.0, be = 0.0;
  for (int n = n0; n < n1; ++n) {
    const double *c = coef + ((size_t)n * L1 + l) * 4;
    const double a = c[0];
    be = fma(a, be, c[1] * Ap[(size_t)n * n_lm]);
    al *= a;
  }
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const double ao = __shfl_up_sync(0xffffffffu, al, off);
    const double bo = __shfl_up_sync(0xffffffffu, be, off);
    if (lane >= off) {
      be = fma(al, bo, be);
      al *= ao;
    }
  }
  double x = __shfl_up_sync(0xffffffffu, be, 1);
  if (lane == 0) x = 0.0;
  for (int n = n0; n < n1; ++n) {
    const double *c = coef + ((size_t)n * L1 + l) * 4;
    x = fma(c[0], x, c[1] * Ap[(size_t)n * n_lm]);
    Cp[(size_t)n * n_lm] = x;
  }

  // ---- outer (suffix) scan
  al = 1.0;
  be = 0.0;
  for (int n = n1 - 1; n >= n0; --n) {
    const double *c = coef + ((size_t)n * L1 + l) * 4;
    const double an = (n + 1 < n_r) ? Ap[(size_t)(n + 1) * n_lm] : 0.0;
    be = fma(c[2], be, c[3] * an);
    al *= c[2];
  }
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const double ao = __shfl_down_sync(0xffffffffu, al, off);
    const double bo = __shfl_down_sync(0xffffffffu, be, off);
    if (lane + off < 32) {
      be = fma(al, bo, be);
      al *= ao;
    }
  }
  double y = __shfl_down_sync(0xffffffffu, be, 1);
  if (lane == 31) y = 0.0;
  const double f_phi = -G * kFourPi / (2.0 * l + 1.0);
  const size_t row2 = 2 * (size_t)n_lm;
  const size_t qsz = (size_t)2 * n_r * row2;
  for (int n = n1 - 1; n >= n0; --n) {
    const double *c = coef + ((size_t)n * L1 + l) * 4;
    const double an = (n + 1 < n_r) ? Ap[(size_t)(n + 1) * n_lm] : 0.0;
    y = fma(c[2], y, c[3] * an);
    const double cn = Cp[(size_t)n * n_lm];
    const double inv_r = 1.0 / r_edges[n + 1];
    const double q = f_phi * (cn + y);
    const double qr = -f_phi * (-(l + 1.0) * cn + l * y) * inv_r;
    const double qt = -q * inv_r;
    const size_t own = (size_t)(p * n_r + n) * row2 + idx;
    const size_t oth = (size_t)((1 - p) * n_r + n) * row2 + n_lm + idx;
    Q[own] = q;
    Q[oth] = q;
    Q[qsz + own] = qr;
    Q[qsz + oth] = qr;
    Q[2 * qsz + own] = qt;
    Q[2 * qsz + oth] = qt;
    if (Q32 != nullptr) {
      Q32[own] = (float)q;
      Q32[oth] = (float)q;
      Q32[qsz + own] = (float)qr;
      Q32[qsz + oth] = (float)qr;
      Q32[2 * qsz + own] = (float)qt;
      Q32[2 * qsz + oth] = (float)qt;
    }
  }
}

}  // namespace

cudaError_t radial_scan(yy_grid *g, bool want_f32, cudaStream_t s) {
  const int warps = 2 * g->n_lm;
  const int blocks = (warps * 32 + 255) / 256;
  k_radial_scan<<<blocks, 256, 0, s>>>(g->n_r, g->lmax, g->n_lm, g->G, g->A, g->scan, g->r_edges,
                                       g->cin, g->Q, want_f32 ? g->Q32 : nullptr);
  g->launches++;
  return cudaGetLastError();
}

}  // namespace yy
