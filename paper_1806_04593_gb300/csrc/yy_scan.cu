// Radial inner / outer sums of the solver (§3 Eqs. phiin / phiout) as
// float64 affine scans over r.
//
// For output radius r_{n+1} (outer interface of zone n):
//   c_n = r_{n+1}^-(l+1) sum_{i<=n} R_in,i A_i  = a_n c_{n-1} + b_n A_n
//   d_n = r_{n+1}^l      sum_{i>n}  R_out,i A_i = e_n d_{n+1} + f_n A_{n+1}
// with per-(zone, l) factors built once per grid.  All homogeneous factors
// are <= 1, so the recurrences are contracting.
//
// The chip's FP64 pipe is narrow, so the work is spread over every SM:
// the zones are cut into NC chunks; lane = mode (32 consecutive modes per
// warp, so every access to A, the scratch and the outputs is a contiguous
// 256-byte row segment); warp = (patch, mode group, chunk).
//   k_scan_maps   folds each chunk into one affine map per direction
//   k_scan_apply  starts each chunk from the composed maps of the chunks
//                 before (inner) / after (outer) it and replays it
// The scans read Atot, the moments of both patches expressed in the frame of
// the patch a row belongs to (k_rotate_moments, below), so each output row
// holds the complete coefficients of its patch.  Outputs [3][2 n_r][n_lm]:
//   Q   = -G 4 pi/(2l+1) (c_n + d_n)                         -> Phi
//   Q_r =  G 4 pi/(2l+1) (-(l+1) c_n + l d_n) / r_{n+1}      -> g_r
//   Q_t =  G 4 pi/(2l+1) (c_n + d_n) / r_{n+1}               -> g_theta, g_phi
#include "yy_internal.h"

namespace yy {
namespace {

__device__ __forceinline__ int mode_degree(int idx) {
  int l = (int)sqrt((double)idx);
  while (l * l > idx) --l;
  while ((l + 1) * (l + 1) <= idx) ++l;
  return l;
}

// exact float64 -> fp32 rounding by integer operations (fp32 copies only)
__device__ __forceinline__ float to_f32(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned int hi = (unsigned int)(u >> 32);
  const int e32 = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
  if (e32 <= 0 || e32 >= 255) return (u << 1) == 0ull ? __uint_as_float(hi & 0x80000000u) : (float)x;
  const unsigned long long man = u & 0xFFFFFFFFFFFFFull;
  const unsigned int m23 = (unsigned int)(man >> 29), rem = (unsigned int)(man & 0x1FFFFFFFull);
  const unsigned int up = (rem > 0x10000000u || (rem == 0x10000000u && (m23 & 1u))) ? 1u : 0u;
  return __uint_as_float((hi & 0x80000000u) | (((unsigned int)e32 << 23) + m23 + up));
}

struct ScanGeom {
  int n_r, lmax, n_lm, nc, ch, wpp;   // chunks, chunk length, warps per patch and chunk
};

__device__ __forceinline__ bool scan_lane(const ScanGeom &s, int &p, int &idx, int &c, int &n0, int &n1) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= 2 * s.wpp * s.nc) return false;
  c = w % s.nc;
  const int rest = w / s.nc;
  p = rest / s.wpp;
  idx = (rest % s.wpp) * 32 + lane;
  n0 = c * s.ch;
  n1 = min(s.n_r, n0 + s.ch);
  return idx < s.n_lm;
}

__global__ void __launch_bounds__(128)
k_scan_maps(ScanGeom s, const double *__restrict__ A, const double *__restrict__ coef, double4 *__restrict__ maps) {
  int p, idx, c, n0, n1;
  if (!scan_lane(s, p, idx, c, n0, n1)) return;
  const int l = mode_degree(idx);
  const int L1 = s.lmax + 1;
  const double *Ap = A + (size_t)p * s.n_r * s.n_lm + idx;
  double ai = 1.0, bi = 0.0, ao = 1.0, bo = 0.0;
  for (int n = n0; n < n1; ++n) {
    const double *k = coef + ((size_t)n * L1 + l) * 8;
    bi = fma(k[0], bi, k[1] * Ap[(size_t)n * s.n_lm]);
    ai *= k[0];
  }
  for (int n = n1 - 1; n >= n0; --n) {
    const double *k = coef + ((size_t)n * L1 + l) * 8;
    const double an = (n + 1 < s.n_r) ? Ap[(size_t)(n + 1) * s.n_lm] : 0.0;
    bo = fma(k[2], bo, k[3] * an);
    ao *= k[2];
  }
  maps[((size_t)p * s.nc + c) * s.n_lm + idx] = make_double4(ai, bi, ao, bo);
}

__global__ void __launch_bounds__(128)
k_scan_apply(ScanGeom s, const double *__restrict__ A, const double *__restrict__ coef,
             const double4 *__restrict__ maps, double *__restrict__ cin, double *__restrict__ Q,
             float *__restrict__ Q32) {
  int p, idx, c, n0, n1;
  if (!scan_lane(s, p, idx, c, n0, n1)) return;
  const int l = mode_degree(idx);
  const int L1 = s.lmax + 1;
  const double4 *mp = maps + (size_t)p * s.nc * s.n_lm + idx;
  double x = 0.0;                       // c_{n0 - 1}
  for (int k = 0; k < c; ++k) {
    const double4 m = mp[(size_t)k * s.n_lm];
    x = fma(m.x, x, m.y);
  }
  double y = 0.0;                       // d_{n1 - 1} comes from the chunks above
  for (int k = s.nc - 1; k > c; --k) {
    const double4 m = mp[(size_t)k * s.n_lm];
    y = fma(m.z, y, m.w);
  }
  const double *Ap = A + (size_t)p * s.n_r * s.n_lm + idx;
  double *Cp = cin + (size_t)p * s.n_r * s.n_lm + idx;
  for (int n = n0; n < n1; ++n) {
    const double *k = coef + ((size_t)n * L1 + l) * 8;
    x = fma(k[0], x, k[1] * Ap[(size_t)n * s.n_lm]);
    Cp[(size_t)n * s.n_lm] = x;
  }
  const size_t qsz = (size_t)2 * s.n_r * s.n_lm;
  for (int n = n1 - 1; n >= n0; --n) {
    const double *k = coef + ((size_t)n * L1 + l) * 8;
    const double an = (n + 1 < s.n_r) ? Ap[(size_t)(n + 1) * s.n_lm] : 0.0;
    y = fma(k[2], y, k[3] * an);
    const double cn = Cp[(size_t)n * s.n_lm];
    const double sum = cn + y;
    const double q = k[4] * sum;
    const double qr = fma(k[5], cn, k[6] * y);
    const double qt = k[7] * sum;
    const size_t o = (size_t)(p * s.n_r + n) * s.n_lm + idx;
    Q[o] = q;
    Q[qsz + o] = qr;
    Q[2 * qsz + o] = qt;
    if (Q32 != nullptr) {
      Q32[o] = to_f32(q);
      Q32[qsz + o] = to_f32(qr);
      Q32[2 * qsz + o] = to_f32(qt);
    }
  }
}

// Combination of the two patches' moments (§4: the potential of a patch is the
// sum of the potentials of both patches' moments, each taken in the target
// patch's angles).  Y_i(M v) = sum_j D^l_ij Y_j(v) turns the other patch's
// moments into own-frame ones of the same degree:
//   Atot[p][n][j] = A[p][n][j] + sum_i D^l_ij A[1-p][n][i],  i, j of degree l.
// The scans and the synthesis are linear and act on each degree alone, so this
// gives the same potential as summing four separate ones.  One block per
// radius; T is the type of the products (float64, or float32 with a float64
// sum onto the own-patch moment).
template <typename T>
__global__ void __launch_bounds__(256)
k_rotate_moments(int n_r, int n_lm, const T *__restrict__ rot, const double *__restrict__ A,
                 double *__restrict__ Atot) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T *a = reinterpret_cast<T *>(smraw);   // [2][n_lm]
  const int n = blockIdx.x;
  for (int e = threadIdx.x; e < 2 * n_lm; e += blockDim.x) {
    const int p = e / n_lm, j = e % n_lm;
    a[e] = (T)A[((size_t)p * n_r + n) * n_lm + j];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 2 * n_lm; e += blockDim.x) {
    const int p = e / n_lm, j = e % n_lm;
    const int l = mode_degree(j);
    const int w = 2 * l + 1, jj = j - l * l;
    const T *D = rot + (size_t)l * (4 * l * l - 1) / 3 + jj;
    const T *x = a + (1 - p) * n_lm + l * l;
    T acc = 0;
    for (int i = 0; i < w; ++i) acc = fma(D[(size_t)i * w], x[i], acc);
    const size_t o = ((size_t)p * n_r + n) * n_lm + j;
    Atot[o] = A[o] + (double)acc;
  }
}

}  // namespace

cudaError_t rotate_moments(yy_grid *g, bool fp64, cudaStream_t st) {
  const size_t smem = 2 * (size_t)g->n_lm * (fp64 ? sizeof(double) : sizeof(float));
  if (smem > 48 * 1024) {
    const cudaError_t e = fp64 ? cudaFuncSetAttribute(k_rotate_moments<double>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                               : cudaFuncSetAttribute(k_rotate_moments<float>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (fp64)
    k_rotate_moments<double><<<g->n_r, 256, smem, st>>>(g->n_r, g->n_lm, g->rot, g->A, g->Atot);
  else
    k_rotate_moments<float><<<g->n_r, 256, smem, st>>>(g->n_r, g->n_lm, g->rot32, g->A, g->Atot);
  g->launches++;
  return cudaGetLastError();
}

void scan_geometry(const yy_grid *g, int *nc, int *ch) {
  const int wpp = (g->n_lm + 31) / 32;
  int n = (4 * 152 + 2 * wpp - 1) / (2 * wpp);   // about four warps per SM
  n = n < 1 ? 1 : (n > g->n_r ? g->n_r : n);
  *ch = (g->n_r + n - 1) / n;
  *nc = (g->n_r + *ch - 1) / *ch;
}

cudaError_t radial_scan(yy_grid *g, bool want_f32, cudaStream_t st) {
  ScanGeom s;
  s.n_r = g->n_r;
  s.lmax = g->lmax;
  s.n_lm = g->n_lm;
  s.wpp = (g->n_lm + 31) / 32;
  scan_geometry(g, &s.nc, &s.ch);
  const int warps = 2 * s.wpp * s.nc;
  const int blocks = (warps * 32 + 127) / 128;
  k_scan_maps<<<blocks, 128, 0, st>>>(s, g->Atot, g->scan, (double4 *)g->scan_maps);
  g->launches++;
  k_scan_apply<<<blocks, 128, 0, st>>>(s, g->Atot, g->scan, (const double4 *)g->scan_maps, g->cin, g->Q,
                                       want_f32 ? g->Q32 : nullptr);
  g->launches++;
  return cudaGetLastError();
}

}  // namespace yy
