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
#include <algorithm>

#include "yy_internal.h"

namespace yy {
namespace {

__device__ __forceinline__ int mode_degree(int idx) {
  int l = (int)sqrtf((float)idx);   // corrected below; exact for idx < 2^24
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

// exact float32 -> float64 widening by integer operations
__device__ __forceinline__ double to_f64(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int ex = (u >> 23) & 0xFFu;
  if (ex == 0u || ex == 255u) {
    if ((u << 1) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
    return (double)f;
  }
  const unsigned int hi = (u & 0x80000000u) | ((ex + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}

struct __align__(32) Map4 {
  double a_in, b_in, a_out, b_out;   // inner c -> a_in c + b_in, outer d -> a_out d + b_out
};

struct ScanGeom {
  int n_r, lmax, n_lm, nc, ch, wpp;   // chunks, chunk length, warps per patch and chunk
  int n_patch;
};

__device__ __forceinline__ bool scan_lane(const ScanGeom &s, int &p, int &idx, int &c, int &n0, int &n1) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= s.n_patch * s.wpp * s.nc) return false;
  c = w % s.nc;
  const int rest = w / s.nc;
  p = rest / s.wpp;
  idx = (rest % s.wpp) * 32 + lane;
  n0 = c * s.ch;
  n1 = min(s.n_r, n0 + s.ch);
  return idx < s.n_lm;
}

__global__ void __launch_bounds__(128)
k_scan_maps(ScanGeom s, const double *__restrict__ A, const double *__restrict__ coef, Map4 *__restrict__ maps) {
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
  maps[((size_t)p * s.nc + c) * s.n_lm + idx] = Map4{ai, bi, ao, bo};
}

__global__ void __launch_bounds__(128)
k_scan_apply(ScanGeom s, const double *__restrict__ A, const double *__restrict__ coef,
             const Map4 *__restrict__ maps, double *__restrict__ cin, double *__restrict__ Q,
             float *__restrict__ Q32) {
  int p, idx, c, n0, n1;
  if (!scan_lane(s, p, idx, c, n0, n1)) return;
  const int l = mode_degree(idx);
  const int L1 = s.lmax + 1;
  const Map4 *mp = maps + (size_t)p * s.nc * s.n_lm + idx;
  double x = 0.0;                       // c_{n0 - 1}
  for (int k = 0; k < c; ++k) {
    const Map4 m = mp[(size_t)k * s.n_lm];
    x = fma(m.a_in, x, m.b_in);
  }
  double y = 0.0;                       // d_{n1 - 1} comes from the chunks above
  for (int k = s.nc - 1; k > c; --k) {
    const Map4 m = mp[(size_t)k * s.n_lm];
    y = fma(m.a_out, y, m.b_out);
  }
  const double *Ap = A + (size_t)p * s.n_r * s.n_lm + idx;
  double *Cp = cin + (size_t)p * s.n_r * s.n_lm + idx;
  for (int n = n0; n < n1; ++n) {
    const double *k = coef + ((size_t)n * L1 + l) * 8;
    x = fma(k[0], x, k[1] * Ap[(size_t)n * s.n_lm]);
    Cp[(size_t)n * s.n_lm] = x;
  }
  const size_t qsz = (size_t)s.n_patch * s.n_r * s.n_lm;
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
// gives the same potential as summing four separate ones.  Blocks of 256
// threads: blockIdx.x is the radius, blockIdx.y a group of 256 modes, one
// thread per mode j, both patches at once (each D entry is loaded once for
// the two sums); every block stages both rows.  Small blocks keep several
// resident per SM.  T is the type of the products: float64, or float32 (the
// moments rounded once, the sum added to the float64 own moment).
template <typename T>
__global__ void __launch_bounds__(256)
k_rotate_moments(int n_r, int n_lm, const T *__restrict__ rot, const double *__restrict__ A,
                 double *__restrict__ Atot) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T *a = reinterpret_cast<T *>(smraw);   // [2][n_lm]
  const int n = blockIdx.x;
  const double *A0 = A + (size_t)n * n_lm, *A1 = A + ((size_t)n_r + n) * n_lm;
  for (int j = threadIdx.x; j < n_lm; j += blockDim.x) {
    if constexpr (sizeof(T) == 4) {
      a[j] = to_f32(A0[j]);
      a[n_lm + j] = to_f32(A1[j]);
    } else {
      a[j] = A0[j];
      a[n_lm + j] = A1[j];
    }
  }
  __syncthreads();
  const int j = (int)(blockIdx.y * blockDim.x + threadIdx.x);
  if (j < n_lm) {
    const int l = mode_degree(j);
    const int w = 2 * l + 1, jj = j - l * l;
    const T *D = rot + (size_t)l * (4 * l * l - 1) / 3 + jj;
    const T *x0 = a + l * l, *x1 = a + n_lm + l * l;
    T s0 = 0, s1 = 0;   // into patch 0 (from patch 1) and into patch 1 (from patch 0)
    rot_class_dot(D, w, jj, x0, x1, s0, s1);
    double r0, r1;
    if constexpr (sizeof(T) == 4) {
      r0 = to_f64(s0);
      r1 = to_f64(s1);
    } else {
      r0 = s0;
      r1 = s1;
    }
    Atot[(size_t)n * n_lm + j] = A0[j] + r0;
    Atot[((size_t)n_r + n) * n_lm + j] = A1[j] + r1;
  }
}

// Radial scans with one warp per (patch, mode): lane L owns the radii
// [L ch, L ch + ch), ch = ceil(n_r / 32) <= CH, and keeps its moments and inner
// sums in registers.  Each recurrence is folded into one affine map per lane,
// the maps are composed across the warp by shuffles (prefix for the inner
// sums, suffix for the outer ones), and each lane then replays its radii from
// the composed start value.  Steps past n_r use the identity map, and every
// load is unconditional (clamped index) so that no load waits behind the
// float64 chain.  F64OUT: output factors applied in float64; otherwise (the
// reduced-precision paths, whose packing rounds Q to fp32 anyway) in fp32
// from fp32 roundings of c_n and d_n, widened back exactly.
template <int CH, bool F64OUT>
__device__ __forceinline__ void scan_warp_body(int w, int n_patch, int n_r, int lmax, int n_lm,
                                               const double *__restrict__ A, const double *__restrict__ coef,
                                               double *__restrict__ Q, float *__restrict__ Q32) {
  const int lane = threadIdx.x & 31;
  if (w >= n_patch * n_lm) return;
  const int p = w / n_lm, j = w % n_lm;
  const int l = mode_degree(j);
  const int L1 = lmax + 1;
  const int ch = (n_r + 31) / 32;
  const int n0 = lane * ch;
  const double *Ap = A + (size_t)p * n_r * n_lm + j;
  const double *cl = coef + (size_t)l * 8;          // + n L1 8
  const size_t cstride = (size_t)L1 * 8;
  double av[CH], cv[CH];
#pragma unroll
  for (int i = 0; i < CH; ++i) {
    const int n = min(n0 + i, n_r - 1);
    const double v = Ap[(size_t)n * n_lm];
    av[i] = (i < ch && n0 + i < n_r) ? v : 0.0;
  }
  // A_{n0 + ch}: first moment of the next lane's radii
  double a_next = __shfl_down_sync(0xffffffffu, av[0], 1);
  if (lane == 31) a_next = 0.0;

  // inner sums c_n = a_n c_{n-1} + b_n A_n
  double al = 1.0, be = 0.0;
#pragma unroll
  for (int i = 0; i < CH; ++i) {
    const bool ok = i < ch && n0 + i < n_r;
    const double2 k01 = *(const double2 *)(cl + (size_t)min(n0 + i, n_r - 1) * cstride);
    const double a = ok ? k01.x : 1.0, b = ok ? k01.y : 0.0;
    be = fma(a, be, b * av[i]);
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
#pragma unroll
  for (int i = 0; i < CH; ++i) {
    const bool ok = i < ch && n0 + i < n_r;
    const double2 k01 = *(const double2 *)(cl + (size_t)min(n0 + i, n_r - 1) * cstride);
    const double a = ok ? k01.x : 1.0, b = ok ? k01.y : 0.0;
    x = fma(a, x, b * av[i]);
    cv[i] = x;
  }

  // outer sums d_n = e_n d_{n+1} + f_n A_{n+1}, d_{n_r - 1} = 0
  al = 1.0;
  be = 0.0;
#pragma unroll
  for (int i = CH - 1; i >= 0; --i) {
    const bool ok = i < ch && n0 + i < n_r;
    const double an = (i + 1 < ch) ? av[i + 1 < CH ? i + 1 : i] : a_next;   // 0 past n_r
    const double2 k23 = *(const double2 *)(cl + (size_t)min(n0 + i, n_r - 1) * cstride + 2);
    const double e = ok ? k23.x : 1.0, f = ok ? k23.y : 0.0;
    be = fma(e, be, f * an);
    al *= e;
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
  const size_t qsz = (size_t)n_patch * n_r * n_lm;
#pragma unroll
  for (int i = CH - 1; i >= 0; --i) {
    const bool ok = i < ch && n0 + i < n_r;
    const double an = (i + 1 < ch) ? av[i + 1 < CH ? i + 1 : i] : a_next;
    const double *k = cl + (size_t)min(n0 + i, n_r - 1) * cstride;
    const double2 k23 = *(const double2 *)(k + 2);
    const double e = ok ? k23.x : 1.0, f = ok ? k23.y : 0.0;
    y = fma(e, y, f * an);
    if (!ok) continue;
    const size_t o = ((size_t)p * n_r + n0 + i) * n_lm + j;
    const double cn = cv[i];
    if constexpr (F64OUT) {
      const double2 k45 = *(const double2 *)(k + 4);
      const double2 k67 = *(const double2 *)(k + 6);
      const double sum = cn + y;
      const double q = k45.x * sum, qr = fma(k45.y, cn, k67.x * y), qt = k67.y * sum;
      Q[o] = q;
      Q[qsz + o] = qr;
      Q[2 * qsz + o] = qt;
      if (Q32 != nullptr) {
        Q32[o] = to_f32(q);
        Q32[qsz + o] = to_f32(qr);
        Q32[2 * qsz + o] = to_f32(qt);
      }
    } else {
      const double2 k45 = *(const double2 *)(k + 4);
      const double2 k67 = *(const double2 *)(k + 6);
      const float cf = to_f32(cn), yf = to_f32(y);
      const float sum = cf + yf;
      Q[o] = to_f64(to_f32(k45.x) * sum);
      Q[qsz + o] = to_f64(fmaf(to_f32(k45.y), cf, to_f32(k67.x) * yf));
      Q[2 * qsz + o] = to_f64(to_f32(k67.y) * sum);
    }
  }
}

template <int CH, bool F64OUT>
__global__ void __launch_bounds__(128, 3)
k_scan_warp(int n_patch, int n_r, int lmax, int n_lm, const double *__restrict__ A, const double *__restrict__ coef,
            double *__restrict__ Q, float *__restrict__ Q32) {
  scan_warp_body<CH, F64OUT>((int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), n_patch, n_r, lmax, n_lm, A, coef,
                             Q, Q32);
}

// Many fields' scans in one launch: block b scans for field block_map[b] >> 24
// (its block block_map[b] & 0xFFFFFF, four (patch, mode) warps each), in the
// register form the field's radial grid needs (ch = 8, 12, 18 or 24 radii per lane).
template <bool F64OUT>
__global__ void __launch_bounds__(128, 3)
k_scan_group(const ScanGroupField *__restrict__ fields, const uint32_t *__restrict__ block_map) {
  const uint32_t m = block_map[blockIdx.x];
  const ScanGroupField f = fields[m >> 24];
  const int w = (int)(m & 0xFFFFFFu) * 4 + (int)(threadIdx.x >> 5);
  switch (f.ch) {
    case 8: scan_warp_body<8, F64OUT>(w, f.n_patch, f.n_r, f.lmax, f.n_lm, f.A, f.coef, f.Q, f.Q32); break;
    case 12: scan_warp_body<12, F64OUT>(w, f.n_patch, f.n_r, f.lmax, f.n_lm, f.A, f.coef, f.Q, f.Q32); break;
    case 18: scan_warp_body<18, F64OUT>(w, f.n_patch, f.n_r, f.lmax, f.n_lm, f.A, f.coef, f.Q, f.Q32); break;
    default: scan_warp_body<24, F64OUT>(w, f.n_patch, f.n_r, f.lmax, f.n_lm, f.A, f.coef, f.Q, f.Q32); break;
  }
}

}  // namespace

bool scan_group_field(yy_grid *g, bool want_f32, ScanGroupField *f) {
  if (g->n_r > 32 * 24) return false;
  f->n_patch = g->n_patch;
  f->n_r = g->n_r;
  f->lmax = g->lmax;
  f->n_lm = g->n_lm;
  f->ch = g->n_r <= 32 * 8 ? 8 : g->n_r <= 32 * 12 ? 12 : g->n_r <= 32 * 18 ? 18 : 24;
  f->A = moments_total(g);
  f->coef = g->scan;
  f->Q = g->Q;
  f->Q32 = want_f32 ? g->Q32 : nullptr;
  return true;
}

int scan_group_blocks(const ScanGroupField &f) { return (f.n_patch * f.n_lm + 3) / 4; }

cudaError_t scan_group_launch(const ScanGroupField *fields, const uint32_t *block_map, int blocks, bool f64_out,
                              cudaStream_t st) {
  if (f64_out)
    k_scan_group<true><<<blocks, 128, 0, st>>>(fields, block_map);
  else
    k_scan_group<false><<<blocks, 128, 0, st>>>(fields, block_map);
  return cudaGetLastError();
}

cudaError_t rotate_moments(yy_grid *g, bool fp64, cudaStream_t st) {
  if (g->n_patch == 1) return cudaSuccess;   // polar grid: the scans read A itself
  const size_t smem = 2 * (size_t)g->n_lm * (fp64 ? sizeof(double) : sizeof(float));
  if (smem > 48 * 1024) {
    // the attribute belongs to the kernel, shared by all grids: the maximum
    const cudaError_t e = fp64 ? cudaFuncSetAttribute(k_rotate_moments<double>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024)
                               : cudaFuncSetAttribute(k_rotate_moments<float>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
  }
  const dim3 grid((unsigned)g->n_r, (unsigned)((g->n_lm + 255) / 256));
  if (fp64)
    k_rotate_moments<double><<<grid, 256, smem, st>>>(g->n_r, g->n_lm, g->rot, g->A, g->Atot);
  else
    k_rotate_moments<float><<<grid, 256, smem, st>>>(g->n_r, g->n_lm, g->rot32, g->A, g->Atot);
  note_launch(g, "k_rotate_moments", st);
  return cudaGetLastError();
}

void scan_geometry(const yy_grid *g, int *nc, int *ch) {
  const int wpp = (g->n_lm + 31) / 32;
  int n = (4 * 152 + 2 * wpp - 1) / (2 * wpp);   // about four warps per SM
  n = n < 1 ? 1 : (n > g->n_r ? g->n_r : n);
  *ch = (g->n_r + n - 1) / n;
  *nc = (g->n_r + *ch - 1) / *ch;
}

cudaError_t radial_scan(yy_grid *g, bool want_f32, bool f64_out, cudaStream_t st) {
  float *q32 = want_f32 ? g->Q32 : nullptr;
  // one warp per block: the SMs get the warps in equal numbers (with four per
  // block, 1352 warps left some SMs three blocks and most two, and the
  // three-block SMs set the time)
  const unsigned wblocks = (unsigned)(g->n_patch * g->n_lm);
  const double *At = moments_total(g);
  if (g->n_r <= 32 * 24) {
#define YY_SCAN_WARP(CH)                                                                               \
  (f64_out ? (k_scan_warp<CH, true><<<wblocks, 32, 0, st>>>(g->n_patch, g->n_r, g->lmax, g->n_lm, At, g->scan, g->Q, q32), 0) \
           : (k_scan_warp<CH, false><<<wblocks, 32, 0, st>>>(g->n_patch, g->n_r, g->lmax, g->n_lm, At, g->scan, g->Q, q32), 0))
    if (g->n_r <= 32 * 8)
      YY_SCAN_WARP(8);
    else if (g->n_r <= 32 * 12)
      YY_SCAN_WARP(12);
    else if (g->n_r <= 32 * 18)
      YY_SCAN_WARP(18);
    else
      YY_SCAN_WARP(24);
#undef YY_SCAN_WARP
    note_launch(g, "k_scan_warp", st);
    return cudaGetLastError();
  }
  // long radial grids: chunks spread over warps, two passes
  ScanGeom s;
  s.n_r = g->n_r;
  s.lmax = g->lmax;
  s.n_lm = g->n_lm;
  s.wpp = (g->n_lm + 31) / 32;
  s.n_patch = g->n_patch;
  scan_geometry(g, &s.nc, &s.ch);
  const int warps = s.n_patch * s.wpp * s.nc;
  const int blocks = (warps * 32 + 127) / 128;
  k_scan_maps<<<blocks, 128, 0, st>>>(s, At, g->scan, (Map4 *)g->scan_maps);
  note_launch(g, "k_scan_maps", st);
  k_scan_apply<<<blocks, 128, 0, st>>>(s, At, g->scan, (const Map4 *)g->scan_maps, g->cin, g->Q,
                                       want_f32 ? g->Q32 : nullptr);
  note_launch(g, "k_scan_apply", st);
  return cudaGetLastError();
}

}  // namespace yy
