// Separable analysis (§3 Eqs. ac/as with the §4 weights):
//
//   A_p[i][lm] = sum_j K_lm T_j^(lm) sum_k rho_p[i][j][k] w_jk {C_k^(m) | S_k^(m)}
//
// The weight w_jk is not a product of a theta and a phi factor (it follows the
// overlap boundary), so it is folded into the density first; the remaining
// double sum factors into an azimuthal stage and a polar stage:
//
//   phi stage    F[p,i][j][t] = sum_k (rho w)_ijk az[t][k],
//                az[0] = d_phi (m = 0), az[2m-1] = C_k^(m), az[2m] = S_k^(m)
//   theta stage  A[p,i][l^2 + t] = sum_j (K_lm T_j^(lm)) F[p,i][j][t]
//
// which costs 2 N_ang (2 l_max + 1) + 2 n_theta n_lm flops per shell instead of
// 2 N_ang n_lm for the dense contraction (12.6 times fewer at the 1-degree grid
// with l_max = 25).  T = double computes everything in float64.  T = float
// computes the azimuthal stage in fp32 on CUDA cores (it is bound by reading
// the density), except that the m = 0 sums, which carry the monopole and so
// dominate Phi, are compensated fp32 pairs in the azimuthal stage and float64
// in the polar stage.
#include <math.h>

#include <algorithm>

#include "yy_internal.h"

namespace yy {
namespace {

// exact float64 -> fp32 rounding by integer operations (round to nearest even)
__device__ __forceinline__ float narrow(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned int hi = (unsigned int)(u >> 32);
  const int e32 = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
  if (e32 <= 0 || e32 >= 255) return (u << 1) == 0ull ? __uint_as_float(hi & 0x80000000u) : (float)x;
  const unsigned long long man = u & 0xFFFFFFFFFFFFFull;
  const unsigned int m23 = (unsigned int)(man >> 29), rem = (unsigned int)(man & 0x1FFFFFFFull);
  const unsigned int up = (rem > 0x10000000u || (rem == 0x10000000u && (m23 & 1u))) ? 1u : 0u;
  return __uint_as_float((hi & 0x80000000u) | (((unsigned int)e32 << 23) + m23 + up));
}

// exact fp32 -> float64 widening by integer operations
__device__ __forceinline__ double widen(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int ex = (u >> 23) & 0xFFu;
  if (ex == 0u || ex == 255u) {
    if ((u << 1) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
    return (double)f;
  }
  const unsigned int hi = (u & 0x80000000u) | ((ex + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}

template <typename T>
__device__ __forceinline__ T to_t(double x) {
  if constexpr (sizeof(T) == 4)
    return narrow(x);
  else
    return x;
}

// Knuth's two-sum into an unevaluated fp32 pair (h, l)
__device__ __forceinline__ void pair_add(float &h, float &l, float b) {
  const float s = h + b;
  const float bb = s - h;
  l += (h - (s - bb)) + (b - bb);
  h = s;
}

__device__ __forceinline__ int degree_of(int idx) {
  int l = (int)sqrtf((float)idx);   // corrected below; exact for idx < 2^24
  while (l * l > idx) --l;
  while ((l + 1) * (l + 1) <= idx) ++l;
  return l;
}

// az[k][t] (t fastest, padded to nt_pad): the azimuthal cell integrals
__global__ void k_az_table(int n_phi, int lmax, int nt_pad, double ph0, double dph, double *__restrict__ az) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_phi * nt_pad) return;
  const int k = e / nt_pad, t = e % nt_pad;
  double v = 0.0;
  if (t == 0) {
    v = dph;
  } else if (t <= 2 * lmax) {
    const int m = (t + 1) / 2;
    const double phc = ph0 + dph * (k + 0.5);
    const double half = 2.0 * sin(0.5 * m * dph) / m;   // closed forms of C_k^(m), S_k^(m) (§2)
    v = (t & 1) ? cos(m * phc) * half : sin(m * phc) * half;
  }
  az[e] = v;
}

// tb0[j][l] = K_l0 T_j^(l0) d_phi as an unevaluated fp32 pair (hi, lo)
__global__ void k_tb0(int n_theta, int lmax, int n_lm, double dph, const double *__restrict__ tbar,
                      float2 *__restrict__ tb0) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_theta * (lmax + 1)) return;
  const int j = e / (lmax + 1), l = e % (lmax + 1);
  const double v = tbar[(size_t)j * n_lm + l * l] * dph;
  const float hi = (float)v;
  tb0[e] = make_float2(hi, (float)(v - (double)hi));
}

__global__ void k_round(size_t n, const double *__restrict__ src, float *__restrict__ dst) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) dst[e] = (float)src[e];
}

constexpr int kJC = 48;    // rows j per work item (kJCSmall where the table leaves too little room)
constexpr int kJCSmall = 16;
constexpr int kTJ = 4;     // rows per thread
constexpr int kTT = 4;     // azimuthal functions per thread
__host__ __device__ constexpr int xpad(int jc) { return jc + 4; }   // padded row stride of the staged densities

// four consecutive values, 16-byte aligned
__device__ __forceinline__ void ld4(const float *p, float (&o)[4]) {
  const float4 v = *reinterpret_cast<const float4 *>(p);
  o[0] = v.x;
  o[1] = v.y;
  o[2] = v.z;
  o[3] = v.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&o)[4]) {
  const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
  o[0] = a.x;
  o[1] = a.y;
  o[2] = b.x;
  o[3] = b.y;
}
__device__ __forceinline__ void st4(float *p, const float (&v)[4]) {
  *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double *p, const double (&v)[4]) {
  reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}

// exact product a b = p + e (fma-based) and an unevaluated-pair dot step
__device__ __forceinline__ void pair_fma(float &h, float &l, float ah, float al, float bh, float bl) {
  const float p = ah * bh;
  const float e = fmaf(ah, bh, -p);
  pair_add(h, l, p);
  l += e + fmaf(ah, bl, al * bh);
}

// Azimuthal stage, persistent: each block keeps the table az in shared
// memory and takes work items (shell, chunk of JC rows j) in turn.
//  1. all threads stage the chunk (JC n_phi consecutive densities) with 16
//     independent loads in flight each, fold in w and store it transposed;
//  2. (fp32) one warp per row forms the row's compensated sum (the m = 0
//     azimuthal sum without the factor d_phi) as an unevaluated fp32 pair;
//  3. each thread accumulates a tile of kTJ rows x kTT functions over all k
//     with two vector shared-memory loads per 16 products.
template <typename T, int JC>
__global__ void k_sep_phi(int n_shells, int n_r, int n_theta, int n_phi, int nt_pad, const double *__restrict__ rho0,
                          const double *__restrict__ rho1, const T *__restrict__ w, const T *__restrict__ az,
                          T *__restrict__ F, float2 *__restrict__ F0) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T *as = reinterpret_cast<T *>(smraw);                  // [n_phi][nt_pad]
  constexpr int XP = xpad(JC);
  T *xs = as + (size_t)n_phi * nt_pad;                   // [n_phi][XP]
  const int tg = nt_pad / kTT;
  const int tt = threadIdx.x % tg, tj = threadIdx.x / tg;   // function group, row group
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
  const size_t n_ang = (size_t)n_theta * n_phi;
  const int chunks = (n_theta + JC - 1) / JC;
  const int items = n_shells * chunks;
  constexpr int kU = 16;
  const float inv_phi = 1.0f / (float)n_phi;

  for (int e = threadIdx.x; e < n_phi * nt_pad; e += blockDim.x) as[e] = az[e];

  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int shell = item / chunks, j0 = (item % chunks) * JC;
    const int p = shell / n_r, i = shell % n_r;
    const int rows = min(JC, n_theta - j0);
    const int count = rows * n_phi;                      // consecutive values of the chunk
    const double *src = (p == 0 ? rho0 : rho1) + (size_t)i * n_ang + (size_t)j0 * n_phi;
    const T *wsrc = w + (size_t)j0 * n_phi;
    __syncthreads();   // the previous item's tiles are done with xs (and as is written)
    for (int e0 = threadIdx.x; e0 < JC * n_phi; e0 += kU * blockDim.x) {
      double rv[kU];
      T wv[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int e = e0 + u * blockDim.x;
        rv[u] = (e < count) ? src[e] : 0.0;
        wv[u] = (e < count) ? wsrc[e] : T(0);
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < JC * n_phi) {
          // e = jj n_phi + k: quotient from the float reciprocal, then corrected
          int jj = (int)((float)e * inv_phi);
          int k = e - jj * n_phi;
          if (k < 0) {
            --jj;
            k += n_phi;
          } else if (k >= n_phi) {
            ++jj;
            k -= n_phi;
          }
          xs[(size_t)k * XP + jj] = to_t<T>(rv[u]) * wv[u];
        }
      }
    }
    __syncthreads();
    if constexpr (sizeof(T) == 4) {
      for (int jj = warp; jj < rows; jj += n_warps) {
        float h = 0.0f, l = 0.0f;
        for (int k = lane; k < n_phi; k += 32) pair_add(h, l, xs[(size_t)k * XP + jj]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          const float oh = __shfl_xor_sync(0xffffffffu, h, off);
          const float ol = __shfl_xor_sync(0xffffffffu, l, off);
          pair_add(h, l, oh);
          l += ol;
        }
        if (lane == 0) F0[(size_t)shell * n_theta + j0 + jj] = make_float2(h, l);
      }
    }
    if (tj < JC / kTJ) {
      T acc[kTJ][kTT];
#pragma unroll
      for (int a = 0; a < kTJ; ++a)
#pragma unroll
        for (int b = 0; b < kTT; ++b) acc[a][b] = T(0);
#pragma unroll 2
      for (int k = 0; k < n_phi; ++k) {
        T x4[4], a4[4];
        ld4(xs + (size_t)k * XP + tj * kTJ, x4);
        ld4(as + (size_t)k * nt_pad + tt * kTT, a4);
#pragma unroll
        for (int a = 0; a < kTJ; ++a)
#pragma unroll
          for (int b = 0; b < kTT; ++b) acc[a][b] = fma(x4[a], a4[b], acc[a][b]);
      }
#pragma unroll
      for (int a = 0; a < kTJ; ++a) {
        const int j = j0 + tj * kTJ + a;
        if (j >= n_theta) continue;
        st4(F + ((size_t)shell * n_theta + j) * nt_pad + tt * kTT, acc[a]);
      }
    }
  }
}

// The fp32 polar stage on one shell: F (shared memory, [n_theta][nt_pad]) and
// the pair row sums f0s; the m = 0 modes as an unevaluated-pair dot product,
// the others as fp32 dot products over j.
__device__ void theta_modes_f32(int n_theta, int n_lm, int lmax1, int nt_pad, const float *__restrict__ tb,
                                const float2 *__restrict__ tb0, const float *fs, const float2 *f0s,
                                double *__restrict__ Arow) {
  if (threadIdx.x < 32) {
    for (int l = threadIdx.x; l < lmax1; l += 32) {
      float h = 0.0f, lo = 0.0f;
      for (int j = 0; j < n_theta; ++j) {
        const float2 a = tb0[(size_t)j * lmax1 + l], b = f0s[j];
        pair_fma(h, lo, a.x, a.y, b.x, b.y);
      }
      Arow[l * l] = widen(h) + widen(lo);
    }
  }
  for (int idx = threadIdx.x; idx < n_lm; idx += blockDim.x) {
    const int l = degree_of(idx);
    const int t = idx - l * l;
    if (t == 0) continue;
    float s = 0.0f;
#pragma unroll 8
    for (int j = 0; j < n_theta; ++j) s = fmaf(tb[(size_t)j * n_lm + idx], fs[j * nt_pad + t], s);
    Arow[idx] = widen(s);
  }
}

// Polar stage: one block per shell, the shell's F staged in shared memory, one
// thread per mode.  The m = 0 modes (fp32 form): an unevaluated-pair dot
// product of the pair-split table (with d_phi folded in) and the pair row
// sums, then one float64 addition; float64 for the float64 form.
template <typename T>
__global__ void __launch_bounds__(256) k_sep_theta(int n_theta, int n_lm, int lmax1, int nt_pad,
                                                   const T *__restrict__ tb, const float2 *__restrict__ tb0,
                                                   const T *__restrict__ F, const float2 *__restrict__ F0,
                                                   double *__restrict__ A) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int shell = blockIdx.x;
  const T *Fs = F + (size_t)shell * n_theta * nt_pad;
  if constexpr (sizeof(T) == 4) {
    float2 *f0s = reinterpret_cast<float2 *>(smraw);       // [n_theta]
    T *fs = reinterpret_cast<T *>(f0s + n_theta + (n_theta & 1));   // [n_theta][nt_pad]
    for (int e = threadIdx.x; e < n_theta * nt_pad; e += blockDim.x) fs[e] = Fs[e];
    for (int j = threadIdx.x; j < n_theta; j += blockDim.x) f0s[j] = F0[(size_t)shell * n_theta + j];
    __syncthreads();
    theta_modes_f32(n_theta, n_lm, lmax1, nt_pad, tb, tb0, fs, f0s, A + (size_t)shell * n_lm);
  } else {
    // The polar cells are symmetric about the equator (cell n_theta - 1 - j is
    // cell j reflected), so the cell integrals of P_l^m(cos theta) sin theta
    // have its parity: T_j' = (-1)^(l + m) T_j.  With S_j = F_j + F_j' and
    // D_j = F_j - F_j', a mode is the sum over j < ceil(n_theta / 2) of T_j S_j
    // (even l + m) or T_j D_j (odd): half the products.  A middle row (odd
    // n_theta) is its own mirror and enters once, as both S and D.
    const int half = (n_theta + 1) >> 1;
    T *cs = reinterpret_cast<T *>(smraw);                  // [2][half][nt_pad]: S, then D
    for (int e = threadIdx.x; e < half * nt_pad; e += blockDim.x) {
      const int j = e / nt_pad, jm = n_theta - 1 - j;
      const T a = Fs[e], b = Fs[(size_t)(jm - j) * nt_pad + e];
      cs[e] = jm == j ? a : a + b;
      cs[(size_t)half * nt_pad + e] = jm == j ? a : a - b;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < n_lm; idx += blockDim.x) {
      const int l = degree_of(idx);
      const int t = idx - l * l;
      const T *c = cs + ((((l + ((t + 1) >> 1)) & 1) != 0) ? (size_t)half * nt_pad : 0) + t;
      T s = T(0);
#pragma unroll 8
      for (int j = 0; j < half; ++j) s = fma(tb[(size_t)j * n_lm + idx], c[j * nt_pad], s);
      A[(size_t)shell * n_lm + idx] = s;
    }
  }
}

// Dynamic shared memory of k_sep_theta: the fp32 form stages F and the m = 0
// pair sums, the float64 form the mirrored sums S and D of ceil(n_theta / 2)
// rows each.
static size_t theta_smem(int n_theta, int nt_pad, size_t el) {
  if (el == sizeof(double)) return (size_t)(n_theta + 1) * nt_pad * sizeof(double);
  return (size_t)n_theta * nt_pad * el + (size_t)(n_theta + 1) * sizeof(float2);
}

// Polar stage after the tensor-core azimuthal stage: F of the rows (shell, j)
// comes from the raw fp32 sums part[t][row] of the centred and scaled rows,
// F = part * row_scale * t_scale + mean * colsum[t] (the centring undone with
// the column sums of the table), and the m = 0 row sums from their float64
// values.  A block takes kThetaShells shells (each table value read serves
// all of them); one measured fastest: with four, 275 blocks of 98 KB left
// most SMs with a single block.
constexpr int kThetaShells = 1;

__global__ void __launch_bounds__(256) k_sep_theta_partials(SepThetaPartials a, int n_shells) {
  constexpr int S = kThetaShells;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2 *f0s = reinterpret_cast<float2 *>(smraw);                          // [S][n_theta]
  float *rsm = reinterpret_cast<float *>(f0s + S * a.n_theta);               // [S][n_theta][2]: scale, mean
  float *fs = rsm + 2 * S * a.n_theta;                                      // [S][n_theta][nt_pad + 1]
  const int fst = a.nt_pad + 1;                                             // odd stride: conflict-free fill
  const int shell0 = blockIdx.x * S;
  const int ns = min(S, n_shells - shell0);
  for (int e = threadIdx.x; e < S * a.n_theta; e += blockDim.x) {
    const int q = e / a.n_theta, j = e - q * a.n_theta;
    float2 f0 = make_float2(0.0f, 0.0f);
    float sc = 0.0f, mn = 0.0f;
    if (q < ns) {
      const size_t row = (size_t)(shell0 + q) * a.n_theta + j;
      const double d = a.F0[row];
      const float hi = narrow(d);
      f0 = make_float2(hi, narrow(d - widen(hi)));
      sc = a.row_scale[row];
      mn = narrow(a.mean[row]);
    }
    f0s[e] = f0;
    rsm[2 * e] = sc;
    rsm[2 * e + 1] = mn;
  }
  __syncthreads();
  const int rows = S * a.n_theta;   // the block's rows are consecutive: (shell0 + q) n_theta + j
  const size_t row0 = (size_t)shell0 * a.n_theta;
  for (int e = threadIdx.x; e < a.nt_pad * rows; e += blockDim.x) {
    const int t = e / rows, qj = e - t * rows;
    float v = 0.0f;
    if (t >= 1 && t < a.nt && qj < ns * a.n_theta)
      v = fmaf(a.part[(size_t)t * a.part_ld + row0 + qj] * rsm[2 * qj], a.t_scale[t], rsm[2 * qj + 1] * a.colsum[t]);
    fs[(size_t)qj * fst + t] = v;
  }
  __syncthreads();
  // m = 0 modes: warp q < S takes shell q, lanes the degrees, compensated
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < ns) {
    for (int l = lane; l < a.lmax1; l += 32) {
      float h = 0.0f, lo = 0.0f;
      for (int j = 0; j < a.n_theta; ++j) {
        const float2 x = a.tb0[(size_t)j * a.lmax1 + l], y = f0s[warp * a.n_theta + j];
        pair_fma(h, lo, x.x, x.y, y.x, y.y);
      }
      a.A[(size_t)(shell0 + warp) * a.n_lm + l * l] = widen(h) + widen(lo);
    }
  }
  // the other modes: fp32 dot products over j, one table read for all S shells
  for (int idx = threadIdx.x; idx < a.n_lm; idx += blockDim.x) {
    const int l = degree_of(idx);
    const int t = idx - l * l;
    if (t == 0) continue;
    float acc[S];
#pragma unroll
    for (int q = 0; q < S; ++q) acc[q] = 0.0f;
#pragma unroll 4
    for (int j = 0; j < a.n_theta; ++j) {
      const float tv = a.tb[(size_t)j * a.n_lm + idx];
#pragma unroll
      for (int q = 0; q < S; ++q) acc[q] = fmaf(tv, fs[((size_t)q * a.n_theta + j) * fst + t], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < S; ++q)
      if (q < ns) a.A[(size_t)(shell0 + q) * a.n_lm + idx] = widen(acc[q]);
  }
}

// launch shape of the azimuthal stage with JC rows per item
int phi_threads(int nt_pad, int jc) { return ((nt_pad / kTT) * (jc / kTJ) + 31) / 32 * 32; }   // whole warps
size_t phi_smem(const yy_grid *g, int nt_pad, int jc, size_t el) {
  return (size_t)g->n_phi * (nt_pad + xpad(jc)) * el;
}

template <typename T>
cudaError_t run_separable(yy_grid *g, const double *rho_yin, const double *rho_yang, const T *w, const T *az,
                          const T *tb, T *F, int blocks, cudaStream_t s) {
  const int nt_pad = g->sep_nt_pad;
  const int jc = g->sep_jc[sizeof(T) == 8];
  const int threads = phi_threads(nt_pad, jc);
  const size_t smem_phi = phi_smem(g, nt_pad, jc, sizeof(T));
  const int shells = grid_rows(g);
  const int grid = std::min(shells * ((g->n_theta + jc - 1) / jc), blocks);
  if (jc == kJC)
    k_sep_phi<T, kJC><<<grid, threads, smem_phi, s>>>(shells, g->n_r, g->n_theta, g->n_phi, nt_pad, rho_yin, rho_yang,
                                                      w, az, F, (float2 *)g->sep_F0);
  else
    k_sep_phi<T, kJCSmall><<<grid, threads, smem_phi, s>>>(shells, g->n_r, g->n_theta, g->n_phi, nt_pad, rho_yin,
                                                           rho_yang, w, az, F, (float2 *)g->sep_F0);
  note_launch(g, "k_sep_phi", s);
  const size_t smem_theta = theta_smem(g->n_theta, nt_pad, sizeof(T));
  k_sep_theta<T><<<shells, 256, smem_theta, s>>>(g->n_theta, g->n_lm, g->lmax + 1, nt_pad, tb, g->sep_tb0, F,
                                                    (const float2 *)g->sep_F0, g->A);
  note_launch(g, "k_sep_theta", s);
  return cudaGetLastError();
}

// Separable synthesis (CUDA-core forms), persistent over shells (p, i).  Each
// block keeps the cell-centre trig table tr[t][k] in shared memory; per field
// (Phi, g_r, g_theta, g_phi):
//   theta stage  G[j][t] = sum_{l >= m} q[l^2 + t] P_f[j][l^2 + t]
//                (g_phi: the cos slot takes the sin coefficients and the sin
//                slot minus the cos ones, from d/dphi of cos / sin (m phi))
//   phi stage    out[j][k] = sum_t G[j][t] tr[t][k]
// with q the combined coefficients of the field (Q, Q_r, Q_t, Q_t).  Both
// sums run from the top down (l from l_max, t from 2 l_max): the monopole
// (l = 0, t = 0) dominates Phi and g_r, and adding it last leaves one
// rounding of the large value instead of one per small term (fp32: Phi
// error about 1e-6 -> a few 1e-7).
struct SepOut {
  double *o[4][2];     // field, patch
};

template <typename T>
__global__ void k_sep_synth(int n_shells, int n_r, int n_theta, int n_phi, int lmax, int n_lm, int n_fields, int jr,
                            const double *__restrict__ Q, const T *__restrict__ P, const T *__restrict__ dP,
                            const T *__restrict__ Qs, const T *__restrict__ tr, const SepOut out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nt = 2 * lmax + 1;
  const int ntr = (n_phi + 3) & ~3;                     // padded row of the trig table
  const int ntp = nt | 1;                               // odd row stride of G
  T *trs = reinterpret_cast<T *>(smraw);                // [nt][ntr]
  T *Gs = trs + (size_t)nt * ntr;                       // [jr][ntp]: G of one chunk of jr rows
  T *qs = Gs + (size_t)jr * ntp;                        // [n_lm]
  for (int e = threadIdx.x; e < nt * ntr; e += blockDim.x) {
    const int t = e / ntr, k = e % ntr;
    trs[e] = (k < n_phi) ? tr[(size_t)t * n_phi + k] : T(0);
  }
  const size_t n_ang = (size_t)n_theta * n_phi;
  const size_t qsz = (size_t)n_shells * n_lm;
  const int kg = ntr / 4;                                // groups of four longitudes
  for (int shell = blockIdx.x; shell < n_shells; shell += gridDim.x) {
    const int p = shell / n_r, i = shell % n_r;
    for (int f = 0; f < n_fields; ++f) {
      const int qb = f < 2 ? f : 2;
      const T *tab = (f <= 1) ? P : (f == 2 ? dP : Qs);
      __syncthreads();   // trs written / the previous field's G and q consumed
      for (int idx = threadIdx.x; idx < n_lm; idx += blockDim.x) qs[idx] = to_t<T>(Q[qb * qsz + (size_t)shell * n_lm + idx]);
      __syncthreads();
      double *dst = out.o[f][p] + (size_t)i * n_ang;
      for (int j0 = 0; j0 < n_theta; j0 += jr) {
        const int rows = min(jr, n_theta - j0);
        for (int e = threadIdx.x; e < rows * nt; e += blockDim.x) {
          const int jj = e / nt, t = e % nt;
          const int m = (t + 1) / 2;
          const T *tj = tab + (size_t)(j0 + jj) * n_lm;
          T g = T(0);
          if (f < 3) {
            for (int l = lmax; l >= m; --l) g = fma(qs[l * l + t], tj[l * l + t], g);
          } else if (t > 0) {
            const int src = (t & 1) ? t + 1 : t - 1;      // cos slot <- sin coefficient, sin slot <- cos
            for (int l = lmax; l >= m; --l) g = fma(qs[l * l + src], tj[l * l + t], g);
            if (!(t & 1)) g = -g;
          }
          Gs[jj * ntp + t] = g;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < rows * kg; e += blockDim.x) {
          const int jj = e / kg, k0 = (e % kg) * 4;
          const int j = j0 + jj;
          T acc[4] = {T(0), T(0), T(0), T(0)};
          const T *gj = Gs + jj * ntp;
          for (int t = nt - 1; t >= 0; --t) {
            T a4[4];
            ld4(trs + (size_t)t * ntr + k0, a4);
            const T gv = gj[t];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fma(gv, a4[u], acc[u]);
          }
          double *o = dst + (size_t)j * n_phi + k0;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (k0 + u < n_phi) {
              if constexpr (sizeof(T) == 4)
                o[u] = widen(acc[u]);
              else
                o[u] = acc[u];
            }
          }
        }
        __syncthreads();   // G of this chunk consumed
      }
    }
  }
}

}  // namespace

cudaError_t separable_prepare(yy_grid *g) {
  const int nt_pad = (2 * g->lmax + 1 + kTT - 1) / kTT * kTT;
  g->sep_nt_pad = nt_pad;
  const size_t n_az = (size_t)g->n_phi * nt_pad;
  const size_t n_tb = (size_t)g->n_theta * g->n_lm;
  const size_t n_f = (size_t)grid_rows(g) * g->n_theta * nt_pad;
  cudaError_t e = cudaSuccess;
  auto A = [&](void **p, size_t bytes) {
    if (e == cudaSuccess) e = dmalloc(p, bytes);
  };
  A((void **)&g->sep_az, n_az * sizeof(double));
  A((void **)&g->sep_az32, n_az * sizeof(float));
  A((void **)&g->sep_w32, (size_t)g->n_ang * sizeof(float));
  A((void **)&g->sep_tb32, n_tb * sizeof(float));
  A((void **)&g->sep_F, n_f * sizeof(double));   // float64 or fp32 partial transforms
  A((void **)&g->sep_F0, (size_t)grid_rows(g) * g->n_theta * sizeof(float2));
  A((void **)&g->sep_tb0, (size_t)g->n_theta * (g->lmax + 1) * sizeof(float2));
  if (e != cudaSuccess) return e;
  k_tb0<<<(g->n_theta * (g->lmax + 1) + 255) / 256, 256>>>(g->n_theta, g->lmax, g->n_lm, g->dph, g->tbar,
                                                           g->sep_tb0);
  k_az_table<<<(unsigned)((n_az + 255) / 256), 256>>>(g->n_phi, g->lmax, nt_pad, g->ph0, g->dph, g->sep_az);
  k_round<<<(unsigned)((n_az + 255) / 256), 256>>>(n_az, g->sep_az, g->sep_az32);
  k_round<<<(unsigned)((g->n_ang + 255) / 256), 256>>>((size_t)g->n_ang, g->w, g->sep_w32);
  k_round<<<(unsigned)((n_tb + 255) / 256), 256>>>(n_tb, g->tbar, g->sep_tb32);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  {
    const size_t n_p = (size_t)g->n_theta * g->n_lm, n_tr = (size_t)(2 * g->lmax + 1) * g->n_phi;
    A((void **)&g->sep_P32, n_p * sizeof(float));
    A((void **)&g->sep_dP32, n_p * sizeof(float));
    A((void **)&g->sep_Qs32, n_p * sizeof(float));
    A((void **)&g->sep_tr32, n_tr * sizeof(float));
    if (e != cudaSuccess) return e;
    k_round<<<(unsigned)((n_p + 255) / 256), 256>>>(n_p, g->sep_P, g->sep_P32);
    k_round<<<(unsigned)((n_p + 255) / 256), 256>>>(n_p, g->sep_dP, g->sep_dP32);
    k_round<<<(unsigned)((n_p + 255) / 256), 256>>>(n_p, g->sep_Qs, g->sep_Qs32);
    k_round<<<(unsigned)((n_tr + 255) / 256), 256>>>(n_tr, g->sep_tr, g->sep_tr32);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // shared memory: the trig table, G of jr rows (all n_theta where they
    // fit, else as many as fit) and one shell's coefficients
    const int nt = 2 * g->lmax + 1, ntr = (g->n_phi + 3) & ~3;
    const void *ks[2] = {(const void *)k_sep_synth<float>, (const void *)k_sep_synth<double>};
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    g->sep_syn_ok = 0;
    for (int q = 0; q < 2; ++q) {
      const size_t el = q == 0 ? sizeof(float) : sizeof(double);
      const size_t fixed = ((size_t)nt * ntr + g->n_lm) * el, per_row = (size_t)(nt | 1) * el;
      if (fixed + per_row > 227 * 1024) continue;
      const int jr = (int)std::min<size_t>(g->n_theta, (227 * 1024 - fixed) / per_row);
      g->sep_syn_rows[q] = jr;
      g->sep_syn_smem[q] = fixed + jr * per_row;
      if ((e = cudaFuncSetAttribute(ks[q], cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024)) != cudaSuccess)
        return e;
      int nb = 0;
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ks[q], 256, g->sep_syn_smem[q])) != cudaSuccess)
        return e;
      g->sep_syn_blocks[q] = std::max(nb, 1) * sms;
      g->sep_syn_ok |= 1 << q;
    }
  }
  // shared memory of the azimuthal stage (the table and one chunk of rows);
  // grids too large for it leave the separable analysis unavailable
  // (the float64 table at l_max 40 on 1-degree cells needs the short chunk)
  const size_t tail_t = (size_t)(g->n_theta + 1) * sizeof(float2);
  g->sep_ok = 0;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
  for (int q = 0; q < 2; ++q) {
    const size_t el = q ? sizeof(double) : sizeof(float);
    if ((size_t)g->n_theta * nt_pad * el + tail_t > 227 * 1024 || theta_smem(g->n_theta, nt_pad, el) > 227 * 1024)
      continue;
    const int jc = phi_smem(g, nt_pad, kJC, el) <= 227 * 1024 ? kJC : kJCSmall;
    const size_t sm = phi_smem(g, nt_pad, jc, el);
    if (sm > 227 * 1024) continue;
    const void *kp = q ? (jc == kJC ? (const void *)k_sep_phi<double, kJC> : (const void *)k_sep_phi<double, kJCSmall>)
                       : (jc == kJC ? (const void *)k_sep_phi<float, kJC> : (const void *)k_sep_phi<float, kJCSmall>);
    // the attribute belongs to the kernel, not to this grid: always the maximum
    if ((e = cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024)) != cudaSuccess)
      return e;
    int nb = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kp, phi_threads(nt_pad, jc), sm)) != cudaSuccess)
      return e;
    g->sep_jc[q] = jc;
    g->sep_phi_blocks[q] = std::max(nb, 1) * sms;
    g->sep_ok |= 1 << q;
  }
  // the attribute belongs to the kernel, not to this grid: always the maximum
  for (auto f : {(const void *)k_sep_theta<float>, (const void *)k_sep_theta<double>, (const void *)k_sep_theta_partials})
    if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024)) != cudaSuccess)
      return e;
  return cudaSuccess;
}

cudaError_t synthesis_separable(yy_grid *g, double *phi_yin, double *phi_yang, double *grad_yin, double *grad_yang,
                                bool fp64, cudaStream_t s) {
  const size_t comp = (size_t)g->n_r * g->n_ang;
  SepOut o = {};
  o.o[0][0] = phi_yin;
  o.o[0][1] = phi_yang;
  for (int c = 0; c < 3 && grad_yin; ++c) {
    o.o[1 + c][0] = grad_yin + c * comp;
    o.o[1 + c][1] = grad_yang ? grad_yang + c * comp : nullptr;
  }
  const int n_fields = grad_yin ? 4 : 1;
  const int q = fp64 ? 1 : 0;
  const int blocks = std::min(grid_rows(g), g->sep_syn_blocks[q]);
  if (fp64)
    k_sep_synth<double><<<blocks, 256, g->sep_syn_smem[1], s>>>(grid_rows(g), g->n_r, g->n_theta, g->n_phi, g->lmax, g->n_lm,
                                                                n_fields, g->sep_syn_rows[1], g->Q, g->sep_P, g->sep_dP, g->sep_Qs,
                                                                g->sep_tr, o);
  else
    k_sep_synth<float><<<blocks, 256, g->sep_syn_smem[0], s>>>(grid_rows(g), g->n_r, g->n_theta, g->n_phi, g->lmax, g->n_lm,
                                                               n_fields, g->sep_syn_rows[0], g->Q, g->sep_P32, g->sep_dP32, g->sep_Qs32,
                                                               g->sep_tr32, o);
  note_launch(g, "k_sep_synth", s);
  return cudaGetLastError();
}

size_t separable_theta_partials_smem(const yy_grid *g, int nt_pad) {
  return (size_t)kThetaShells * g->n_theta * (sizeof(float2) + 2 * sizeof(float) + (nt_pad + 1) * sizeof(float));
}

cudaError_t separable_theta_partials(yy_grid *g, SepThetaPartials a, cudaStream_t s) {
  a.n_theta = g->n_theta;
  a.n_lm = g->n_lm;
  a.lmax1 = g->lmax + 1;
  a.tb = g->sep_tb32;
  a.tb0 = (const float2 *)g->sep_tb0;
  a.A = g->A;
  const int S = kThetaShells;
  const size_t smem = separable_theta_partials_smem(g, a.nt_pad);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  k_sep_theta_partials<<<(grid_rows(g) + S - 1) / S, 256, smem, s>>>(a, grid_rows(g));
  note_launch(g, "k_sep_theta_partials", s);
  return cudaGetLastError();
}

cudaError_t separable_theta_f64(yy_grid *g, cudaStream_t s) {
  const int nt_pad = g->sep_nt_pad;
  const size_t smem_theta = theta_smem(g->n_theta, nt_pad, sizeof(double));
  k_sep_theta<double><<<grid_rows(g), 256, smem_theta, s>>>(g->n_theta, g->n_lm, g->lmax + 1, nt_pad, g->tbar,
                                                            g->sep_tb0, g->sep_F, (const float2 *)g->sep_F0, g->A);
  note_launch(g, "k_sep_theta<double>", s);
  return cudaGetLastError();
}

cudaError_t analysis_separable(yy_grid *g, const double *rho_yin, const double *rho_yang, bool fp64, cudaStream_t s) {
  if (fp64)
    return run_separable<double>(g, rho_yin, rho_yang, g->w, g->sep_az, g->tbar, g->sep_F, g->sep_phi_blocks[1], s);
  return run_separable<float>(g, rho_yin, rho_yang, g->sep_w32, g->sep_az32, g->sep_tb32, (float *)g->sep_F,
                              g->sep_phi_blocks[0], s);
}

}  // namespace yy
