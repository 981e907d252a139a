// Tensor-core forms of the two contractions: operand packing, tables,
// launches and the C entry points behind them.  The pair kernel itself
// (k_tc_pair, its forms and PTX wrappers) is in yy_tc_pair.cuh.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "yy_internal.h"
#include "yy_tc_pair.cuh"
#include "yy_oz_synth.cuh"
#include "yy_oz_analysis.cuh"

namespace yy {

// ---------------------------------------------------------------------------
// operand packing: float64 rows -> scaled narrow pieces [P][rows_pad][k_pad]
// ---------------------------------------------------------------------------
//
// One CTA per row.  Pass 1 converts the row to fp32 (cached in shared memory
// when it is short) and gathers, with compensated fp32 sums: the row sum (for
// the optional mean subtraction), the minimum / maximum, and an optional dot
// product with an fp32 vector (the float64 monopole of the analysis).  Pass 2
// scales (x - mean) by a power of two so that the row maximum lies in
// [2^14, 2^15) and splits it into the form's pieces, 8 elements per store.

struct PackArgs {
  int rows;              // valid rows
  int rows_pad;          // rows of one piece
  int K, k_pad;          // valid / padded row length
  const double *src0, *src1;
  int split_row;         // rows < split_row from src0
  long long ld;          // source row stride
  int zero_k0, zero_k1;  // source columns left out (-1: none)
  int zero_row;          // source row left out (-1: none)
  const float *dot_vec;  // optional: dot_out[row] = sum_k x[k] dot_vec[k]
  double *dot_out;
  double add_factor;     // optional: row_add[row] = add_factor x[zero_k0]
  float *row_add;
  double *mean_out;      // optional: pack x - mean, store the mean used
  double *scale_out;     // [rows_pad] power of two undoing the scaling (float64)
  float *scale_out_f;    // the same in fp32 (optional)
  void *out;             // pieces
  int cache;             // 1: row cached in shared memory (K floats)
  const float *wrow;     // optional (register-resident form only): x[k] *= wrow[(row % w_rows) K + k]
  int w_rows;
};

struct PackBatch {
  PackArgs job[3];       // blockIdx.y selects the job
};

// compensated accumulation (Neumaier) in fp32
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
  const float t = s + x;
  c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
  s = t;
}

template <class F>
__device__ __forceinline__ void split8(const float (&y)[8], typename F::elem *base, size_t piece_stride) {
  if constexpr (F::kKind == KIND_F16) {
    __align__(16) __half h[8], l[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      h[i] = __float2half_rn(y[i]);
      l[i] = __float2half_rn(y[i] - __half2float(h[i]));
    }
    *(uint4 *)base = *(const uint4 *)h;
    *(uint4 *)(base + piece_stride) = *(const uint4 *)l;
  } else if constexpr (F::kKind == KIND_BF16) {
    __align__(16) __nv_bfloat16 h[8], m[8], l[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      h[i] = __float2bfloat16_rn(y[i]);
      const float r = y[i] - __bfloat162float(h[i]);
      m[i] = __float2bfloat16_rn(r);
      l[i] = __float2bfloat16_rn(r - __bfloat162float(m[i]));
    }
    *(uint4 *)base = *(const uint4 *)h;
    *(uint4 *)(base + piece_stride) = *(const uint4 *)m;
    *(uint4 *)(base + 2 * piece_stride) = *(const uint4 *)l;
  } else {
    __align__(16) uint32_t t[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t[i]) : "f"(y[i]));
    *(uint4 *)base = *(const uint4 *)t;
    *(uint4 *)(base + 4) = *(const uint4 *)(t + 4);
  }
}

template <class F>
__global__ void __launch_bounds__(256) k_pack_rows(PackBatch batch) {
  extern __shared__ float rowbuf[];
  __shared__ double red[4][256];
  const PackArgs &p = batch.job[blockIdx.y];
  const int row = blockIdx.x;
  if (row >= p.rows_pad) return;
  typedef typename F::elem E;
  const size_t piece_stride = (size_t)p.rows_pad * p.k_pad;
  E *orow = (E *)p.out + (size_t)row * p.k_pad;
  const bool valid = row < p.rows && row != p.zero_row;
  const double *src = nullptr;
  if (valid) src = (row < p.split_row) ? p.src0 + (size_t)row * p.ld : p.src1 + (size_t)(row - p.split_row) * p.ld;

  float s = 0.f, sc_ = 0.f, d = 0.f, dc = 0.f, mn = INFINITY, mx = -INFINITY;
  if (valid) {
    // 4 consecutive values per thread and step, all loads issued before use
#pragma unroll 2
    for (int k0 = threadIdx.x * 4; k0 < p.K; k0 += blockDim.x * 4) {
      double xv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) xv[i] = (k0 + i < p.K) ? src[k0 + i] : 0.0;
      float bv[4] = {0.f, 0.f, 0.f, 0.f};
      if (p.dot_vec) {
#pragma unroll
        for (int i = 0; i < 4; ++i) bv[i] = (k0 + i < p.K) ? p.dot_vec[k0 + i] : 0.f;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int k = k0 + i;
        if (k >= p.K) break;
        const bool used = (k != p.zero_k0 && k != p.zero_k1);
        const float x = used ? f64_to_f32(xv[i]) : 0.0f;
        if (p.cache) rowbuf[k] = x;
        if (!used) continue;
        kahan_add(s, sc_, x);
        mn = fminf(mn, x);
        mx = fmaxf(mx, x);
        if (p.dot_vec) {
          const float pr = x * bv[i];
          kahan_add(d, dc, pr);
          kahan_add(d, dc, fmaf(x, bv[i], -pr));
        }
      }
    }
  }
  red[0][threadIdx.x] = (double)s + (double)sc_;
  red[1][threadIdx.x] = (double)d + (double)dc;
  red[2][threadIdx.x] = (double)mn;
  red[3][threadIdx.x] = (double)mx;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
      red[2][threadIdx.x] = fmin(red[2][threadIdx.x], red[2][threadIdx.x + w]);
      red[3][threadIdx.x] = fmax(red[3][threadIdx.x], red[3][threadIdx.x + w]);
    }
    __syncthreads();
  }
  const int n_used = p.K - (p.zero_k0 >= 0 ? 1 : 0) - ((p.zero_k1 >= 0 && p.zero_k1 != p.zero_k0) ? 1 : 0);
  float mean = 0.0f;
  if (p.mean_out && valid && n_used > 0) mean = (float)(red[0][0] / n_used);
  float amax = 0.0f;
  if (valid && n_used > 0) amax = fmaxf((float)red[3][0] - mean, mean - (float)red[2][0]);
  float scf = 1.0f;
  if (amax > 0.0f && isfinite(amax)) scf = ldexpf(1.0f, 14 - ilogbf(amax));
  if (threadIdx.x == 0) {
    p.scale_out[row] = 1.0 / (double)scf;
    if (p.scale_out_f) p.scale_out_f[row] = 1.0f / scf;
    if (p.mean_out) p.mean_out[row] = (double)mean;
    if (p.dot_vec && row < p.rows) p.dot_out[row] = valid ? red[1][0] : 0.0;
    if (p.row_add && row < p.rows)
      p.row_add[row] = (valid && p.zero_k0 >= 0) ? (float)(p.add_factor * src[p.zero_k0]) : 0.0f;
  }
  if (p.cache) __syncthreads();
  for (int k0 = threadIdx.x * 8; k0 < p.k_pad; k0 += blockDim.x * 8) {
    float xs[8];
    if (p.cache) {
#pragma unroll
      for (int i = 0; i < 8; ++i) xs[i] = (valid && k0 + i < p.K) ? rowbuf[k0 + i] : 0.0f;
    } else {
      double xv[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) xv[i] = (valid && k0 + i < p.K) ? src[k0 + i] : 0.0;
#pragma unroll
      for (int i = 0; i < 8; ++i) xs[i] = f64_to_f32(xv[i]);
    }
    float y[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = k0 + i;
      const bool used = valid && k < p.K && k != p.zero_k0 && k != p.zero_k1;
      y[i] = used ? (xs[i] - mean) * scf : 0.0f;
    }
    split8<F>(y, orow + k0, piece_stride);
  }
}

// Two adjacent elements split into the form's pieces (piece p at base + p
// piece_stride); base is 4-byte aligned (8-byte for tf32).
template <class F>
__device__ __forceinline__ void split2(float y0, float y1, typename F::elem *base, size_t piece_stride) {
  if constexpr (F::kKind == KIND_F16) {
    const __half2 h = __floats2half2_rn(y0, y1);
    const float2 hb = __half22float2(h);
    *(__half2 *)base = h;
    *(__half2 *)(base + piece_stride) = __floats2half2_rn(y0 - hb.x, y1 - hb.y);
  } else if constexpr (F::kKind == KIND_BF16) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(y0, y1);
    const float2 hb = __bfloat1622float2(h);
    const float r0 = y0 - hb.x, r1 = y1 - hb.y;
    const __nv_bfloat162 m = __floats2bfloat162_rn(r0, r1);
    const float2 mb = __bfloat1622float2(m);
    *(__nv_bfloat162 *)base = h;
    *(__nv_bfloat162 *)(base + piece_stride) = m;
    *(__nv_bfloat162 *)(base + 2 * piece_stride) = __floats2bfloat162_rn(r0 - mb.x, r1 - mb.y);
  } else {
    uint2 t;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t.x) : "f"(y0));
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t.y) : "f"(y1));
    *(uint2 *)base = t;
  }
}

// Register-resident form of the packing: TPR threads per row, each holding 2P
// values (pair c: elements 2 (c TPR + thread) + {0, 1}), so the row is read
// once, every load and store instruction covers consecutive elements across
// the threads, and the statistics need only shuffles (plus shared memory
// across warps when TPR > 32).  TPR = 32: one warp per row, 8 rows per block
// (short rows); TPR = 1024: one block per row (long rows).  Requires
// k_pad <= 2 P TPR.  The chip's float64 pipe is narrow, so all per-thread
// arithmetic is fp32: the row sum (it only fixes the centring value; the
// same float is used again in the correction), the minimum and maximum, and
// the optional dot product as an unevaluated fp32 pair (hi + lo, Knuth's
// two-sum); one thread forms the float64 results.

struct RowStats {
  float s, dh, dl, mn, mx;
};

__device__ __forceinline__ void two_sum_add(float &h, float &l, float bh, float bl) {
  const float s = h + bh;
  const float bb = s - h;
  const float e = (h - (s - bb)) + (bh - bb);
  const float t = l + bl + e;
  h = s + t;
  l = t - (h - s);
}

__device__ __forceinline__ void warp_stats(RowStats &r) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    r.s += __shfl_xor_sync(0xffffffffu, r.s, off);
    const float oh = __shfl_xor_sync(0xffffffffu, r.dh, off);
    const float ol = __shfl_xor_sync(0xffffffffu, r.dl, off);
    two_sum_add(r.dh, r.dl, oh, ol);
    r.mn = fminf(r.mn, __shfl_xor_sync(0xffffffffu, r.mn, off));
    r.mx = fmaxf(r.mx, __shfl_xor_sync(0xffffffffu, r.mx, off));
  }
}

template <int TPR>
__device__ __forceinline__ void row_stats(RowStats &r, RowStats *red) {
  warp_stats(r);
  if constexpr (TPR > 32) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = r;
    __syncthreads();
    if (w == 0) {
      r = (lane < TPR / 32) ? red[lane] : RowStats{0.f, 0.f, 0.f, INFINITY, -INFINITY};
      warp_stats(r);
      if (lane == 0) red[0] = r;
    }
    __syncthreads();
    r = red[0];
  }
}

// The row's values in fp32 registers (x) and its partial statistics; src may
// point to global or shared memory.
template <int TPR, int P>
__device__ __forceinline__ void pack_load(const PackArgs &p, int row, const double *src, bool valid, bool vec,
                                          int tid, float (&x)[2 * P], RowStats &st) {
  const int K = p.K, z0 = p.zero_k0, z1 = p.zero_k1;
  // loads in runs of 4 pairs; the dot product adds fp32 runs of 8 products
  st = RowStats{0.f, 0.f, 0.f, INFINITY, -INFINITY};
#pragma unroll
  for (int c0 = 0; c0 < P; c0 += 4) {
    double xv[8];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = 2 * ((c0 + i) * TPR + tid);
      if (valid && k + 1 < K && vec) {
        const double2 t = *(const double2 *)(src + k);
        xv[2 * i] = t.x;
        xv[2 * i + 1] = t.y;
      } else {
        xv[2 * i] = (valid && k < K) ? src[k] : 0.0;
        xv[2 * i + 1] = (valid && k + 1 < K) ? src[k + 1] : 0.0;
      }
    }
    float run = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int c = 2 * c0 + i;
      const int k = 2 * ((c0 + i / 2) * TPR + tid) + (i & 1);
      const bool used = valid && k < K && k != z0 && k != z1;
      float v = used ? f64_to_f32(xv[i]) : 0.0f;
      if (p.wrow && used) v *= p.wrow[(size_t)(row % p.w_rows) * K + k];
      x[c] = v;
      st.s += v;
      if (used) {
        st.mn = fminf(st.mn, v);
        st.mx = fmaxf(st.mx, v);
      }
      if (p.dot_vec) run = fmaf(v, (k < K) ? p.dot_vec[k] : 0.0f, run);
    }
    if (p.dot_vec) two_sum_add(st.dh, st.dl, run, 0.0f);
  }
}

// The row's statistics across its threads, the per-row outputs, and the
// scaled, centred values split into the form's pieces (src: the row in
// global memory, for row_add).
template <class F, int TPR, int P>
__device__ __forceinline__ void pack_store(const PackArgs &p, int row, const double *src, bool valid, int tid,
                                           const float (&x)[2 * P], RowStats st, RowStats *red) {
  typedef typename F::elem E;
  const size_t piece_stride = (size_t)p.rows_pad * p.k_pad;
  E *orow = (E *)p.out + (size_t)row * p.k_pad;
  const int K = p.K, z0 = p.zero_k0, z1 = p.zero_k1;
  row_stats<TPR>(st, red);
  const int n_used = K - (z0 >= 0 ? 1 : 0) - ((z1 >= 0 && z1 != z0) ? 1 : 0);
  float mean = 0.0f;
  if (p.mean_out && valid && n_used > 0) mean = st.s / (float)n_used;
  float amax = 0.0f;
  if (valid && n_used > 0) amax = fmaxf(st.mx - mean, mean - st.mn);
  float scf = 1.0f;
  if (amax > 0.0f && isfinite(amax)) scf = ldexpf(1.0f, 14 - ilogbf(amax));
  if (tid == 0) {
    p.scale_out[row] = (double)(1.0f / scf);   // a power of two: exact in fp32
    if (p.scale_out_f) p.scale_out_f[row] = 1.0f / scf;
    if (p.mean_out) p.mean_out[row] = (double)mean;
    if (p.dot_vec && row < p.rows) p.dot_out[row] = valid ? (double)st.dh + (double)st.dl : 0.0;
    if (p.row_add && row < p.rows)
      p.row_add[row] = (valid && z0 >= 0) ? (float)(p.add_factor * src[z0]) : 0.0f;
  }
  // (x - mean) scf as one rounding: scf is a power of two
  const float off = -mean * scf;
#pragma unroll
  for (int c = 0; c < P; ++c) {
    const int k = 2 * (c * TPR + tid);
    if (k >= p.k_pad) break;
    const bool u0 = valid && k < K && k != z0 && k != z1;
    const bool u1 = valid && k + 1 < K && k + 1 != z0 && k + 1 != z1;
    split2<F>(u0 ? fmaf(x[2 * c], scf, off) : 0.0f, u1 ? fmaf(x[2 * c + 1], scf, off) : 0.0f, orow + k,
              piece_stride);
  }
}

template <class F, int TPR, int P>
__global__ void __launch_bounds__(TPR > 256 ? TPR : 256, (TPR <= 32 && P <= 6) ? 4 : ((TPR <= 32 && P <= 12) ? 3 : 1))
k_pack_reg(PackBatch batch) {
  constexpr int TPB = TPR > 256 ? TPR : 256;
  __shared__ RowStats red[32];
  const PackArgs &p = batch.job[blockIdx.y];
  const int tid = threadIdx.x % TPR;
  const int row = blockIdx.x * (TPB / TPR) + threadIdx.x / TPR;
  if (row >= p.rows_pad) return;   // whole rows (and, for TPR > 32, whole blocks) leave together
  const bool valid = row < p.rows && row != p.zero_row;
  const double *src = nullptr;
  if (valid) src = (row < p.split_row) ? p.src0 + (size_t)row * p.ld : p.src1 + (size_t)(row - p.split_row) * p.ld;
  const bool vec = ((uintptr_t)src & 15u) == 0;
  float x[2 * P];
  RowStats st;
  pack_load<TPR, P>(p, row, src, valid, vec, tid, x, st);
  pack_store<F, TPR, P>(p, row, src, valid, tid, x, st, red);
}

// Streaming form for long rows of densities: a persistent block of 1024
// threads per SM walks the rows blockIdx.x, blockIdx.x + gridDim.x, ...  One
// thread starts the bulk copy of the block's next float64 row into shared
// memory as soon as every thread holds the current one in registers, so that
// row's reads stay in flight while the block reduces and stores the current
// one.  Only the density job takes this form (no columns or rows left out, no
// weight rows, an even row length, 16-byte aligned rows; the launcher checks),
// so its predicates are per pair of elements; the arithmetic and its order are
// those of k_pack_reg<F, 1024, kStreamP>.
constexpr int kStreamP = 12;
constexpr int kStreamMaxK = 2 * kStreamP * 1024;
constexpr int kStreamChunk = 4096;   // doubles per bulk copy

// float64 -> fp32, round to nearest even, for values in fp32's normal range:
// add the rounding bias at bit 29 of the 64-bit word (0x0FFFFFFF, plus one
// when the kept part is odd, so that a tie goes to the even neighbour), keep
// bits 29..60 (23 mantissa bits and the low 9 exponent bits) and rebias the
// exponent by 1023 - 127 = 896 modulo 2^8 (the range check makes that exact;
// a carry out of the mantissa steps the exponent, to infinity at the top).
// Every other input (zero, subnormal, out of range, inf, nan) takes
// f64_to_f32.  Same results as f64_to_f32 with about half the operations.
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const uint32_t lo = (uint32_t)__double2loint(x), hi = (uint32_t)__double2hiint(x);
  const uint32_t ex = (hi >> 20) & 0x7FFu;
  if (ex - 897u >= 254u) return f64_to_f32(x);
  const uint32_t bias = 0x0FFFFFFFu + ((lo >> 29) & 1u);
  uint32_t l2, h2;
  asm("add.cc.u32 %0, %2, %3;\n\taddc.u32 %1, %4, 0;" : "=r"(l2), "=r"(h2) : "r"(lo), "r"(bias), "r"(hi));
  const uint32_t m = __funnelshift_r(l2, h2, 29);
  // 896 << 23 modulo 2^32 is 0xC0000000
  return __uint_as_float(((m - 0xC0000000u) & 0x7FFFFFFFu) | (hi & 0x80000000u));
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

template <class F>
__global__ void __launch_bounds__(1024, 1) k_pack_stream(PackArgs p, int *err) {
  extern __shared__ __align__(16) double rowbuf_f64[];
  __shared__ RowStats red[32];
  __shared__ __align__(8) uint64_t bar;
  typedef typename F::elem E;
  const int tid = threadIdx.x;
  const int K = p.K;
  const size_t piece_stride = (size_t)p.rows_pad * p.k_pad;
  auto row_src = [&](int r) {
    return (r < p.split_row) ? p.src0 + (size_t)r * p.ld : p.src1 + (size_t)(r - p.split_row) * p.ld;
  };
  auto issue = [&](int r) {   // one thread
    const double *src = row_src(r);
    mbar_expect_tx(&bar, (uint32_t)K * 8u);
    for (int k0 = 0; k0 < K; k0 += kStreamChunk) {
      const int n = min(kStreamChunk, K - k0);
      bulk_load(smem_u32(rowbuf_f64 + k0), src + k0, (uint32_t)n * 8u, &bar);
    }
  };
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  int row = blockIdx.x;
  if (tid == 0 && row < p.rows) issue(row);
  uint32_t phase = 0;
  for (; row < p.rows_pad; row += gridDim.x) {
    const bool valid = row < p.rows;
    if (valid) {
      const bool ok = mbar_wait(&bar, phase, err);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {   // timed out: let the copy finish (bounded), then leave
        if (tid == 0) mbar_wait(&bar, phase ^ 1u, err);
        return;
      }
    }
    // the row in fp32 registers and its statistics (runs of 4 pairs for the dot product)
    float x[2 * kStreamP];
    RowStats st = {0.f, 0.f, 0.f, INFINITY, -INFINITY};
#pragma unroll
    for (int c0 = 0; c0 < kStreamP; c0 += 4) {
      float run = 0.0f;
#pragma unroll
      for (int c = c0; c < c0 + 4; ++c) {
        const int k = 2 * (c * 1024 + tid);
        float v0 = 0.0f, v1 = 0.0f, d0 = 0.0f, d1 = 0.0f;
        if (valid && k < K) {
          const double2 t = *(const double2 *)(rowbuf_f64 + k);
          v0 = f64_to_f32_rn(t.x);
          v1 = f64_to_f32_rn(t.y);
          st.mn = fminf(st.mn, fminf(v0, v1));
          st.mx = fmaxf(st.mx, fmaxf(v0, v1));
          if (p.dot_vec) {
            const float2 d = *(const float2 *)(p.dot_vec + k);
            d0 = d.x;
            d1 = d.y;
          }
        }
        x[2 * c] = v0;
        x[2 * c + 1] = v1;
        st.s += v0;
        st.s += v1;
        run = fmaf(v0, d0, run);
        run = fmaf(v1, d1, run);
      }
      if (p.dot_vec) two_sum_add(st.dh, st.dl, run, 0.0f);
    }
    __syncthreads();   // every thread holds the row: the buffer is free
    const int next = row + gridDim.x;
    if (tid == 0 && next < p.rows) issue(next);
    row_stats<1024>(st, red);
    float mean = 0.0f;
    if (p.mean_out && valid) mean = st.s / (float)K;
    float amax = 0.0f;
    if (valid) amax = fmaxf(st.mx - mean, mean - st.mn);
    float scf = 1.0f;
    if (amax > 0.0f && isfinite(amax)) scf = ldexpf(1.0f, 14 - ilogbf(amax));
    if (tid == 0) {
      p.scale_out[row] = (double)(1.0f / scf);   // a power of two: exact in fp32
      if (p.scale_out_f) p.scale_out_f[row] = 1.0f / scf;
      if (p.mean_out) p.mean_out[row] = (double)mean;
      if (p.dot_vec && valid) p.dot_out[row] = (double)st.dh + (double)st.dl;
    }
    // (x - mean) scf as one rounding: scf is a power of two
    const float off = -mean * scf;
    E *orow = (E *)p.out + (size_t)row * p.k_pad;
#pragma unroll
    for (int c = 0; c < kStreamP; ++c) {
      const int k = 2 * (c * 1024 + tid);
      if (k >= p.k_pad) break;
      const bool u = valid && k < K;
      split2<F>(u ? fmaf(x[2 * c], scf, off) : 0.0f, u ? fmaf(x[2 * c + 1], scf, off) : 0.0f, orow + k,
                piece_stride);
    }
  }
}

// The streaming form over the long, even rows of many jobs: the grid walks
// the concatenated rows (row_map[i] = job << 24 | the job's own row, padding
// rows included), each row with its job's arguments, the next row's copy in
// flight as above.
template <class F>
__global__ void __launch_bounds__(1024, 1)
k_pack_stream_group(const PackArgs *__restrict__ jobs, const uint32_t *__restrict__ row_map, int n_rows, int *err) {
  extern __shared__ __align__(16) double rowbuf_f64[];
  __shared__ RowStats red[32];
  __shared__ __align__(8) uint64_t bar;
  typedef typename F::elem E;
  const int tid = threadIdx.x;
  auto issue = [&](const PackArgs &q, int r) {   // one thread
    const double *src = (r < q.split_row) ? q.src0 + (size_t)r * q.ld : q.src1 + (size_t)(r - q.split_row) * q.ld;
    mbar_expect_tx(&bar, (uint32_t)q.K * 8u);
    for (int k0 = 0; k0 < q.K; k0 += kStreamChunk) {
      const int n = min(kStreamChunk, q.K - k0);
      bulk_load(smem_u32(rowbuf_f64 + k0), src + k0, (uint32_t)n * 8u, &bar);
    }
  };
  // the job and row of global row i, and whether it carries data
  auto at = [&](int i, int &job, int &r) {
    const uint32_t m = row_map[i];
    job = (int)(m >> 24);
    r = (int)(m & 0xFFFFFFu);
  };
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (tid == 0 && (int)blockIdx.x < n_rows) {
    int j0, r0;
    at((int)blockIdx.x, j0, r0);
    if (r0 < jobs[j0].rows) issue(jobs[j0], r0);
  }
  uint32_t phase = 0;
  for (int gi = blockIdx.x; gi < n_rows; gi += gridDim.x) {
    int jb, row;
    at(gi, jb, row);
    const PackArgs &p = jobs[jb];
    const int K = p.K;
    const size_t piece_stride = (size_t)p.rows_pad * p.k_pad;
    const bool valid = row < p.rows;
    if (valid) {
      const bool ok = mbar_wait(&bar, phase, err);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {   // timed out: let the copy finish (bounded), then leave
        if (tid == 0) mbar_wait(&bar, phase ^ 1u, err);
        return;
      }
    }
    // the row in fp32 registers and its statistics (runs of 4 pairs for the dot product)
    float x[2 * kStreamP];
    RowStats st = {0.f, 0.f, 0.f, INFINITY, -INFINITY};
#pragma unroll
    for (int c0 = 0; c0 < kStreamP; c0 += 4) {
      float run = 0.0f;
#pragma unroll
      for (int c = c0; c < c0 + 4; ++c) {
        const int k = 2 * (c * 1024 + tid);
        float v0 = 0.0f, v1 = 0.0f, d0 = 0.0f, d1 = 0.0f;
        if (valid && k < K) {
          const double2 t = *(const double2 *)(rowbuf_f64 + k);
          v0 = f64_to_f32_rn(t.x);
          v1 = f64_to_f32_rn(t.y);
          st.mn = fminf(st.mn, fminf(v0, v1));
          st.mx = fmaxf(st.mx, fmaxf(v0, v1));
          if (p.dot_vec) {
            const float2 d = *(const float2 *)(p.dot_vec + k);
            d0 = d.x;
            d1 = d.y;
          }
        }
        x[2 * c] = v0;
        x[2 * c + 1] = v1;
        st.s += v0;
        st.s += v1;
        run = fmaf(v0, d0, run);
        run = fmaf(v1, d1, run);
      }
      if (p.dot_vec) two_sum_add(st.dh, st.dl, run, 0.0f);
    }
    __syncthreads();   // every thread holds the row: the buffer is free
    const int next = gi + gridDim.x;
    if (tid == 0 && next < n_rows) {
      int jn, rn;
      at(next, jn, rn);
      if (rn < jobs[jn].rows) issue(jobs[jn], rn);
    }
    row_stats<1024>(st, red);
    float mean = 0.0f;
    if (p.mean_out && valid) mean = st.s / (float)K;
    float amax = 0.0f;
    if (valid) amax = fmaxf(st.mx - mean, mean - st.mn);
    float scf = 1.0f;
    if (amax > 0.0f && isfinite(amax)) scf = ldexpf(1.0f, 14 - ilogbf(amax));
    if (tid == 0) {
      p.scale_out[row] = (double)(1.0f / scf);   // a power of two: exact in fp32
      if (p.scale_out_f) p.scale_out_f[row] = 1.0f / scf;
      if (p.mean_out) p.mean_out[row] = (double)mean;
      if (p.dot_vec && valid) p.dot_out[row] = (double)st.dh + (double)st.dl;
    }
    // (x - mean) scf as one rounding: scf is a power of two
    const float off = -mean * scf;
    E *orow = (E *)p.out + (size_t)row * p.k_pad;
#pragma unroll
    for (int c = 0; c < kStreamP; ++c) {
      const int k = 2 * (c * 1024 + tid);
      if (k >= p.k_pad) break;
      const bool u = valid && k < K;
      split2<F>(u ? fmaf(x[2 * c], scf, off) : 0.0f, u ? fmaf(x[2 * c + 1], scf, off) : 0.0f, orow + k,
                piece_stride);
    }
  }
}

// ---------------------------------------------------------------------------
// separable synthesis on the tensor cores: the polar stage
// ---------------------------------------------------------------------------
//
// For every output row (shell, j) and field f, the azimuthal coefficients
//   G_f[t] = sum_{l >= m(t)} q_f[l^2 + t] T_f[j][l^2 + t]
// (T = K_lm P_l^m, its theta derivative, or m K_lm P_l^m / sin theta; g_phi
// takes the sin coefficient into the cos slot and minus the cos one into the
// sin slot), so that the field is sum_t G_f[t] trig_t(phi_k): the azimuthal
// stage is a contraction with K = 2 l_max + 1 done by k_tc_pair (out_mode 2).
// t = 0 (cos 0 = 1 at every phi_k) carries the monopole; it is summed as an
// unevaluated fp32 pair and added per cell, and its slot of the operand is
// zero.  The other slots are scaled per row by a power of two (row maximum in
// [2^14, 2^15)) and split into the form's pieces.  One block per shell, one
// warp per (j, field); each lane owns slots 2 lane + {0, 1} + 64 i.

struct ThetaArgs {
  int n_shells, n_theta, lmax, n_lm, nt, k_pad, n_jobs, rows_pad;
  const double *Q;              // [3][n_shells][n_lm]: Phi, g_r and angular coefficients
  const float *tab[3];          // [n_theta][n_lm]: P, dP/dtheta, m P / sin theta
  const double *tab64[2];       // [n_theta][n_lm]: P and dP in float64 (their l = 0 column is used)
  void *G[4];                   // per field: bf16 pieces [3][rows_pad][k_pad]
  float *add[4];                // per field: [rows_pad] slot-0 term
};

constexpr int kThetaSmemMax = 200 * 1024;

// exact split of an fp32 value into three bf16 pieces (hi + mid + lo)
__device__ __forceinline__ void split_bf16x3(float y, __nv_bfloat16 *base, size_t stride) {
  const __nv_bfloat16 h = __float2bfloat16_rn(y);
  const float r = y - __bfloat162float(h);
  const __nv_bfloat16 m = __float2bfloat16_rn(r);
  base[0] = h;
  base[stride] = m;
  base[2 * stride] = __float2bfloat16_rn(r - __bfloat162float(m));
}

// Blocks take S consecutive shells (coefficients in shared memory, shell
// fastest so that one vector load serves all S); a warp task is two polar
// rows j of one field.  Slots come in blocks of 64; lane i takes slots
// c0 + i and c0 + 63 - i, whose l-ranges (l >= m(t), m = ceil(t / 2)) add up
// to about the same length in every lane, walked as one loop.  G goes out
// unscaled as three bf16 pieces (bf16 has the fp32 exponent range); slot 0 is
// zero and its value (the m = 0 cos term, which holds the monopole) goes to
// add[] with the l = 0 product in float64.
template <int S, bool STAGE>
__global__ void __launch_bounds__(256) k_theta_g(ThetaArgs a) {
  extern __shared__ __align__(16) float qs[];                 // [3][n_lm][S], then (STAGE) [8 warps][2][n_lm]
  const int shell0 = blockIdx.x * S;
  const int ns = min(S, a.n_shells - shell0);
  const size_t qsz = (size_t)a.n_shells * a.n_lm;
  for (int e = threadIdx.x; e < 3 * a.n_lm * S; e += blockDim.x) {
    const int sh = e % S, ci = e / S;                         // ci = c n_lm + idx
    const int c = ci / a.n_lm, idx = ci - c * a.n_lm;
    qs[e] = sh < ns ? f64_to_f32(a.Q[c * qsz + (size_t)(shell0 + sh) * a.n_lm + idx]) : 0.0f;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t ps = (size_t)a.rows_pad * a.k_pad;
  const int L = a.lmax;
  const int pairs_j = (a.n_theta + 1) >> 1;
  for (int task = warp; task < pairs_j * a.n_jobs; task += blockDim.x >> 5) {
    const int job = task % a.n_jobs, j0 = 2 * (task / a.n_jobs);
    const bool two = j0 + 1 < a.n_theta;
    const int c = job < 2 ? job : 2;
    const float *T0 = a.tab[job < 2 ? 0 : job - 1] + (size_t)j0 * a.n_lm;
    const float *T1 = two ? T0 + a.n_lm : T0;
    if constexpr (STAGE) {
      // the task's two table rows, read once with coalesced loads
      float *tw = qs + (size_t)3 * a.n_lm * S + (size_t)warp * 2 * a.n_lm;
      __syncwarp();
      for (int e = lane; e < a.n_lm; e += 32) {
        tw[e] = T0[e];
        tw[a.n_lm + e] = T1[e];
      }
      __syncwarp();
      T0 = tw;
      T1 = tw + a.n_lm;
    }
    const float *qc = qs + (size_t)c * a.n_lm * S;
    for (int c0 = 0; c0 < a.k_pad; c0 += 64) {
      const int ta = c0 + lane, tb = c0 + 63 - lane;
      const int ma = (ta + 1) >> 1, mb = (tb + 1) >> 1;
      const int na = (ta >= 1 && ta < a.nt) ? L + 1 - ma : 0;
      const int nb = (tb >= 1 && tb < a.nt) ? L + 1 - mb : 0;
      // d/dphi (g_phi): the sin slot takes minus the cos coefficient, the cos slot the sin one
      const int sa = job == 3 ? ((ta & 1) ? ta + 1 : ta - 1) : ta;
      const int sb = job == 3 ? ((tb & 1) ? tb + 1 : tb - 1) : tb;
      float acc[2][S], va[2][S];
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int q = 0; q < S; ++q) acc[r][q] = va[r][q] = 0.0f;
      int t = ta, src = sa, l = ma;
      for (int k = 0; k < na + nb; ++k) {
        if (k == na) {
#pragma unroll
          for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int q = 0; q < S; ++q) {
              va[r][q] = acc[r][q];
              acc[r][q] = 0.0f;
            }
          t = tb;
          src = sb;
          l = mb;
        }
        const int b = l * l;
        const float x0 = T0[b + t], x1 = T1[b + t];
        const float *qv = qc + (size_t)(b + src) * S;
        float qq[S];
        if constexpr (S % 4 == 0) {
#pragma unroll
          for (int q = 0; q < S; q += 4) {
            const float4 v = *reinterpret_cast<const float4 *>(qv + q);
            qq[q] = v.x;
            qq[q + 1] = v.y;
            qq[q + 2] = v.z;
            qq[q + 3] = v.w;
          }
        } else {
#pragma unroll
          for (int q = 0; q < S; ++q) qq[q] = qv[q];
        }
#pragma unroll
        for (int q = 0; q < S; ++q) {
          acc[0][q] = fmaf(qq[q], x0, acc[0][q]);
          acc[1][q] = fmaf(qq[q], x1, acc[1][q]);
        }
        ++l;
      }
      if (nb == 0) {   // the loop never reached the switch: acc holds slot ta
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
          for (int q = 0; q < S; ++q) {
            va[r][q] = acc[r][q];
            acc[r][q] = 0.0f;
          }
      }
      const float sga = (job == 3 && !(ta & 1)) ? -1.0f : 1.0f, sgb = (job == 3 && !(tb & 1)) ? -1.0f : 1.0f;
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        if (r == 1 && !two) break;
#pragma unroll
        for (int q = 0; q < S; ++q) {
          if (q >= ns) break;
          __nv_bfloat16 *row = (__nv_bfloat16 *)a.G[job] + ((size_t)(shell0 + q) * a.n_theta + j0 + r) * a.k_pad;
          split_bf16x3(sga * va[r][q], row + ta, ps);
          split_bf16x3(sgb * acc[r][q], row + tb, ps);
        }
      }
    }
    // slot 0: lane 2 q + r sums shell q, row j0 + r
    if (lane < 2 * ns && (lane & 1) <= (two ? 1 : 0)) {
      const int q = lane >> 1, r = lane & 1;
      float add = 0.0f;
      if (job < 3) {
        const float *T = r ? T1 : T0;
        float sum = 0.0f;
        for (int l = L; l >= 1; --l) sum = fmaf(qc[(size_t)(l * l) * S + q], T[l * l], sum);
        const double q00 = a.Q[c * qsz + (size_t)(shell0 + q) * a.n_lm];
        const double t00 = a.tab64[job < 2 ? 0 : 1][(size_t)(j0 + r) * a.n_lm];
        add = f64_to_f32(fma(q00, t00, f32_to_f64(sum)));
      }
      a.add[job][(size_t)(shell0 + q) * a.n_theta + j0 + r] = add;
    }
  }
}

// The polar stage of the separable tensor-core synthesis: one warp per (field,
// shell, mirrored row pair j, j' = n_theta - 1 - j), the terms of even and of
// odd l + m summed apart so that one pass gives both rows (P and m P / sin
// theta keep the parity of l + m across the equator, dP/dtheta takes the
// opposite one).  Lane L takes the slot pairs 64 g + L and 64 g + 63 - L
// (their term counts add up to about l_max + 1 whatever L), the coefficients
// in fp32 from the scan.  Slot 0 sums l >= 1 here and adds the l = 0 product
// in float64 into add[] (its operand column stays zero).  g_phi needs no sum
// of its own: its coefficients are -Q / r and its table m / sin theta times
// Phi's, so Phi's warps form it from their values of the other slot of the
// same m.
struct ThetaF32Args {
  int n_shells, n_theta, n_r, lmax, n_lm, nt, k_pad, n_jobs, rows_pad;
  const float *Q32;             // [3][n_shells][n_lm]: Phi, g_r and angular coefficients in fp32
  const double *Q;              // float64 (the l = 0 coefficient of slot 0)
  const float *tab[3];          // [n_theta][n_lm]: P, dP/dtheta, m P / sin theta
  const double *tab64[2];       // P and dP in float64 (their l = 0 column)
  const float *inv_sin, *inv_r; // 1 / sin theta_j, 1 / r_(n+1)
  void *G[4];                   // per field: bf16 pieces [3][rows_pad][k_pad]
  float *add[4];                // per field: [rows_pad] slot-0 term
};

__device__ __forceinline__ void store_bf16x3(float y, uint16_t *base, size_t stride) {
  const __nv_bfloat16 h = __float2bfloat16_rn(y);
  const float r = y - __bfloat162float(h);
  const __nv_bfloat16 m = __float2bfloat16_rn(r);
  base[0] = __bfloat16_as_ushort(h);
  base[stride] = __bfloat16_as_ushort(m);
  base[2 * stride] = __bfloat16_as_ushort(__float2bfloat16_rn(r - __bfloat162float(m)));
}

template <int NG>
__global__ void __launch_bounds__(256) k_theta_f32(ThetaF32Args a) {
  const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  const int half = (a.n_theta + 1) >> 1;
  const int pairs = a.n_shells * half;
  const int n_f = a.n_jobs == 4 ? 3 : a.n_jobs;
  if (warp >= pairs * n_f) return;
  const int f = warp / pairs, pr = warp % pairs;
  const int shell = pr / half, j = pr % half, jm = a.n_theta - 1 - j;
  const int qb = f < 2 ? f : 2;
  const float *q = a.Q32 + ((size_t)qb * a.n_shells + shell) * a.n_lm;
  const float *tab = f <= 1 ? a.tab[0] : a.tab[1];
  const float *tj = tab + (size_t)j * a.n_lm;
  const int L = a.lmax;
  float gj[NG][2], gm[NG][2];   // this lane's slots (64 g + lane, 64 g + 63 - lane) at rows j and j'
#pragma unroll
  for (int g = 0; g < NG; ++g) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int t = 64 * g + (h == 0 ? lane : 63 - lane);
      const int m = (t + 1) >> 1;
      const int l_lo = t == 0 ? 1 : m;                      // slot 0: l >= 1 here
      float a1 = 0.f, a2 = 0.f;                            // l = L, L - 2, ... and l = L - 1, L - 3, ...
      if (t < a.nt) {
        int l = L;
        const float *pq = q + L * L + t, *pt = tj + L * L + t;
#pragma unroll 2
        for (; l >= l_lo + 1; l -= 2) {
          a1 = fmaf(pq[0], pt[0], a1);
          const int d1 = 2 * l - 1;                        // l^2 - (l - 1)^2
          a2 = fmaf(pq[-d1], pt[-d1], a2);
          pq -= 4 * l - 4;                                 // l^2 - (l - 2)^2
          pt -= 4 * l - 4;
        }
        if (l == l_lo) a1 = fmaf(pq[0], pt[0], a1);
      }
      // row j: E + O; row j': E - O when a1 holds even l + m (L + m even), else O - E;
      // dP/dtheta has the opposite parity
      const float e_o = ((L + m) & 1) ? a2 - a1 : a1 - a2;
      gj[g][h] = a1 + a2;
      gm[g][h] = f == 2 ? -e_o : e_o;
    }
  }
  const size_t ps = (size_t)a.rows_pad * a.k_pad;
  const size_t row = (size_t)shell * a.n_theta + j, rowm = (size_t)shell * a.n_theta + jm;
  uint16_t *const Gf = (uint16_t *)(f == 0 ? a.G[0] : f == 1 ? a.G[1] : a.G[2]);
#pragma unroll
  for (int g = 0; g < NG; ++g)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int t = 64 * g + (h == 0 ? lane : 63 - lane);
      if (t < 1 || t >= a.nt) continue;                    // slot 0 and the padding stay zero
      store_bf16x3(gj[g][h], Gf + row * a.k_pad + t, ps);
      if (jm != j) store_bf16x3(gm[g][h], Gf + rowm * a.k_pad + t, ps);
    }
  // slot 0 (lane 0, first slot): the l = 0 product in float64
  if (lane == 0) {
    float *const add = f == 0 ? a.add[0] : f == 1 ? a.add[1] : a.add[2];
    const double q00 = a.Q[((size_t)qb * a.n_shells + shell) * a.n_lm];
    const double t00 = (f == 2 ? a.tab64[1] : a.tab64[0])[(size_t)j * a.n_lm];
    add[row] = f64_to_f32(fma(q00, t00, f32_to_f64(gj[0][0])));
    if (jm != j) add[rowm] = f64_to_f32(fma(q00, f == 2 ? -t00 : t00, f32_to_f64(gm[0][0])));
  }
  if (f != 0 || a.n_jobs < 4) return;
  // g_phi: G_phi[t] = (+1 for t even, -1 for t odd) (m / (r sin theta)) G_Phi[swap t]
  const float c = a.inv_r[shell % a.n_r] * a.inv_sin[j];
  uint16_t *const Gp = (uint16_t *)a.G[3];
  const int src = (lane & 1) ? lane + 1 : lane - 1;
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    // the other slot of the same m: the neighbouring lane's slot in the
    // same half of the group, or for lanes 0 and 31 a slot of their own
    float sj0 = __shfl_sync(0xffffffffu, gj[g][0], src & 31), sm0 = __shfl_sync(0xffffffffu, gm[g][0], src & 31);
    float sj1 = __shfl_sync(0xffffffffu, gj[g][1], src & 31), sm1 = __shfl_sync(0xffffffffu, gm[g][1], src & 31);
    if (lane == 31) {
      sj0 = gj[g][1]; sm0 = gm[g][1];
      sj1 = gj[g][0]; sm1 = gm[g][0];
    } else if (lane == 0) {
      sj0 = g > 0 ? gj[g > 0 ? g - 1 : 0][1] : 0.f;       // slot 64 g - 1
      sm0 = g > 0 ? gm[g > 0 ? g - 1 : 0][1] : 0.f;
      sj1 = g + 1 < NG ? gj[g + 1 < NG ? g + 1 : g][0] : 0.f;   // slot 64 g + 64
      sm1 = g + 1 < NG ? gm[g + 1 < NG ? g + 1 : g][0] : 0.f;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int t = 64 * g + (h == 0 ? lane : 63 - lane);
      if (t < 1 || t >= a.nt) continue;
      const int m = (t + 1) >> 1;
      const float ct = ((t & 1) ? -c : c) * (float)m;
      store_bf16x3(ct * (h == 0 ? sj0 : sj1), Gp + row * a.k_pad + t, ps);
      if (jm != j) store_bf16x3(ct * (h == 0 ? sm0 : sm1), Gp + rowm * a.k_pad + t, ps);
    }
  }
  if (lane == 0) {
    a.add[3][row] = 0.f;
    if (jm != j) a.add[3][rowm] = 0.f;
  }
}

template <int S, bool STAGE>
size_t theta_smem(const yy_grid *g) {
  return ((size_t)3 * S + (STAGE ? 16 : 0)) * g->n_lm * sizeof(float);
}

// rows t of the azimuthal analysis table: dst[t][k] = az[k][t] (zero past nt)
__global__ void k_az_rows(int n_phi, int nt, int nt_src, int rows, const double *__restrict__ az,
                          double *__restrict__ dst) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * n_phi) return;
  const int t = e / n_phi, k = e - t * n_phi;
  dst[e] = t < nt ? az[(size_t)k * nt_src + t] : 0.0;
}

// colsum[t] = sum_k rows[t][k] (float64, fixed order), one block per row
__global__ void __launch_bounds__(256) k_row_total(int K, const double *__restrict__ rows, float *__restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) s += rows[(size_t)blockIdx.x * K + k];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = (float)red[0];
}

__global__ void k_fill_ones(int n, float *__restrict__ dst) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) dst[e] = 1.0f;
}

// rows k of the trig table: dst[k][t] = src[t][k]
__global__ void k_transpose_trig(int nt, int n_phi, const double *__restrict__ src, double *__restrict__ dst) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nt * n_phi) return;
  const int k = e / nt, t = e - k * nt;
  dst[e] = src[(size_t)t * n_phi + k];
}

// A[row][col] = (sum_z part[z][row][col]) row_scale col_scale + mean[row] colsum[col]
// (the tensor cores saw rho - mean); column 0 is the float64 monopole.
__global__ void k_reduce_partials(int M, int N, int S, const float *__restrict__ part,
                                  const double *__restrict__ rs, const double *__restrict__ cs,
                                  const double *__restrict__ mono, const double *__restrict__ mean,
                                  const double *__restrict__ colsum, double *__restrict__ A) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)M * N) return;
  const int row = (int)(e / N), col = (int)(e % N);
  if (col == 0) {
    A[e] = mono[row];
    return;
  }
  float s = 0.f, c = 0.f;
  for (int z = 0; z < S; ++z) kahan_add(s, c, part[(size_t)z * M * N + e]);
  const double sum = f32_to_f64(s) + f32_to_f64(c);
  A[e] = fma(sum * rs[row], cs[col], mean[row] * colsum[col]);
}

// degree l of mode index idx (l^2 <= idx < (l + 1)^2): fp32 square root and
// an integer correction
__device__ __forceinline__ int degree_of_mode(int idx) {
  int l = (int)sqrtf((float)idx);
  while (l * l > idx) --l;
  while ((l + 1) * (l + 1) <= idx) ++l;
  return l;
}

// The split-K sum of the analysis fused with the combination of the two
// patches' moments (Atot = A + D^T A(other patch), fp32 products as in the
// separate combination kernel).  Block (radius n, group of 256 modes): the
// moments of the degrees the group touches, both patches, are formed from the
// partials exactly as k_reduce_partials forms them (written to A for the
// group's own modes) and kept in shared memory; each thread then combines
// one mode.  Same values as the two kernels in sequence.
struct ReduceRotateArgs {
  int n_r, n_lm, S;             // radii, modes, segment partials
  const float *part;            // [S][2 n_r][n_lm]
  const double *rs, *cs, *mono, *mean, *colsum;
  const float *rot;             // per-degree rotation matrices
  double *A, *Atot;
};

// Block (n, group): radius n, modes [256 group, 256 group + 256) of both patches.
__device__ __forceinline__ void reduce_rotate_block(const ReduceRotateArgs &ra, int n, int group) {
  __shared__ double ad[2 * 640];   // two rows of at most 640 modes (group of 256 plus its degrees' ends)
  __shared__ float af[2 * 640];
  // the arguments in registers: the stores to A and Atot could otherwise alias them
  const ReduceRotateArgs r = ra;
  const int n_r = r.n_r, n_lm = r.n_lm;
  const int M = 2 * n_r;
  const int j0 = group * blockDim.x;
  const int j1 = min(n_lm, j0 + (int)blockDim.x);   // this group's modes [j0, j1)
  const int la = degree_of_mode(j0), lb = degree_of_mode(j1 - 1);
  const int m0 = la * la, m1 = (lb + 1) * (lb + 1), span = m1 - m0;
  const size_t zs = (size_t)M * n_lm;
  for (int e = threadIdx.x; e < 2 * span; e += blockDim.x) {
    const int p = e / span, c = m0 + e % span;
    const int row = p * n_r + n;
    const size_t idx = (size_t)row * n_lm + c;
    double v;
    if (c == 0) {
      v = r.mono[row];
    } else {
      float sum = 0.f, comp = 0.f;
#pragma unroll 4
      for (int z = 0; z < r.S; ++z) kahan_add(sum, comp, r.part[(size_t)z * zs + idx]);   // loads in flight, sums in order
      const double tot = f32_to_f64(sum) + f32_to_f64(comp);
      v = fma(tot * r.rs[row], r.cs[c], r.mean[row] * r.colsum[c]);
    }
    ad[p * span + (c - m0)] = v;
    af[p * span + (c - m0)] = f64_to_f32(v);
    if (c >= j0 && c < j1) r.A[idx] = v;
  }
  __syncthreads();
  const int j = j0 + (int)threadIdx.x;
  if (j >= j1) return;
  const int l = degree_of_mode(j);
  const int w = 2 * l + 1, jj = j - l * l;
  const float *D = r.rot + (size_t)l * (4 * l * l - 1) / 3 + jj;
  const float *x0 = af + (l * l - m0), *x1 = af + span + (l * l - m0);
  float s0 = 0.f, s1 = 0.f;   // into patch 0 (from patch 1) and into patch 1 (from patch 0)
#pragma unroll 4
  for (int i = 0; i < w; ++i) {   // all 2l + 1 terms (fp32: the loads, not the products, bound it)
    const float d = D[(size_t)i * w];
    s0 = fmaf(d, x1[i], s0);
    s1 = fmaf(d, x0[i], s1);
  }
  r.Atot[(size_t)n * n_lm + j] = ad[j - m0] + f32_to_f64(s0);
  r.Atot[((size_t)n_r + n) * n_lm + j] = ad[span + (j - m0)] + f32_to_f64(s1);
}

__global__ void __launch_bounds__(256) k_reduce_rotate(ReduceRotateArgs r) {
  reduce_rotate_block(r, (int)blockIdx.x, (int)blockIdx.y);
}


// Grouped packing: the rows of many jobs in one launch, each row as
// k_pack_reg<F, TPR, P> packs it.  Block b packs rows of job block_map[b] >> 24
// (its block block_map[b] & 0xFFFFFF, TPB / TPR rows per block), and
// pclass[j] picks the job's register form: P = 4, 8, 12 for TPR = 1024 (rows up to
// 8192, 16384, 24576 values), P = 4, 6, 12, 32 for TPR = 32 (up to 256, 384,
// 768, 2048).
template <class F, int TPR, int P>
__device__ __forceinline__ void pack_group_row(const PackArgs &p, int row, RowStats *red) {
  const int tid = threadIdx.x % TPR;
  const bool valid = row < p.rows && row != p.zero_row;
  const double *src = nullptr;
  if (valid) src = (row < p.split_row) ? p.src0 + (size_t)row * p.ld : p.src1 + (size_t)(row - p.split_row) * p.ld;
  const bool vec = ((uintptr_t)src & 15u) == 0;
  float x[2 * P];
  RowStats st;
  pack_load<TPR, P>(p, row, src, valid, vec, tid, x, st);
  pack_store<F, TPR, P>(p, row, src, valid, tid, x, st, red);
}

template <class F, int TPR>
__global__ void __launch_bounds__(TPR > 256 ? TPR : 256, 1)
k_pack_group(const PackArgs *__restrict__ jobs, const uint32_t *__restrict__ block_map,
             const unsigned char *__restrict__ pclass) {
  constexpr int TPB = TPR > 256 ? TPR : 256;
  __shared__ RowStats red[32];
  const uint32_t m = block_map[blockIdx.x];   // job << 24 | the job's own block
  const int j = (int)(m >> 24);
  const PackArgs &p = jobs[j];
  const int row = (int)(m & 0xFFFFFFu) * (TPB / TPR) + (int)threadIdx.x / TPR;
  if (row >= p.rows_pad) return;   // whole rows (and, for TPR > 32, whole blocks) leave together
  if constexpr (TPR > 32) {
    switch (pclass[j]) {
      case 0: pack_group_row<F, TPR, 4>(p, row, red); break;
      case 1: pack_group_row<F, TPR, 8>(p, row, red); break;
      default: pack_group_row<F, TPR, 12>(p, row, red); break;
    }
  } else {
    switch (pclass[j]) {
      case 0: pack_group_row<F, TPR, 4>(p, row, red); break;
      case 1: pack_group_row<F, TPR, 6>(p, row, red); break;
      case 2: pack_group_row<F, TPR, 12>(p, row, red); break;
      default: pack_group_row<F, TPR, 32>(p, row, red); break;
    }
  }
}

// The register form of a job for k_pack_group (-1: the row is too long).
static int pack_class(int tpr, int k_pad) {
  if (tpr > 32) return k_pad <= 1024 * 8 ? 0 : k_pad <= 1024 * 16 ? 1 : k_pad <= 1024 * 24 ? 2 : -1;
  return k_pad <= 32 * 8 ? 0 : k_pad <= 32 * 12 ? 1 : k_pad <= 32 * 24 ? 2 : k_pad <= 32 * 64 ? 3 : -1;
}

// All fields of a group: block_map[b] = field << 24 | the field's own block
// (n_r x ceil(n_lm / 256) of them).
__global__ void __launch_bounds__(256) k_reduce_rotate_group(const ReduceRotateArgs *__restrict__ fields,
                                                             const uint32_t *__restrict__ block_map) {
  const uint32_t m = block_map[blockIdx.x];
  const ReduceRotateArgs &r = fields[m >> 24];
  const int b = (int)(m & 0xFFFFFFu);
  reduce_rotate_block(r, b % r.n_r, b / r.n_r);
}

// colsum[row] = sum_k table[row][k] (float64, fixed order); b0[k] = fp32(table[0][k])
__global__ void __launch_bounds__(256) k_row_sums(int K, const double *__restrict__ table, double *__restrict__ out,
                                                  float *__restrict__ b0) {
  __shared__ double red[256];
  const double *src = table + (size_t)blockIdx.x * K;
  double s = 0.0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    s += src[k];
    if (blockIdx.x == 0) b0[k] = (float)src[k];
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void *ptr = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
  }
  return fn;
}

template <class F>
static bool make_map(CUtensorMap *map, void *base, int k_pad, int rows_total, int box_rows) {
  auto enc = get_encode();
  if (!enc) return false;
  const CUtensorMapDataType dt = (F::kKind == KIND_F16)    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                 : (F::kKind == KIND_BF16) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                           : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const cuuint64_t dims[2] = {(cuuint64_t)k_pad, (cuuint64_t)rows_total};
  const cuuint64_t strides[1] = {(cuuint64_t)k_pad * F::kElem};
  const cuuint32_t box[2] = {(cuuint32_t)(kRowBytes / F::kElem), (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, dt, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static int round_up(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace yy

struct yy_tc_tables {
  yy_precision prec;
  int pair_slots;                         // co-resident CTA pairs of the contraction kernel
  int bn, row_tiles, rows_pad;            // the 2 n_r rows (operand B) in tiles of bn
  int stages;                             // shared-memory stages of the contraction kernel
  // analysis: table rows (modes) as operand A, densities as operand B
  int an_kpad, an_modes_pad;
  void *an_tab, *an_rho;
  double *an_tabs, *an_rhos, *an_mono, *an_mean, *an_colsum;
  float *an_b0;                           // fp32 copy of the monopole row of the analysis table
  float *part;                            // K-segment partial sums [segment][2 n_r][n_lm]
  int an_splits, an_kb_per;               // K split: tiles along K, K blocks per tile (whole segments)
  int an_kb_total, an_splits_rule;        // K blocks; the rule's split count
  int an_segs, an_segs_per;               // K segments (one partial each); segments per split
  yy::PairMaps an_maps;                   // a[0]: table, b[0]: densities
  // synthesis: tables (cells) as operand A, coefficient sets as operand B
  int sy_kpad, sy_cells_pad;
  void *sy_q[3], *sy_tab[3];
  double *sy_qs[3], *sy_tabs[3];          // scales (float64 copies)
  float *sy_qsf[3], *sy_tabsf[3], *sy_add[3];
  yy::PairMaps sy_maps;                   // a: tables, b: coefficient sets
  // separable synthesis: G rows (shell, j) per field as operand A, the
  // cell-centre trig table (rows phi_k, slots t) as operand B, both as
  // three bf16 pieces whatever the requested form
  int sp_ok, sp_kpad, sp_rows, sp_rows_pad, sp_bn, sp_row_tiles, sp_b_rows_pad, sp_stages;
  void *sp_G[4], *sp_trig;
  float *sp_ones, *sp_ga[4], *sp_trigs_f;   // unit cell scales, slot-0 terms, trig row scales
  float *sp_inv_sin, *sp_inv_r;             // 1 / sin theta_j, 1 / r_(n+1) (g_phi of the polar stage)
  double *sp_trigs;
  yy::PairMaps sp_maps;                   // a[field]: G, b[0]: trig table
  // separable analysis: rows (shell, j) of rho w as operand A, the azimuthal
  // table (rows t, columns phi_k) as operand B
  int san_ok, san_kpad, san_rows, san_rows_pad, san_bn, san_stages;
  int sep_built;   // the separable tables above were built (each _ok says whether it is available)
  void *san_x, *san_az;
  double *san_rs, *san_mean, *san_F0, *san_azs;
  float *san_rsf, *san_azsf, *san_colsum, *san_ones, *san_part;
  yy::PairMaps san_maps;                  // a[0]: rho w rows, b[0]: table
};

// The dense analysis split into `splits` tiles along K, each of whole
// segments (splits <= an_segs).
static void set_an_splits(yy_tc_tables *t, int splits) {
  t->an_segs_per = (t->an_segs + splits - 1) / splits;
  t->an_splits = (t->an_segs + t->an_segs_per - 1) / t->an_segs_per;
  t->an_kb_per = (t->an_kb_total + t->an_splits - 1) / t->an_splits;   // about; the segments decide
}

namespace yy {

// Rows up to this many values are cached in shared memory by the two-pass packing.
constexpr int kPackCacheMax = 16 * 1024 / 4;
// k_reduce_rotate keeps two rows of at most 640 modes: a group of 256 modes
// plus the ends of its first and last degrees (2 (2 l + 1) <= 384 at l <= 95)
constexpr int kReduceRotateLmax = 80;

static size_t pack_smem(const PackBatch &b, int n) {
  size_t m = 0;
  for (int i = 0; i < n; ++i)
    if (b.job[i].cache) m = std::max(m, (size_t)b.job[i].K * sizeof(float));
  return m;
}

template <class F>
static cudaError_t launch_pack(PackBatch &b, int n, cudaStream_t s) {
  int rows = 0, kp = 0;
  for (int i = 0; i < n; ++i) {
    b.job[i].cache = b.job[i].K <= kPackCacheMax ? 1 : 0;
    rows = std::max(rows, b.job[i].rows_pad);
    kp = std::max(kp, b.job[i].k_pad);
  }
  // register-resident forms where the row fits, else the two-pass kernel
  const unsigned wblocks = (unsigned)((rows + 7) / 8);
  if (kp <= 32 * 8)
    k_pack_reg<F, 32, 4><<<dim3(wblocks, n), 256, 0, s>>>(b);
  else if (kp <= 32 * 12)
    k_pack_reg<F, 32, 6><<<dim3(wblocks, n), 256, 0, s>>>(b);
  else if (kp <= 32 * 24)
    k_pack_reg<F, 32, 12><<<dim3(wblocks, n), 256, 0, s>>>(b);
  else if (kp <= 32 * 64)
    k_pack_reg<F, 32, 32><<<dim3(wblocks, n), 256, 0, s>>>(b);
  else if (kp <= 1024 * 8)
    k_pack_reg<F, 1024, 4><<<dim3(rows, n), 1024, 0, s>>>(b);
  else if (kp <= 1024 * 16)
    k_pack_reg<F, 1024, 8><<<dim3(rows, n), 1024, 0, s>>>(b);
  else if (kp <= 1024 * 24)
    k_pack_reg<F, 1024, 12><<<dim3(rows, n), 1024, 0, s>>>(b);
  else
    k_pack_rows<F><<<dim3(rows, n), 256, pack_smem(b, n), s>>>(b);
  return cudaGetLastError();
}

// One job of long density rows: the streaming form where its rules hold
// (16-byte aligned rows of an even length, nothing left out), else
// launch_pack.
template <class F>
static cudaError_t launch_pack_long(PackBatch &b, int *err, cudaStream_t s) {
  const PackArgs &p = b.job[0];
  const bool fits = ((uintptr_t)p.src0 % 16) == 0 && ((uintptr_t)p.src1 % 16) == 0 && (p.ld % 2) == 0 &&
                    (p.K % 2) == 0 && p.wrow == nullptr && p.row_add == nullptr && p.zero_k0 < 0 &&
                    p.zero_k1 < 0 && p.zero_row < 0 && (p.dot_vec == nullptr || (uintptr_t)p.dot_vec % 8 == 0);
  if (!fits || p.K <= 32 * 64 || p.K > kStreamMaxK || p.k_pad > kStreamMaxK) return launch_pack<F>(b, 1, s);
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm < 1) n_sm = 1;
  const int grid = std::min(p.rows_pad, n_sm);
  k_pack_stream<F><<<grid, 1024, (size_t)p.K * sizeof(double), s>>>(p, err);
  return cudaGetLastError();
}

static cudaLaunchConfig_t pair_config(int pairs, int smem, cudaStream_t s, cudaLaunchAttribute *attr) {
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * pairs);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

template <class F>
static cudaError_t launch_pair(yy_grid *g, yy_tc_tables *t, const PairMaps &maps, const PairArgs &a, cudaStream_t s) {
  const int tiles = a.cell_tiles * a.row_tiles * a.k_splits * a.n_jobs;
  const int pairs = tiles < t->pair_slots ? tiles : t->pair_slots;
  cudaLaunchAttribute attr[1];
  const int smem = a.stages * pair_stage_bytes<F>(a.bn) + kSmemFixed + (a.out_mode >= 2 ? kEpiStageBytes : 0);
  cudaLaunchConfig_t cfg = pair_config(pairs, smem, s, attr);
  const cudaError_t e = a.out_mode == 2   ? cudaLaunchKernelEx(&cfg, k_tc_pair<F, 2>, maps, a)
                        : a.out_mode == 1 ? cudaLaunchKernelEx(&cfg, k_tc_pair<F, 1>, maps, a)
                                          : cudaLaunchKernelEx(&cfg, k_tc_pair<F, 0>, maps, a);
  note_launch(g, a.out_mode == 0 ? "k_tc_pair/split-K" : a.out_mode == 1 ? "k_tc_pair/synthesis" : "k_tc_pair/azimuthal", s);
  return e;
}

// Tables of the separable synthesis (out_mode 2): the trig table packed as
// operand B in three bf16 pieces (slot 0 left out: it is 1 at every phi_k and
// goes in per cell), unit cell scales, and the G operands of the four fields
// (rows past the last (shell, j) stay zero).  The azimuthal contraction is
// K = 2 l_max + 1 long, so its six products cost next to nothing whatever
// the requested form.
static yy_status prepare_separable_synthesis(yy_grid *g, yy_tc_tables *t) {
  typedef FormBF16x3 F;
  const int nt = 2 * g->lmax + 1;
  t->sp_kpad = round_up(nt, kPadK);
  t->sp_rows = grid_rows(g) * g->n_theta;
  t->sp_rows_pad = round_up(t->sp_rows, 2 * kPairRows);
  t->sp_row_tiles = (g->n_phi + 255) / 256;
  t->sp_bn = round_up((g->n_phi + t->sp_row_tiles - 1) / t->sp_row_tiles, 16);
  t->sp_b_rows_pad = t->sp_row_tiles * t->sp_bn;
  t->sp_stages = pair_stages<F>(t->sp_bn, kEpiStageBytes);
  if (t->sp_stages < 2) return YY_OK;   // not available: the dense synthesis stays
  // the polar stage keeps S shells' coefficients in shared memory
  if (cudaFuncSetAttribute(k_tc_pair<F, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit) != cudaSuccess ||
      cudaFuncSetAttribute(k_theta_g<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kThetaSmemMax) != cudaSuccess ||
      cudaFuncSetAttribute(k_theta_g<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kThetaSmemMax) != cudaSuccess ||
      cudaFuncSetAttribute(k_theta_g<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kThetaSmemMax) != cudaSuccess)
    return YY_ERR_NOT_SUPPORTED;
  if (nt > 128 && theta_smem<2, false>(g) > (size_t)kThetaSmemMax) return YY_OK;
  const size_t g_bytes = (size_t)F::kPA * t->sp_rows_pad * t->sp_kpad * F::kElem;
  cudaError_t e = cudaSuccess;
  auto A = [&](void **ptr, size_t bytes) {
    if (e == cudaSuccess) e = dmalloc(ptr, bytes);
  };
  for (int f = 0; f < 4; ++f) {
    A(&t->sp_G[f], g_bytes);
    A((void **)&t->sp_ga[f], t->sp_rows_pad * sizeof(float));
  }
  A((void **)&t->sp_ones, t->sp_rows_pad * sizeof(float));
  A(&t->sp_trig, (size_t)F::kPB * t->sp_b_rows_pad * t->sp_kpad * F::kElem);
  A((void **)&t->sp_trigs, t->sp_b_rows_pad * sizeof(double));
  A((void **)&t->sp_trigs_f, t->sp_b_rows_pad * sizeof(float));
  A((void **)&t->sp_inv_sin, g->n_theta * sizeof(float));
  A((void **)&t->sp_inv_r, g->n_r * sizeof(float));
  if (!g->Q32) A((void **)&g->Q32, 3 * (size_t)grid_rows(g) * g->n_lm * sizeof(float));   // the scan's fp32 copy
  double *trig_rows = nullptr;
  A((void **)&trig_rows, (size_t)g->n_phi * nt * sizeof(double));
  if (e != cudaSuccess) {
    if (trig_rows) cudaFree(trig_rows);
    return e == cudaErrorMemoryAllocation ? YY_ERR_OOM : YY_ERR_CUDA;
  }
  for (int f = 0; f < 4 && e == cudaSuccess; ++f) e = cudaMemset(t->sp_G[f], 0, g_bytes);
  if (e == cudaSuccess) {
    // the polar cell centres of the tables and the scan's 1 / r
    std::vector<float> is(g->n_theta), ir(g->n_r);
    std::vector<double> re(g->n_r + 1);
    for (int j = 0; j < g->n_theta; ++j) is[j] = (float)(1.0 / sin(g->th0 + g->dth * (j + 0.5)));
    e = cudaMemcpy(re.data(), g->r_edges, re.size() * sizeof(double), cudaMemcpyDeviceToHost);
    for (int n = 0; n < g->n_r; ++n) ir[n] = (float)(1.0 / re[n + 1]);
    if (e == cudaSuccess) e = cudaMemcpy(t->sp_inv_sin, is.data(), is.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(t->sp_inv_r, ir.data(), ir.size() * sizeof(float), cudaMemcpyHostToDevice);
  }
  k_fill_ones<<<(t->sp_rows_pad + 255) / 256, 256>>>(t->sp_rows_pad, t->sp_ones);
  k_transpose_trig<<<(nt * g->n_phi + 255) / 256, 256>>>(nt, g->n_phi, g->sep_tr, trig_rows);
  PackBatch b = {};
  PackArgs &p = b.job[0];
  p.rows = g->n_phi;
  p.rows_pad = t->sp_b_rows_pad;
  p.K = nt;
  p.k_pad = t->sp_kpad;
  p.src0 = p.src1 = trig_rows;
  p.split_row = g->n_phi;
  p.ld = nt;
  p.zero_k0 = 0;
  p.zero_k1 = -1;
  p.zero_row = -1;
  p.scale_out = t->sp_trigs;
  p.scale_out_f = t->sp_trigs_f;
  p.out = t->sp_trig;
  if (e == cudaSuccess) e = launch_pack<F>(b, 1, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(trig_rows);
  if (e != cudaSuccess) return YY_ERR_CUDA;
  bool ok = make_map<F>(&t->sp_maps.b[0], t->sp_trig, t->sp_kpad, F::kPB * t->sp_b_rows_pad, t->sp_bn / 2);
  for (int f = 0; f < 4 && ok; ++f)
    ok = make_map<F>(&t->sp_maps.a[f], t->sp_G[f], t->sp_kpad, F::kPA * t->sp_rows_pad, kPairRows);
  if (!ok) return YY_ERR_NOT_SUPPORTED;
  t->sp_ok = 1;
  return YY_OK;
}

// Tables of the separable analysis on the tensor cores: the azimuthal table
// packed as operand B (rows t; row 0, the constant d_phi, left out: its sums
// come from the packing's compensated row sums), its column sums for the
// centring, and the buffers of the weighted density rows.  Rows longer than
// the register-resident packing takes (2048) leave it unavailable.
template <class F>
static yy_status prepare_separable_analysis(yy_grid *g, yy_tc_tables *t) {
  const int nt = 2 * g->lmax + 1;
  t->san_kpad = round_up(g->n_phi, kPadK);
  t->san_rows = grid_rows(g) * g->n_theta;
  t->san_rows_pad = round_up(t->san_rows, 2 * kPairRows);
  t->san_bn = round_up(nt, 16);
  if (t->san_kpad > 32 * 64 || t->san_bn > 256 || !g->sep_az || !g->sep_w32 || !g->sep_tb32 ||
      separable_theta_partials_smem(g, t->san_bn) > 227 * 1024)
    return YY_OK;
  t->san_stages = pair_stages<F>(t->san_bn);
  cudaError_t e = cudaSuccess;
  auto A = [&](void **ptr, size_t bytes) {
    if (e == cudaSuccess) e = dmalloc(ptr, bytes);
  };
  const size_t rp = t->san_rows_pad;
  A(&t->san_x, (size_t)F::kPA * rp * t->san_kpad * F::kElem);
  A((void **)&t->san_rs, rp * sizeof(double));
  A((void **)&t->san_rsf, rp * sizeof(float));
  A((void **)&t->san_mean, rp * sizeof(double));
  A((void **)&t->san_F0, rp * sizeof(double));
  A(&t->san_az, (size_t)F::kPB * t->san_bn * t->san_kpad * F::kElem);
  A((void **)&t->san_azs, t->san_bn * sizeof(double));
  A((void **)&t->san_azsf, t->san_bn * sizeof(float));
  A((void **)&t->san_colsum, t->san_bn * sizeof(float));
  A((void **)&t->san_ones, g->n_phi * sizeof(float));
  A((void **)&t->san_part, (size_t)t->san_bn * rp * sizeof(float));
  double *az_rows = nullptr;
  A((void **)&az_rows, (size_t)t->san_bn * g->n_phi * sizeof(double));
  if (e != cudaSuccess) {
    if (az_rows) cudaFree(az_rows);
    return e == cudaErrorMemoryAllocation ? YY_ERR_OOM : YY_ERR_CUDA;
  }
  const int n_az = t->san_bn * g->n_phi;
  k_az_rows<<<(n_az + 255) / 256, 256>>>(g->n_phi, nt, g->sep_nt_pad, t->san_bn, g->sep_az, az_rows);
  k_row_total<<<t->san_bn, 256>>>(g->n_phi, az_rows, t->san_colsum);
  k_fill_ones<<<(g->n_phi + 255) / 256, 256>>>(g->n_phi, t->san_ones);
  PackBatch b = {};
  PackArgs &p = b.job[0];
  p.rows = t->san_bn;
  p.rows_pad = t->san_bn;
  p.K = g->n_phi;
  p.k_pad = t->san_kpad;
  p.src0 = p.src1 = az_rows;
  p.split_row = t->san_bn;
  p.ld = g->n_phi;
  p.zero_k0 = p.zero_k1 = -1;
  p.zero_row = 0;
  p.scale_out = t->san_azs;
  p.scale_out_f = t->san_azsf;
  p.out = t->san_az;
  if ((e = cudaGetLastError()) == cudaSuccess) e = launch_pack<F>(b, 1, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(az_rows);
  if (e != cudaSuccess) return YY_ERR_CUDA;
  const bool ok = make_map<F>(&t->san_maps.a[0], t->san_x, t->san_kpad, F::kPA * t->san_rows_pad, kPairRows) &&
                  make_map<F>(&t->san_maps.b[0], t->san_az, t->san_kpad, F::kPB * t->san_bn, t->san_bn / 2);
  if (!ok) return YY_ERR_NOT_SUPPORTED;
  t->san_ok = 1;
  return YY_OK;
}

template <class F>
static yy_status prepare_form(yy_grid *g, yy_tc_tables *t) {
  const int M = grid_rows(g);
  if (cudaFuncSetAttribute(k_tc_pair<F, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit) != cudaSuccess ||
      cudaFuncSetAttribute(k_tc_pair<F, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit) != cudaSuccess ||
      cudaFuncSetAttribute(k_pack_stream<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           kStreamMaxK * (int)sizeof(double)) != cudaSuccess)
    return YY_ERR_NOT_SUPPORTED;
  // the n_patch n_r rows: tiles of at most 256, each a multiple of 16
  t->row_tiles = (M + 255) / 256;
  t->bn = round_up((M + t->row_tiles - 1) / t->row_tiles, 16);
  t->rows_pad = t->row_tiles * t->bn;
  t->stages = pair_stages<F>(t->bn);
  {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = pair_config(64, t->stages * pair_stage_bytes<F>(t->bn) + kSmemFixed, 0, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (void *)k_tc_pair<F, 1>, &cfg) != cudaSuccess || n < 1) {
      cudaGetLastError();
      return YY_ERR_NOT_SUPPORTED;
    }
    t->pair_slots = n;
  }
  t->an_kpad = round_up(g->n_ang, kPadK);
  t->an_modes_pad = round_up(g->n_lm, 2 * kPairRows);
  t->sy_kpad = round_up(g->n_lm, kPadK);
  t->sy_cells_pad = round_up(g->n_ang, 2 * kPairRows);
  // split K of the analysis: about two tiles per CTA pair.  K is cut into
  // that many segments of (nearly) equal length, each summed in fills of
  // kAnalysisFill into its own partial; a split takes whole segments, so the
  // moments do not depend on it (coarser splits are the tuning range; finer
  // segments would cost a partial's traffic each at every split).
  const int an_tiles = (t->an_modes_pad / (2 * kPairRows)) * t->row_tiles;
  const int kb_total = t->an_kpad * F::kElem / kRowBytes;
  int splits = (2 * t->pair_slots + an_tiles / 2) / an_tiles;
  splits = splits < 1 ? 1 : (splits > kb_total ? kb_total : splits);
  t->an_kb_total = kb_total;
  t->an_segs = splits;
  set_an_splits(t, splits);
  t->an_splits_rule = t->an_splits;

  cudaError_t e = cudaSuccess;
  auto A = [&](void **ptr, size_t bytes) {
    if (e == cudaSuccess) e = dmalloc(ptr, bytes);
  };
  A(&t->an_tab, (size_t)F::kPA * t->an_modes_pad * t->an_kpad * F::kElem);
  A(&t->an_rho, (size_t)F::kPB * t->rows_pad * t->an_kpad * F::kElem);
  A((void **)&t->an_tabs, t->an_modes_pad * sizeof(double));
  A((void **)&t->an_rhos, t->rows_pad * sizeof(double));
  A((void **)&t->an_mono, t->rows_pad * sizeof(double));
  A((void **)&t->an_mean, t->rows_pad * sizeof(double));
  A((void **)&t->an_colsum, g->n_lm * sizeof(double));
  A((void **)&t->an_b0, g->n_ang * sizeof(float));
  A((void **)&t->part, (size_t)t->an_segs * M * g->n_lm * sizeof(float));
  for (int c = 0; c < 3; ++c) {
    A(&t->sy_q[c], (size_t)F::kPB * t->rows_pad * t->sy_kpad * F::kElem);
    A(&t->sy_tab[c], (size_t)F::kPA * t->sy_cells_pad * t->sy_kpad * F::kElem);
    A((void **)&t->sy_qs[c], t->rows_pad * sizeof(double));
    A((void **)&t->sy_tabs[c], t->sy_cells_pad * sizeof(double));
    A((void **)&t->sy_qsf[c], t->rows_pad * sizeof(float));
    A((void **)&t->sy_tabsf[c], t->sy_cells_pad * sizeof(float));
    A((void **)&t->sy_add[c], t->rows_pad * sizeof(float));
  }
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? YY_ERR_OOM : YY_ERR_CUDA;

  if (cudaFuncSetAttribute(k_pack_rows<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           kPackCacheMax * (int)sizeof(float)) != cudaSuccess)
    return YY_ERR_NOT_SUPPORTED;
  // static operands: the analysis table (mode 0 left out: done in float64)
  // and the three synthesis tables, each row scaled separately
  k_row_sums<<<g->n_lm, 256>>>(g->n_ang, g->ban, t->an_colsum, t->an_b0);
  if ((e = cudaGetLastError()) != cudaSuccess) return YY_ERR_CUDA;
  PackBatch b = {};
  PackArgs &p = b.job[0];
  p.rows = g->n_lm;
  p.rows_pad = t->an_modes_pad;
  p.K = g->n_ang;
  p.k_pad = t->an_kpad;
  p.src0 = p.src1 = g->ban;
  p.split_row = g->n_lm;
  p.ld = g->n_ang;
  p.zero_k0 = p.zero_k1 = -1;
  p.zero_row = 0;
  p.scale_out = t->an_tabs;
  p.out = t->an_tab;
  if ((e = launch_pack<F>(b, 1, 0)) != cudaSuccess) return YY_ERR_CUDA;
  const double *tabs[3] = {g->ysyn, g->ysyn_t, g->ysyn_p};
  PackBatch bs = {};
  for (int c = 0; c < 3; ++c) {
    PackArgs &q = bs.job[c];
    q.rows = g->n_ang;
    q.rows_pad = t->sy_cells_pad;
    q.K = g->n_lm;
    q.k_pad = t->sy_kpad;
    q.src0 = q.src1 = tabs[c];
    q.split_row = g->n_ang;
    q.ld = g->n_lm;
    q.zero_k0 = q.zero_k1 = -1;
    q.zero_row = -1;
    q.scale_out = t->sy_tabs[c];
    q.scale_out_f = t->sy_tabsf[c];
    q.out = t->sy_tab[c];
  }
  if ((e = launch_pack<F>(bs, 3, 0)) != cudaSuccess) return YY_ERR_CUDA;
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return YY_ERR_CUDA;

  const int bh = t->bn / 2;
  bool ok = make_map<F>(&t->an_maps.a[0], t->an_tab, t->an_kpad, F::kPA * t->an_modes_pad, kPairRows) &&
            make_map<F>(&t->an_maps.b[0], t->an_rho, t->an_kpad, F::kPB * t->rows_pad, bh);
  for (int c = 0; c < 3 && ok; ++c)
    ok = make_map<F>(&t->sy_maps.a[c], t->sy_tab[c], t->sy_kpad, F::kPA * t->sy_cells_pad, kPairRows) &&
         make_map<F>(&t->sy_maps.b[c], t->sy_q[c], t->sy_kpad, F::kPB * t->rows_pad, bh);
  if (!ok) return YY_ERR_NOT_SUPPORTED;
  return YY_OK;
}

// the tables of the separable tensor-core paths, built only while they are selected
static void release_separable(yy_tc_tables *t) {
  for (int f = 0; f < 4; ++f) {
    void *q[] = {t->sp_G[f], t->sp_ga[f]};
    for (void *p : q)
      if (p) cudaFree(p);
    t->sp_G[f] = nullptr;
    t->sp_ga[f] = nullptr;
  }
  void **sp[] = {&t->sp_trig, (void **)&t->sp_trigs_f, (void **)&t->sp_trigs, (void **)&t->sp_ones,
                 (void **)&t->sp_inv_sin, (void **)&t->sp_inv_r,
                 &t->san_x, &t->san_az, (void **)&t->san_rs, (void **)&t->san_mean, (void **)&t->san_F0,
                 (void **)&t->san_azs, (void **)&t->san_rsf, (void **)&t->san_azsf, (void **)&t->san_colsum,
                 (void **)&t->san_ones, (void **)&t->san_part};
  for (void **p : sp) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  t->sp_ok = t->san_ok = t->sep_built = 0;
}

static void free_tables(yy_tc_tables *t) {
  if (!t) return;
  void *ptrs[] = {t->an_tab, t->an_rho,    t->an_tabs, t->an_rhos, t->an_mono,
                  t->an_mean, t->an_colsum, t->an_b0,   t->part};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (int c = 0; c < 3; ++c) {
    void *q[] = {t->sy_q[c], t->sy_tab[c], t->sy_qs[c], t->sy_tabs[c], t->sy_qsf[c], t->sy_tabsf[c], t->sy_add[c]};
    for (void *p : q)
      if (p) cudaFree(p);
  }
  release_separable(t);
  delete t;
}

yy_status tc_prepare(yy_grid *g, yy_precision prec) {
  if (g->tc[prec]) return YY_OK;
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, g->device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, g->device);
  if (major != 10 || minor != 3) return YY_ERR_NOT_SUPPORTED;   // built for sm_103a only
  yy_tc_tables *t = new (std::nothrow) yy_tc_tables();
  if (!t) return YY_ERR_OOM;
  memset((void *)t, 0, sizeof(*t));
  t->prec = prec;
  yy_status st;
  switch (prec) {
    case YY_FP16X2: st = prepare_form<FormFP16x2>(g, t); break;
    case YY_BF16X3: st = prepare_form<FormBF16x3>(g, t); break;
    case YY_TF32: st = prepare_form<FormTF32>(g, t); break;
    default: st = YY_ERR_INVALID_ARG;
  }
  if (st != YY_OK) {
    cudaGetLastError();
    free_tables(t);
    return st;
  }
  g->tc[prec] = t;
  if (g->analysis_method == YY_ANALYSIS_SEPARABLE) return tc_build_separable(g, prec);
  return YY_OK;
}

yy_status tc_build_separable(yy_grid *g, yy_precision prec) {
  yy_tc_tables *t = ((int)prec >= 0 && (int)prec < 5) ? g->tc[prec] : nullptr;
  if (!t || t->sep_built) return YY_OK;   // not prepared, or already built
  yy_status st;
  switch (prec) {
    case YY_FP16X2: st = prepare_separable_analysis<FormFP16x2>(g, t); break;
    case YY_BF16X3: st = prepare_separable_analysis<FormBF16x3>(g, t); break;
    case YY_TF32: st = prepare_separable_analysis<FormTF32>(g, t); break;
    default: return YY_ERR_INVALID_ARG;
  }
  if (st == YY_OK) st = prepare_separable_synthesis(g, t);
  if (st != YY_OK) {
    cudaGetLastError();
    release_separable(t);
  } else {
    t->sep_built = 1;
  }
  return st;
}

void tc_release_separable(yy_grid *g, yy_precision prec) {
  yy_tc_tables *t = ((int)prec >= 0 && (int)prec < 5) ? g->tc[prec] : nullptr;
  if (!t) return;
  cudaDeviceSynchronize();   // nothing in flight may still read them
  release_separable(t);
}

void tc_free(yy_grid *g) {
  for (int i = 0; i < 5; ++i) {
    free_tables(g->tc[i]);
    g->tc[i] = nullptr;
  }
}

// The density packing and the contraction of the dense analysis.
template <class F>
static void analysis_args(yy_grid *g, yy_tc_tables *t, const double *ry, const double *rg, PackArgs &p, PairArgs &a) {
  const int M = grid_rows(g);
  p = PackArgs{};
  p.rows = M;
  p.rows_pad = t->rows_pad;
  p.K = g->n_ang;
  p.k_pad = t->an_kpad;
  p.src0 = ry;
  p.src1 = rg;
  p.split_row = g->n_r;
  p.ld = g->n_ang;
  p.zero_k0 = p.zero_k1 = -1;
  p.zero_row = -1;
  p.dot_vec = t->an_b0;         // monopole row of the analysis table
  p.dot_out = t->an_mono;
  p.mean_out = t->an_mean;      // the tensor cores see rho - (row mean)
  p.scale_out = t->an_rhos;
  p.out = t->an_rho;
  a = PairArgs{};
  a.stages = t->stages;
  a.cells = g->n_lm;
  a.cell_tiles = t->an_modes_pad / (2 * kPairRows);
  a.rows = M;
  a.row_tiles = t->row_tiles;
  a.bn = t->bn;
  a.kb_total = t->an_kpad * F::kElem / kRowBytes;
  a.k_splits = t->an_splits;
  a.kb_per_split = t->an_kb_per;
  a.kb_chunk = kAnalysisFill * F::kElem / kRowBytes;
  a.k_segs = t->an_segs;
  a.segs_per_split = t->an_segs_per;
  a.a_rows = t->an_modes_pad;
  a.b_rows = t->rows_pad;
  a.out_mode = 0;
  a.part = t->part;
  a.part_ld = g->n_lm;
  a.n_jobs = 1;
  a.err = g->err;
}

// The split-K sum and the combination of the patches (Yin-Yang grids up to
// l_max kReduceRotateLmax).
static void reduce_rotate_args(yy_grid *g, yy_tc_tables *t, ReduceRotateArgs &r) {
  r = ReduceRotateArgs{};
  r.n_r = g->n_r;
  r.n_lm = g->n_lm;
  r.S = t->an_segs;
  r.part = t->part;
  r.rs = t->an_rhos;
  r.cs = t->an_tabs;
  r.mono = t->an_mono;
  r.mean = t->an_mean;
  r.colsum = t->an_colsum;
  r.rot = g->rot32;
  r.A = g->A;
  r.Atot = g->Atot;
}

template <class F>
static cudaError_t analysis_form(yy_grid *g, yy_tc_tables *t, const double *ry, const double *rg, cudaStream_t s) {
  PackBatch b = {};
  PairArgs a;
  analysis_args<F>(g, t, ry, rg, b.job[0], a);
  cudaError_t e = launch_pack_long<F>(b, g->err, s);
  note_launch(g, "k_pack_stream", s);
  if (e != cudaSuccess) return e;
  if ((e = launch_pair<F>(g, t, t->an_maps, a, s)) != cudaSuccess) return e;
  if (g->n_patch == 2 && g->lmax <= kReduceRotateLmax) {
    // the split-K sum and the combination of the patches in one launch
    ReduceRotateArgs r;
    reduce_rotate_args(g, t, r);
    const dim3 grid((unsigned)g->n_r, (unsigned)((g->n_lm + 255) / 256));
    k_reduce_rotate<<<grid, 256, 0, s>>>(r);
    note_launch(g, "k_reduce_rotate", s);
    g->atot_done = 1;
    return cudaGetLastError();
  }
  const int M = grid_rows(g);
  const size_t cnt = (size_t)M * g->n_lm;
  k_reduce_partials<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(M, g->n_lm, t->an_segs, t->part, t->an_rhos,
                                                                  t->an_tabs, t->an_mono, t->an_mean, t->an_colsum,
                                                                  g->A);
  note_launch(g, "k_reduce_partials", s);
  return cudaGetLastError();
}

// The three coefficient sets' packing (Phi and g_r: the monopole, column 0,
// is added in the epilogue).
static void coefficient_args(yy_grid *g, yy_tc_tables *t, PackArgs (&jobs)[3]) {
  const int M = grid_rows(g);
  const size_t qsz = (size_t)M * g->n_lm;
  const double add[3] = {kY00, kY00, 0.0};
  for (int c = 0; c < 3; ++c) {
    PackArgs &p = jobs[c];
    p = PackArgs{};
    p.rows = M;
    p.rows_pad = t->rows_pad;
    p.K = g->n_lm;
    p.k_pad = t->sy_kpad;
    p.src0 = p.src1 = g->Q + c * qsz;
    p.split_row = M;
    p.ld = g->n_lm;
    p.zero_k0 = 0;
    p.zero_k1 = -1;
    p.zero_row = -1;
    p.add_factor = add[c];
    p.row_add = t->sy_add[c];
    p.scale_out = t->sy_qs[c];
    p.scale_out_f = t->sy_qsf[c];
    p.out = t->sy_q[c];
  }
}

template <class F>
static cudaError_t pack_coefficients_form(yy_grid *g, yy_tc_tables *t, cudaStream_t s) {
  PackBatch b = {};
  coefficient_args(g, t, b.job);
  cudaError_t e = launch_pack<F>(b, 3, s);
  note_launch(g, "k_pack_reg/coefficients", s);
  return e;
}

template <class F>
static void synthesis_args(yy_grid *g, yy_tc_tables *t, double *py, double *pg, double *gy, double *gg, PairArgs &a) {
  const size_t comp = (size_t)g->n_r * g->n_ang;
  // (coefficient set, table, outputs): Phi = Q.Y, g_r = Q_r.Y, g_theta = Q_t.Y_t, g_phi = Q_t.Y_p
  const struct {
    int q, tab;
    double *o0, *o1;
  } jobs[4] = {{0, 0, py, pg},
               {1, 0, gy, gg},
               {2, 1, gy ? gy + comp : nullptr, gg ? gg + comp : nullptr},
               {2, 2, gy ? gy + 2 * comp : nullptr, gg ? gg + 2 * comp : nullptr}};
  a = PairArgs{};
  a.stages = t->stages;
  a.cells = g->n_ang;
  a.cell_tiles = t->sy_cells_pad / (2 * kPairRows);
  a.rows = grid_rows(g);
  a.row_tiles = t->row_tiles;
  a.bn = t->bn;
  a.kb_total = t->sy_kpad * F::kElem / kRowBytes;
  a.k_splits = 1;
  a.kb_per_split = a.kb_total;
  a.a_rows = t->sy_cells_pad;
  a.b_rows = t->rows_pad;
  a.out_mode = 1;
  a.out_split = g->n_r;
  a.ldo = g->n_ang;
  a.n_jobs = gy ? 4 : 1;
  a.err = g->err;
  for (int j = 0; j < a.n_jobs; ++j) {
    PairJob &J = a.job[j];
    J.out0 = jobs[j].o0;
    J.out1 = jobs[j].o1;
    J.cell_scale = t->sy_tabsf[jobs[j].tab];
    J.row_scale = t->sy_qsf[jobs[j].q];
    J.row_add = t->sy_add[jobs[j].q];
    J.ta = jobs[j].tab;
    J.tb = jobs[j].q;
  }
}

template <class F>
static cudaError_t synthesis_form(yy_grid *g, yy_tc_tables *t, double *py, double *pg, double *gy, double *gg,
                                  cudaStream_t s) {
  PairArgs a;
  synthesis_args<F>(g, t, py, pg, gy, gg, a);
  return launch_pair<F>(g, t, t->sy_maps, a, s);
}

cudaError_t tc_analysis(yy_grid *g, yy_precision prec, const double *ry, const double *rg, cudaStream_t s) {
  yy_tc_tables *t = g->tc[prec];
  switch (prec) {
    case YY_FP16X2: return analysis_form<FormFP16x2>(g, t, ry, rg, s);
    case YY_BF16X3: return analysis_form<FormBF16x3>(g, t, ry, rg, s);
    case YY_TF32: return analysis_form<FormTF32>(g, t, ry, rg, s);
    default: return cudaErrorInvalidValue;
  }
}

static cudaError_t theta_form(yy_grid *g, yy_tc_tables *t, bool grad, cudaStream_t s) {
  if (t->sp_kpad <= 128 && g->Q32) {
    ThetaF32Args b = {};
    b.n_shells = grid_rows(g);
    b.n_theta = g->n_theta;
    b.n_r = g->n_r;
    b.lmax = g->lmax;
    b.n_lm = g->n_lm;
    b.nt = 2 * g->lmax + 1;
    b.k_pad = t->sp_kpad;
    b.n_jobs = grad ? 4 : 1;
    b.rows_pad = t->sp_rows_pad;
    b.Q32 = g->Q32;
    b.Q = g->Q;
    b.tab[0] = g->sep_P32;
    b.tab[1] = g->sep_dP32;
    b.tab[2] = g->sep_Qs32;
    b.tab64[0] = g->sep_P;
    b.tab64[1] = g->sep_dP;
    b.inv_sin = t->sp_inv_sin;
    b.inv_r = t->sp_inv_r;
    for (int f = 0; f < 4; ++f) {
      b.G[f] = t->sp_G[f];
      b.add[f] = t->sp_ga[f];
    }
    const size_t warps = (size_t)b.n_shells * ((g->n_theta + 1) / 2) * (grad ? 3 : 1);
    const unsigned blocks = (unsigned)((warps * 32 + 255) / 256);
    if (t->sp_kpad <= 64)
      k_theta_f32<1><<<blocks, 256, 0, s>>>(b);
    else
      k_theta_f32<2><<<blocks, 256, 0, s>>>(b);
    note_launch(g, "k_theta_f32", s);
    return cudaGetLastError();
  }
  ThetaArgs a = {};
  a.n_shells = grid_rows(g);
  a.n_theta = g->n_theta;
  a.lmax = g->lmax;
  a.n_lm = g->n_lm;
  a.nt = 2 * g->lmax + 1;
  a.k_pad = t->sp_kpad;
  a.n_jobs = grad ? 4 : 1;
  a.rows_pad = t->sp_rows_pad;
  a.Q = g->Q;
  a.tab[0] = g->sep_P32;
  a.tab[1] = g->sep_dP32;
  a.tab[2] = g->sep_Qs32;
  a.tab64[0] = g->sep_P;
  a.tab64[1] = g->sep_dP;
  for (int f = 0; f < 4; ++f) {
    a.G[f] = t->sp_G[f];
    a.add[f] = t->sp_ga[f];
  }
  // four shells per block and the table rows staged while they fit in shared memory
  if (theta_smem<4, true>(g) <= (size_t)kThetaSmemMax)
    k_theta_g<4, true><<<(a.n_shells + 3) / 4, 256, theta_smem<4, true>(g), s>>>(a);
  else if (theta_smem<2, true>(g) <= (size_t)kThetaSmemMax)
    k_theta_g<2, true><<<(a.n_shells + 1) / 2, 256, theta_smem<2, true>(g), s>>>(a);
  else
    k_theta_g<2, false><<<(a.n_shells + 1) / 2, 256, theta_smem<2, false>(g), s>>>(a);
  note_launch(g, "k_theta_g", s);
  return cudaGetLastError();
}

static cudaError_t sep_synthesis_form(yy_grid *g, yy_tc_tables *t, double *py, double *pg, double *gy, double *gg,
                                      cudaStream_t s) {
  typedef FormBF16x3 F;
  const size_t comp = (size_t)g->n_r * g->n_ang;
  double *o0[4] = {py, gy, gy ? gy + comp : nullptr, gy ? gy + 2 * comp : nullptr};
  double *o1[4] = {pg, gg, gg ? gg + comp : nullptr, gg ? gg + 2 * comp : nullptr};
  PairArgs a = {};
  a.stages = t->sp_stages;
  a.cells = t->sp_rows;
  a.cell_tiles = t->sp_rows_pad / (2 * kPairRows);
  a.rows = g->n_phi;
  a.row_tiles = t->sp_row_tiles;
  a.bn = t->sp_bn;
  a.kb_total = t->sp_kpad * F::kElem / kRowBytes;
  a.k_splits = 1;
  a.kb_per_split = a.kb_total;
  a.a_rows = t->sp_rows_pad;
  a.b_rows = t->sp_b_rows_pad;
  a.out_mode = 2;
  a.out_split = g->n_r * g->n_theta;
  a.ldo = g->n_phi;
  a.n_jobs = gy ? 4 : 1;
  a.err = g->err;
  for (int f = 0; f < a.n_jobs; ++f) {
    PairJob &J = a.job[f];
    J.out0 = o0[f];
    J.out1 = o1[f];
    J.cell_scale = t->sp_ones;
    J.cell_add = t->sp_ga[f];
    J.row_scale = t->sp_trigs_f;
    J.ta = f;
    J.tb = 0;
  }
  return launch_pair<F>(g, t, t->sp_maps, a, s);
}

int tc_analysis_splits(const yy_grid *g, yy_precision prec, int *rule, int *cap) {
  const yy_tc_tables *t = ((int)prec >= 0 && (int)prec < 5) ? g->tc[prec] : nullptr;
  if (!t) return 0;
  if (rule) *rule = t->an_splits_rule;
  if (cap) *cap = t->an_segs;
  return t->an_splits;
}

yy_status tc_set_analysis_splits(yy_grid *g, yy_precision prec, int splits) {
  yy_tc_tables *t = ((int)prec >= 0 && (int)prec < 5) ? g->tc[prec] : nullptr;
  if (!t) return YY_ERR_NOT_SUPPORTED;
  if (splits < 1 || splits > t->an_segs) return YY_ERR_INVALID_ARG;
  set_an_splits(t, splits);
  return YY_OK;
}

// Separable analysis on the tensor cores: the weighted density rows (shell,
// j) are centred, scaled and split by the packing (which also forms their
// compensated sums, slot 0), contracted with the azimuthal table (K = n_phi,
// raw fp32 sums), and the polar stage turns the sums into the moments.
template <class F>
static cudaError_t separable_analysis_form(yy_grid *g, yy_tc_tables *t, const double *ry, const double *rg,
                                           cudaStream_t s) {
  PackBatch b = {};
  PackArgs &p = b.job[0];
  p.rows = t->san_rows;
  p.rows_pad = t->san_rows_pad;
  p.K = g->n_phi;
  p.k_pad = t->san_kpad;
  p.src0 = ry;
  p.src1 = rg;
  p.split_row = g->n_r * g->n_theta;
  p.ld = g->n_phi;
  p.zero_k0 = p.zero_k1 = -1;
  p.zero_row = -1;
  p.dot_vec = t->san_ones;        // row sums (slot 0)
  p.dot_out = t->san_F0;
  p.mean_out = t->san_mean;
  p.scale_out = t->san_rs;
  p.scale_out_f = t->san_rsf;
  p.out = t->san_x;
  p.wrow = g->sep_w32;            // rho w
  p.w_rows = g->n_theta;
  cudaError_t e = launch_pack<F>(b, 1, s);
  note_launch(g, "k_pack_reg/rho_rows", s);
  if (e != cudaSuccess) return e;
  PairArgs a = {};
  a.stages = t->san_stages;
  a.cells = t->san_rows;
  a.cell_tiles = t->san_rows_pad / (2 * kPairRows);
  a.rows = 2 * g->lmax + 1;
  a.row_tiles = 1;
  a.bn = t->san_bn;
  a.kb_total = t->san_kpad * F::kElem / kRowBytes;
  a.k_splits = 1;
  a.kb_per_split = a.kb_total;
  a.kb_chunk = kAnalysisFill * F::kElem / kRowBytes;
  a.a_rows = t->san_rows_pad;
  a.b_rows = t->san_bn;
  a.out_mode = 0;
  a.part = t->san_part;
  a.part_ld = t->san_rows_pad;
  a.n_jobs = 1;
  a.err = g->err;
  if ((e = launch_pair<F>(g, t, t->san_maps, a, s)) != cudaSuccess) return e;
  SepThetaPartials th = {};
  th.nt_pad = t->san_bn;
  th.nt = 2 * g->lmax + 1;
  th.part = t->san_part;
  th.part_ld = t->san_rows_pad;
  th.row_scale = t->san_rsf;
  th.mean = t->san_mean;
  th.t_scale = t->san_azsf;
  th.colsum = t->san_colsum;
  th.F0 = t->san_F0;
  return separable_theta_partials(g, th, s);
}

bool tc_separable_analysis_ready(const yy_grid *g, yy_precision prec) {
  const yy_tc_tables *t = ((int)prec >= 0 && (int)prec < 5) ? g->tc[prec] : nullptr;
  return t && t->san_ok;
}

cudaError_t tc_separable_analysis(yy_grid *g, yy_precision prec, const double *ry, const double *rg, cudaStream_t s) {
  yy_tc_tables *t = g->tc[prec];
  switch (prec) {
    case YY_FP16X2: return separable_analysis_form<FormFP16x2>(g, t, ry, rg, s);
    case YY_BF16X3: return separable_analysis_form<FormBF16x3>(g, t, ry, rg, s);
    case YY_TF32: return separable_analysis_form<FormTF32>(g, t, ry, rg, s);
    default: return cudaErrorInvalidValue;
  }
}

bool tc_separable_synthesis_ready(const yy_grid *g, yy_precision prec) {
  const yy_tc_tables *t = ((int)prec >= 0 && (int)prec < 5) ? g->tc[prec] : nullptr;
  return t && t->sp_ok;
}

cudaError_t tc_theta(yy_grid *g, yy_precision prec, bool grad, cudaStream_t s) {
  return theta_form(g, g->tc[prec], grad, s);
}

cudaError_t tc_separable_synthesis(yy_grid *g, yy_precision prec, double *py, double *pg, double *gy, double *gg,
                                   cudaStream_t s) {
  return sep_synthesis_form(g, g->tc[prec], py, pg, gy, gg, s);
}

cudaError_t tc_pack_coefficients(yy_grid *g, yy_precision prec, cudaStream_t s) {
  yy_tc_tables *t = g->tc[prec];
  switch (prec) {
    case YY_FP16X2: return pack_coefficients_form<FormFP16x2>(g, t, s);
    case YY_BF16X3: return pack_coefficients_form<FormBF16x3>(g, t, s);
    case YY_TF32: return pack_coefficients_form<FormTF32>(g, t, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t tc_synthesis(yy_grid *g, yy_precision prec, double *py, double *pg, double *gy, double *gg,
                         cudaStream_t s) {
  yy_tc_tables *t = g->tc[prec];
  switch (prec) {
    case YY_FP16X2: return synthesis_form<FormFP16x2>(g, t, py, pg, gy, gg, s);
    case YY_BF16X3: return synthesis_form<FormBF16x3>(g, t, py, pg, gy, gg, s);
    case YY_TF32: return synthesis_form<FormTF32>(g, t, py, pg, gy, gg, s);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// float64 synthesis by the Ozaki scheme (YY_FP64_OZAKI)
// ---------------------------------------------------------------------------
//
// The separable synthesis with its azimuthal stage on the tensor cores at
// float64 accuracy: a float64 polar stage forms G[t] per output row (shell,
// j) and field and cuts each row into FormOzaki's six fixed-point slices
// under the row's power-of-two scale; k_tc_pair (out_mode 3) contracts them
// with the slices of the trig table (scaled by 1/2: cos 0 = 1 must lie inside
// (-1, 1)) over K = 2 l_max + 1 <= 127 (rows of 64 or 128 slots, one fill),
// exact per level, and rounds each value once.  The monopole slot t = 0 is
// part of the contraction: it is exact too.

// Balanced base-256 digits of X < 2^48 (most significant first): each
// digit taken in [-127, 128] with a carry into the next; the top one is at
// most 128 for X <= 2^47.
__host__ __device__ __forceinline__ void oz_digits(unsigned long long X, int (&d)[6]) {
#pragma unroll
  for (int s = 5; s > 0; --s) {
    int v = (int)(X & 255u);
    X >>= 8;
    if (v > 128) {
      v -= 256;
      X += 1;
    }
    d[s] = v;
  }
  d[0] = (int)X;
}

// ---- the polar stage in float-float arithmetic (k_q_ff, k_theta_ff) --------
//
// The polar stage of the synthesis, G[t] = sum_l Q[l^2 + t] T_j[l^2 + t]
// per output row (shell, j) and slot t (m = (t + 1) / 2), with the even / odd
// split over the mirrored rows (cells j and n_theta - 1 - j are reflections
// about the equator and P_l^m(-x) = (-1)^(l + m) P_l^m(x): with E and O the
// sums over even and odd l + m, row j gets E + O and its mirror E - O;
// dP/dtheta has the opposite parity), on the fp32 pipe in
// float-float arithmetic: a value is the unevaluated sum hi + lo of two fp32
// numbers (about 48 significant bits, the precision of the digits the sums
// are cut into next).  A product is exact as x + fma(a, b, -x) (Dekker's
// TwoProduct with a fused multiply-add), a sum as s + err (Knuth's TwoSum);
// the cross terms hi lo' + lo hi' go into the low part and lo lo' (2^-48 of
// the product) is dropped -- the accurate dot product of Ogita, Rump and
// Oishi (2005) with split inputs.  Every step is an explicitly rounded
// intrinsic or packed instruction (inline PTX with .rn) so that the compiler
// neither fuses nor reorders it.
//
// The stage is a small product per slot t (m = (t + 1) / 2): the polar table
// T_j[l, t] (rows j, l = m..l_max) times the coefficients Q[l, t] of every
// shell.  So a block takes 32 shells (the lanes: coefficient loads from a
// shell-minor copy of Q are coalesced) and TP mirrored row pairs (their
// table rows in shared memory: every lane of a warp reads the same entry),
// each warp the slots of one or two orders m with about the same number of
// terms (m and l_max + 1 - m), and stages the sums in shared memory; then
// each warp cuts whole rows into digits (lanes on slots 2 L and 2 L + 1: one
// 4-byte store per slice and lane), Phi's rows giving g_phi's as well.  The
// cos and sin slots of an order share their table value, so their
// multiply-adds run as one on the packed fp32 instructions (ff_fma_x2), the
// coefficients stored as slot pairs by k_q_ff.

// (hi, lo) of Q 2^-qexp per (field, shell), the scale from the row's largest
// |Q| (|Q| 2^-qexp < 1), in a shell-minor layout of the two slots of each
// (l, m) side by side: [field][l (l + 1) / 2 + m][shells_pad] as
// (hi_cos, hi_sin, lo_cos, lo_sin), the slots l^2 + 2m - 1 and l^2 + 2m
// (m = 0: the slot l^2 and zeros); entries below 2^-126 of the scale (and the
// padding shells) are zero.
struct OzQffArgs {
  int n_shells, shells_pad, lmax, n_lm, n_pm;
  int one_pass;                 // the block's 8 rows fit in dynamic shared memory
  const double *Q;              // [n_q][n_shells][n_lm]
  float4 *Qf;                   // [n_q][n_pm][shells_pad]
  int *qexp;                    // [n_q][n_shells]
};

// pairs (l, m), 0 <= m <= l <= lmax
__host__ __device__ constexpr int n_pm_of(int lmax) { return (lmax + 1) * (lmax + 2) / 2; }

// (l, m) of the triangular index pm = l (l + 1) / 2 + m, 0 <= m <= l
__device__ __forceinline__ void pm_decode(int pm, int &l, int &m) {
  int x = (int)((sqrtf(8.f * (float)pm + 1.f) - 1.f) * 0.5f);
  while (x > 0 && x * (x + 1) / 2 > pm) --x;
  while ((x + 1) * (x + 2) / 2 <= pm) ++x;
  l = x;
  m = pm - x * (x + 1) / 2;
}

// the slot pair of (l, m) from per-slot pairs, slot k at row[(k - k0) stride]
__device__ __forceinline__ float4 slot_pair(const float2 *row, int k0, int l, int m, int stride) {
  const int k = l * l + (m == 0 ? 0 : 2 * m - 1) - k0;
  const float2 c = row[(size_t)k * stride];
  const float2 sn = m == 0 ? make_float2(0.f, 0.f) : row[(size_t)(k + 1) * stride];
  return make_float4(c.x, sn.x, c.y, sn.y);
}

__device__ __forceinline__ float2 ff_split(double x, int qe) {
  const uint32_t lo = (uint32_t)__double2loint(x), hi = (uint32_t)__double2hiint(x);
  const int ex0 = (int)((hi >> 20) & 0x7FFu);
  const int ex = ex0 - qe;                             // biased exponent of x 2^-qe
  if (ex0 == 0 || ex < 897) return make_float2(0.f, 0.f);   // zero, subnormal, or below 2^-126 of the scale
  const double y = __hiloint2double((int)(hi - ((uint32_t)qe << 20)), (int)lo);   // |y| < 1: exact
  const float h = f64_to_f32_rn(y);
  // y - h: the 29 bits below h's last, less h's rounding step; times 2^(ex - 1075)
  const uint32_t r29 = lo & 0x1FFFFFFFu;
  const uint32_t m23 = (lo >> 29) & 1u;
  const int up = (r29 > 0x10000000u || (r29 == 0x10000000u && m23)) ? 1 : 0;
  const int r = (int)r29 - (up << 29);                 // |r| <= 2^28
  float l = __fmul_rn(__fmul_rn(__int2float_rn(r), __uint_as_float(63u << 23)),   // 2^-64
                      __uint_as_float((uint32_t)(ex - 1011 + 127) << 23));        // 2^(ex - 1011)
  if (hi >> 31) l = -l;
  return make_float2(h, l);
}

// One block per (field, 8 shells), two warps per shell: the row's scale,
// then its pairs, and the 8 rows written out shell-minor as 128-byte runs.
// Rows that fit in shared memory (one_pass) are read once: the loads of a
// lane all in flight, the values staged in place of their pairs, each warp
// of a row taking alternate 32-value pieces.  Longer rows take a warp each,
// in chunks of whole degrees through a shared tile.
constexpr int kQffShells = 8, kQffChunk = 512;
constexpr size_t kQffOnePassSmem = 200 * 1024;

__global__ void __launch_bounds__(512) k_q_ff(OzQffArgs a) {
  extern __shared__ float2 qrow[];                         // one_pass: [8][n_lm]; else [kQffChunk][8 + 1]
  __shared__ unsigned long long part[2][kQffShells];
  float2 (*tile)[kQffShells + 1] = reinterpret_cast<float2 (*)[kQffShells + 1]>(qrow);
  const int n_sb = a.shells_pad / kQffShells;
  const int f = (int)blockIdx.x / n_sb, s0 = ((int)blockIdx.x % n_sb) * kQffShells;
  const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
  const int r = warp % kQffShells, h = warp / kQffShells;  // the row, and which of its two warps
  const int s = s0 + r;
  const bool on = s < a.n_shells;
  const double *row = a.Q + ((size_t)f * a.n_shells + (on ? s : 0)) * a.n_lm;
  float4 *Qfb = a.Qf + (size_t)f * a.n_pm * a.shells_pad + s0;
  unsigned long long mb = 0ull;
  if (a.one_pass) {
    float2 *mine = qrow + (size_t)r * a.n_lm;
#pragma unroll 8
    for (int k = lane + 32 * h; k < a.n_lm; k += 64) {
      const double x = on ? row[k] : 0.0;
      mb = max(mb, (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull);
      mine[k] = *reinterpret_cast<const float2 *>(&x);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, off));
    if (lane == 0) part[h][r] = mb;
    __syncthreads();
    mb = max(part[0][r], part[1][r]);
    const int exm = (int)(mb >> 52);
    const int qe = exm == 0 ? 0 : exm - 1022;
    if (lane == 0 && h == 0 && on) a.qexp[(size_t)f * a.n_shells + s] = qe;
    for (int k = lane + 32 * h; k < a.n_lm; k += 64) {
      const float2 b = mine[k];
      mine[k] = ff_split(*reinterpret_cast<const double *>(&b), qe);
    }
    __syncthreads();
    // thread: shell c, pairs pm, pm + step, ...; (l, m) walked along
    const int c = (int)threadIdx.x % kQffShells, step = (int)blockDim.x / kQffShells;
    int pm = (int)threadIdx.x / kQffShells, l, m;
    pm_decode(pm, l, m);
    for (; pm < a.n_pm; pm += step) {
      Qfb[(size_t)pm * a.shells_pad + c] = slot_pair(qrow + (size_t)c * a.n_lm, 0, l, m, 1);
      for (m += step; m > l;) m -= ++l;
    }
    return;
  }
  int qe = 0;
  if (h == 0) {
    if (on)
      for (int k = lane; k < a.n_lm; k += 32)
        mb = max(mb, (unsigned long long)__double_as_longlong(row[k]) & 0x7FFFFFFFFFFFFFFFull);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, off));
    const int exm = (int)(mb >> 52);
    qe = exm == 0 ? 0 : exm - 1022;
    if (lane == 0 && on) a.qexp[(size_t)f * a.n_shells + s] = qe;
  }
  // degrees la..lb per chunk: their slots [la^2, (lb + 1)^2) and pairs
  // [la (la + 1) / 2, (lb + 1) (lb + 2) / 2)  (2 l_max + 1 <= kQffChunk)
  for (int la = 0; la <= a.lmax;) {
    int lb = la;
    while (lb < a.lmax && (lb + 2) * (lb + 2) - la * la <= kQffChunk) ++lb;
    const int k0 = la * la, kn = (lb + 1) * (lb + 1) - k0;
    if (h == 0)
      for (int k = lane; k < kn; k += 32) tile[k][r] = on ? ff_split(row[k0 + k], qe) : make_float2(0.f, 0.f);
    __syncthreads();
    const int p0 = la * (la + 1) / 2, pn = (lb + 1) * (lb + 2) / 2 - p0;
    for (int i = (int)threadIdx.x; i < pn * kQffShells; i += (int)blockDim.x) {
      const int pm = p0 + i / kQffShells, c = i % kQffShells;
      int l, m;
      pm_decode(pm, l, m);
      Qfb[(size_t)pm * a.shells_pad + c] = slot_pair(&tile[0][c], k0, l, m, kQffShells + 1);
    }
    __syncthreads();
    la = lb + 1;
  }
}

// acc += q p (q, p, acc float-float)
__device__ __forceinline__ void ff_fma(float2 q, float2 p, float2 &acc) {
  const float x = __fmul_rn(q.x, p.x);
  const float xe = __fmaf_rn(q.x, p.y, __fmaf_rn(q.y, p.x, __fmaf_rn(q.x, p.x, -x)));
  const float s = __fadd_rn(acc.x, x);
  const float bb = __fsub_rn(s, acc.x);
  const float err = __fadd_rn(__fsub_rn(acc.x, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  acc.y = __fadd_rn(acc.y, __fadd_rn(err, xe));
  acc.x = s;
}

// a + sg b, renormalised (|lo| <= half an ulp of hi)
__device__ __forceinline__ float2 ff_sum(float2 a, float2 b, float sg) {
  const float bx = sg * b.x, by = sg * b.y;
  const float s = __fadd_rn(a.x, bx);
  const float bb = __fsub_rn(s, a.x);
  const float err = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(bx, bb));
  const float lo = __fadd_rn(err, __fadd_rn(a.y, by));
  const float h = __fadd_rn(s, lo);
  return make_float2(h, __fsub_rn(lo, __fsub_rn(h, s)));
}

// Two float-float values at once, on the packed fp32 instructions (each
// half rounded exactly as the scalar instruction rounds it): a 64-bit
// register holds two fp32 numbers, the lower address's in its low half.
typedef unsigned long long ffx2;

__device__ __forceinline__ ffx2 mul_x2(ffx2 a, ffx2 b) {
  ffx2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ ffx2 fma_x2(ffx2 a, ffx2 b, ffx2 c) {
  ffx2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ ffx2 add_x2(ffx2 a, ffx2 b) {
  ffx2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ ffx2 sub_x2(ffx2 a, ffx2 b) {
  ffx2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ float x2_half(ffx2 a, int h) {
  return __uint_as_float(h ? (uint32_t)(a >> 32) : (uint32_t)a);
}
// (hi, hi), (lo, lo) of one float-float value
__device__ __forceinline__ ulonglong2 ff_dup(float2 v) {
  const ffx2 h = __float_as_uint(v.x), l = __float_as_uint(v.y);
  return make_ulonglong2((h << 32) | h, (l << 32) | l);
}

// (aH, aL) += q p for two slots at once, ff_fma's steps in its order: q =
// (hi of both slots, lo of both slots), qn_hi = -(q's hi), p = (hi, hi),
// (lo, lo) of one table value.  With xn = -x the error of the product is
// q_hi p_hi + xn, the sum a + x is a - xn, and x - bb is -(xn + bb): every
// rounding is the scalar one's (up to the sign of a zero low part).
__device__ __forceinline__ void ff_fma_x2(ulonglong2 q, ffx2 qn_hi, ulonglong2 p, ffx2 &aH, ffx2 &aL) {
  const ffx2 xn = mul_x2(qn_hi, p.x);
  const ffx2 xe = fma_x2(q.x, p.y, fma_x2(q.y, p.x, fma_x2(q.x, p.x, xn)));
  const ffx2 s = sub_x2(aH, xn);
  const ffx2 bb = sub_x2(s, aH);
  const ffx2 err = sub_x2(sub_x2(aH, sub_x2(s, bb)), add_x2(xn, bb));
  aL = add_x2(aL, add_x2(err, xe));
  aH = s;
}

// The balanced base-256 digits of 0 <= X <= 2^47 in one step: with
// Y = X + 127 (1 + 2^8 + ... + 2^32), the low five digits are Y's bytes less
// 127 (each in [-127, 128], the carries done by the addition) and the top
// one is Y >> 40.  Each digit comes out as the fp32 bit pattern of its
// value, whose upper half is the bf16 pattern (an integer below 2^8 in
// magnitude has sixteen zero low bits), most significant digit first:
// x_digit_pre gives the patterns of 2^23 + digit + 127 (the top one's of
// 2^23 + digit), from which one fp32 subtraction each leaves the digit.
__device__ __forceinline__ void x_digit_pre(unsigned long long X, uint32_t (&pre)[6]) {
  const unsigned long long Y = X + 0x7F7F7F7F7Full;
  const uint32_t ylo = (uint32_t)Y, yhi = (uint32_t)(Y >> 32);
  pre[0] = 0x4B000000u | (yhi >> 8);
  pre[1] = __byte_perm(yhi, 0x4B000000u, 0x7540);
  pre[2] = __byte_perm(ylo, 0x4B000000u, 0x7543);
  pre[3] = __byte_perm(ylo, 0x4B000000u, 0x7542);
  pre[4] = __byte_perm(ylo, 0x4B000000u, 0x7541);
  pre[5] = __byte_perm(ylo, 0x4B000000u, 0x7540);
}

__device__ __forceinline__ void x_digit_bits(unsigned long long X, uint32_t (&bits)[6]) {
  const unsigned long long Y = X + 0x7F7F7F7F7Full;
  const uint32_t ylo = (uint32_t)Y, yhi = (uint32_t)(Y >> 32);
  bits[0] = __float_as_uint(__fsub_rn(__uint_as_float(0x4B000000u | (yhi >> 8)), 8388608.f));
  bits[1] = __float_as_uint(__fsub_rn(__uint_as_float(__byte_perm(yhi, 0x4B000000u, 0x7540)), 8388735.f));
  bits[2] = __float_as_uint(__fsub_rn(__uint_as_float(__byte_perm(ylo, 0x4B000000u, 0x7543)), 8388735.f));
  bits[3] = __float_as_uint(__fsub_rn(__uint_as_float(__byte_perm(ylo, 0x4B000000u, 0x7542)), 8388735.f));
  bits[4] = __float_as_uint(__fsub_rn(__uint_as_float(__byte_perm(ylo, 0x4B000000u, 0x7541)), 8388735.f));
  bits[5] = __float_as_uint(__fsub_rn(__uint_as_float(__byte_perm(ylo, 0x4B000000u, 0x7540)), 8388735.f));
}

__device__ __forceinline__ ffx2 x2_pack(uint32_t lo, uint32_t hi) { return ((ffx2)hi << 32) | lo; }

// The digit patterns (x_digit_pre) of two float-float values (hi, lo) at
// once, both halves of each packed register: X = round(|value| 2^K), 2^K =
// p1 p2 the row's scale, as described below for ff_row.  The scalings by
// 2^-32 and 2^-16 are exact (or leave a sum of 1.5 2^23 that rounds to it
// either way), so each multiply-and-add is one fused operation.
__device__ __forceinline__ void ff_digit_pre_x2(ffx2 hi, ffx2 lo, ffx2 p1, ffx2 p2, uint32_t (&pre)[2][6]) {
  constexpr ffx2 kSign = 0x8000000080000000ull;
  constexpr ffx2 kM = 0x4B4000004B400000ull;             // 1.5 2^23 in both halves
  constexpr uint32_t kMBits = 0x4B400000u;
  const ffx2 sg = hi & kSign;
  const ffx2 A = mul_x2(mul_x2(hi ^ sg, p1), p2);        // |hi| 2^K
  const ffx2 B = mul_x2(mul_x2(lo ^ sg, p1), p2);        // +-lo 2^K, the sign of |value|
  const ffx2 s2 = fma_x2(A, 0x2F8000002F800000ull, kM);                              // A 2^-32 + M
  const ffx2 R1 = fma_x2(sub_x2(s2, kM), 0xCF800000CF800000ull, A);                  // A - T2 2^32
  const ffx2 s1 = fma_x2(R1, 0x3780000037800000ull, kM);                             // R1 2^-16 + M
  const ffx2 R2 = fma_x2(sub_x2(s1, kM), 0xC7800000C7800000ull, R1);                 // R1 - T1 2^16
  const ffx2 s0 = add_x2(add_x2(R2, B), kM);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const long long X = ((long long)(int)((uint32_t)(s2 >> (32 * h)) - kMBits) << 32) +
                        ((long long)(int)((uint32_t)(s1 >> (32 * h)) - kMBits) << 16) +
                        (long long)(int)((uint32_t)(s0 >> (32 * h)) - kMBits);
    x_digit_pre((unsigned long long)X, pre[h]);
  }
}

// the row scale of ff_row: 2^K with K = 48 - e as two normal fp32 factors
__device__ __forceinline__ void ff_row_scale(int e, float &p1, float &p2) {
  const int K = 48 - e, K1 = K >> 1, K2 = K - K1;
  p1 = __uint_as_float((uint32_t)(K1 + 127) << 23);
  p2 = __uint_as_float((uint32_t)(K2 + 127) << 23);
}

// The bias digits of output mode 4 in a lane's two slots of each 64-slot
// group (slots nt and nt + 1 hold G = 0): the top digit slice gets bf16 6144
// (kOzBiasG) at slot nt, the next one at slot nt + 1; zero without a bias.
template <int NG>
__device__ __forceinline__ void ff_bias_masks(int lane, int nt, int bias, uint32_t (&bmask)[NG][2]) {
  constexpr uint32_t kBiasBits = 0x45C0u;               // bf16 of kOzBiasG (6144)
#pragma unroll
  for (int g = 0; g < NG; ++g)
#pragma unroll
    for (int sl = 0; sl < 2; ++sl) {
      const int t = 64 * g + 2 * lane, tb = nt + sl;
      bmask[g][sl] = !bias ? 0u : (t == tb ? kBiasBits : 0u) | (t + 1 == tb ? kBiasBits << 16 : 0u);
    }
}

// One row of float-float values cut into digits: lane L holds slots
// 64 g + 2 L and 64 g + 2 L + 1.  The row's scale 2^e: the largest |hi|
// stepped up by one ulp bounds every |hi + lo| (|lo| is at most half an ulp),
// so every value is below 2^(e - 1).  X = round(|value| 2^(48 - e)) <= 2^47
// on the fp32 pipe, 16 bits at a time: A = |hi| 2^(48 - e) and B = +-lo
// 2^(48 - e) (exact power-of-two scalings), T2 = rint(A 2^-32), T1 =
// rint((A - T2 2^32) 2^-16) (the remainders exact by fused multiply-add), T0
// = rint(remainder + B), each rint by adding and removing 1.5 2^23 (whose
// bit pattern then holds the integer), X = T2 2^32 + T1 2^16 + T0.  The last
// addition rounds only where the remainder and B span more than 24 bits, so
// X is the nearest integer except within 2^-9 of a tie.  Then the balanced
// base-256 digits in one step: with Y = X + 127 (1 + 2^8 + ... + 2^32), the
// low five digits are Y's bytes less 127 (each in [-127, 128], the carries
// done by the addition) and the top one is Y >> 40.  qe: the power of two
// the values carry.
template <int NG>
__device__ __forceinline__ void ff_row(const float2 (&v)[NG][2], int lane, __nv_bfloat16 *dst, size_t stride,
                                       int *gexp, const uint32_t (&bmask)[NG][2], int qe) {
  uint32_t mb = 0u;
#pragma unroll
  for (int g = 0; g < NG; ++g)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t u = __float_as_uint(v[g][h].x) & 0x7FFFFFFFu;
      mb = max(mb, u == 0u ? 0u : u + 1u);
    }
  mb = __reduce_max_sync(0xffffffffu, mb);
  const int exm = (int)(mb >> 23);
  const int e = exm - 125;                              // every |value| < 2^(exm - 126) = 2^(e - 1)
  float p1, p2;
  ff_row_scale(e, p1, p2);
  const ffx2 p1x = x2_pack(__float_as_uint(p1), __float_as_uint(p1));
  const ffx2 p2x = x2_pack(__float_as_uint(p2), __float_as_uint(p2));
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    // the lane's two values, one in each half
    const uint32_t h0 = __float_as_uint(v[g][0].x), h1 = __float_as_uint(v[g][1].x);
    uint32_t pre[2][6];
    ff_digit_pre_x2(x2_pack(h0, h1), x2_pack(__float_as_uint(v[g][0].y), __float_as_uint(v[g][1].y)), p1x, p2x,
                    pre);
    const int t = 64 * g + 2 * lane;
    const uint32_t sm = ((h0 >> 31) << 15) | (h1 & 0x80000000u);
    uint32_t *d32 = reinterpret_cast<uint32_t *>(dst + t);
#pragma unroll
    for (int sl = 0; sl < 6; ++sl) {
      // 2^23 + 127 (the top digit: 2^23) off both halves: the digits' fp32 patterns
      const ffx2 d = sub_x2(x2_pack(pre[0][sl], pre[1][sl]), sl == 0 ? 0x4B0000004B000000ull : 0x4B00007F4B00007Full);
      uint32_t w = __byte_perm((uint32_t)d, (uint32_t)(d >> 32), 0x7632) ^ sm;
      if (sl < 2) w |= bmask[g][sl];                    // the bias digits (ff_bias_masks)
      d32[sl * (stride / 2)] = w;
    }
  }
  // value = 2^(e + qe + 1 - 64) (digit sums): trig scale 2^1, digit weights 2^-64
  if (lane == 0) *gexp = exm == 0 ? 0 : e + qe + 1 - 64;
}

struct OzThetaFFArgs {
  int n_shells, shells_pad, n_theta, half, lmax, n_lm, n_pm, nt, gphi, rows_pad, gk, n_r, bias;
  const float4 *Qf;             // [3][n_pm][shells_pad] (k_q_ff)
  const int *qexp;              // [3][n_shells]
  const float2 *Pf[2];          // [n_theta][n_lm]: P and dP/dtheta as (hi, lo)
  const double *inv_sin, *inv_r;
  __nv_bfloat16 *G[4];
  int *gexp[4];
};

// Shared memory of k_theta_ff: TP table rows of (l, m) entries (hi, hi, lo,
// lo), in float2 units, and the staged sums, 32 shells x (2 TP rows of gk
// slots + 1).
__host__ __device__ constexpr int theta_ff_tp(int gk) { return gk == 64 ? 2 : 1; }
__host__ __device__ inline int theta_ff_tab(int lmax, int gk) {
  return 2 * theta_ff_tp(gk) * ((lmax + 1) * (lmax + 2) / 2);
}
__host__ __device__ inline int theta_ff_pitch(int gk) { return 2 * theta_ff_tp(gk) * gk + 1; }
inline size_t theta_ff_smem(int lmax, int gk) {
  return ((size_t)theta_ff_tab(lmax, gk) + 32 * (size_t)theta_ff_pitch(gk)) * sizeof(float2);
}

// Blocks: (field, 32 shells, TP mirrored row pairs); warps: one or two
// orders m at a time (m and l_max + 1 - m, about 2 (l_max + 1) terms).
template <int NG>
__global__ void __launch_bounds__(512, 2) k_theta_ff(OzThetaFFArgs a) {
  constexpr int TP = NG == 1 ? 2 : 1;
  constexpr int R = 2 * TP;
  extern __shared__ float4 ffsm4[];
  float2 *const ffsm = reinterpret_cast<float2 *>(ffsm4);
  float4 *ptab = ffsm4;                                  // [TP][n_pm]: (hi, hi, lo, lo)
  float2 *stg = ffsm + theta_ff_tab(a.lmax, a.gk);       // [32][pitch]
  const int pitch = theta_ff_pitch(a.gk);
  const int W = (int)(blockDim.x >> 5), warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
  const int n_pt = (a.half + TP - 1) / TP, n_st = a.shells_pad >> 5;
  const int pt = (int)blockIdx.x % n_pt, st = ((int)blockIdx.x / n_pt) % n_st, f = (int)blockIdx.x / (n_pt * n_st);
  const int pair0 = pt * TP, shell0 = st * 32;
  const float2 *tsrc = f == 2 ? a.Pf[1] : a.Pf[0];
  // the table value of (l, m), the same in both of its slots, twice
  for (int i = (int)threadIdx.x; i < TP * a.n_pm; i += (int)blockDim.x) {
    const int r = i / a.n_pm;
    int l, m;
    pm_decode(i - r * a.n_pm, l, m);
    const float2 v = pair0 + r < a.half ? tsrc[(size_t)(pair0 + r) * a.n_lm + l * l + (m == 0 ? 0 : 2 * m - 1)]
                                        : make_float2(0.f, 0.f);
    ptab[i] = make_float4(v.x, v.x, v.y, v.y);
  }
  // the rows' scales, and g_phi's factor 1 / (r sin theta_j) as an fp32 pair
  __shared__ int qe_s[32];
  __shared__ float2 cphi[32][R];
  if (threadIdx.x < 32) {
    const int sh = shell0 + (int)threadIdx.x;
    qe_s[threadIdx.x] = sh < a.n_shells ? a.qexp[(size_t)f * a.n_shells + sh] : 0;
  }
  if (f == 0 && a.gphi)
    for (int i = (int)threadIdx.x; i < 32 * R; i += (int)blockDim.x) {
      const int sl = i / R, ri = i - sl * R;
      const int sh = shell0 + sl, p = pair0 + (ri >> 1);
      float2 c2 = make_float2(0.f, 0.f);
      if (sh < a.n_shells && p < a.half) {
        const int j = (ri & 1) ? a.n_theta - 1 - p : p;
        const double c = a.inv_r[sh % a.n_r] * a.inv_sin[j];
        const float ch = f64_to_f32_rn(c);
        c2 = make_float2(ch, f64_to_f32_rn(c - f32_to_f64(ch)));
      }
      cphi[sl][ri] = c2;
    }
  __syncthreads();
  const int L = a.lmax, n_groups = L / 2 + 1;
  const ulonglong2 *qf = reinterpret_cast<const ulonglong2 *>(a.Qf + (size_t)f * a.n_pm * a.shells_pad + shell0 + lane);
  const int qs = a.shells_pad;
  float2 *srow = stg + lane * pitch;
  constexpr ffx2 kSign2 = 0x8000000080000000ull;
  for (int gi = warp; gi < n_groups; gi += W) {
#pragma unroll 1
    for (int k = 0; k < 2; ++k) {
      int m;
      if (gi == 0) {
        if (k == 1 && !(L & 1)) break;
        m = k == 0 ? 0 : (L + 1) / 2;
      } else {
        m = k == 0 ? gi : L + 1 - gi;
      }
      const int t0 = m == 0 ? 0 : 2 * m - 1;
      const bool two_slots = m > 0;
      // both slots of m at once (m = 0: the second is zero); aH[i][0], aL[i][0]:
      // terms l = l_max, l_max - 2, ...; [1]: l = l_max - 1, ...
      ffx2 aH[TP][2], aL[TP][2];
#pragma unroll
      for (int i = 0; i < TP; ++i) aH[i][0] = aH[i][1] = aL[i][0] = aL[i][1] = 0ull;
      // terms l and l - 1 per step, the pairs index (l, m) -> l (l + 1) / 2 + m;
      // the next step's coefficients are loaded before this step's
      // multiply-adds.  Past the last term the same index steps stay in
      // [0, n_pm) (at l = m: b2 = m (m + 1) / 2, b1n = (m^2 - m + 2) / 2, b2n
      // = (m^2 - 3m + 6) / 2), so every load is unconditional; a value is
      // used only where its term exists.  (l_max = 0 reaches rows 1 and 3:
      // the allocation has four spare rows after the last field.)
      int b1 = L * (L + 1) / 2 + m;
      ulonglong2 q1 = qf[b1 * qs];
      ulonglong2 q2 = qf[(b1 - L) * qs];
#pragma unroll 1
      for (int l = L; l >= m; l -= 2) {
        const bool second = l - 1 >= m;
        const int b2 = b1 - l;                           // (l - 1, m)
        const int b1n = b2 - (l - 1);                    // (l - 2, m)
        const int b2n = b1n - (l - 2);                   // (l - 3, m)
        const ulonglong2 n1 = qf[b1n * qs];
        const ulonglong2 n2 = qf[b2n * qs];
        const ffx2 qn1 = q1.x ^ kSign2, qn2 = q2.x ^ kSign2;
#pragma unroll
        for (int i = 0; i < TP; ++i) {
          ff_fma_x2(q1, qn1, *reinterpret_cast<const ulonglong2 *>(ptab + i * a.n_pm + b1), aH[i][0], aL[i][0]);
          if (second)
            ff_fma_x2(q2, qn2, *reinterpret_cast<const ulonglong2 *>(ptab + i * a.n_pm + b2), aH[i][1], aL[i][1]);
        }
        q1 = n1;
        q2 = n2;
        b1 = b1n;
      }
      // row j: E + O = a0 + a1; row j': E - O, which is a0 - a1 when a0
      // holds the terms of even l + m (l_max + m even), else a1 - a0;
      // dP/dtheta has the opposite parity
      const float sg = (((L + m) & 1) ^ (f == 2 ? 1 : 0)) ? -1.f : 1.f;
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        if (s == 1 && !two_slots) break;
#pragma unroll
        for (int i = 0; i < TP; ++i) {
          const float2 a0 = make_float2(x2_half(aH[i][0], s), x2_half(aL[i][0], s));
          const float2 a1 = make_float2(x2_half(aH[i][1], s), x2_half(aL[i][1], s));
          srow[(2 * i) * a.gk + t0 + s] = ff_sum(a0, a1, 1.f);
          const float2 d = ff_sum(a0, a1, -1.f);
          srow[(2 * i + 1) * a.gk + t0 + s] = make_float2(sg * d.x, sg * d.y);
        }
      }
    }
  }
  __syncthreads();
  // rows: digits of each staged row; Phi's rows also give g_phi's from its
  // values: its coefficients are the angular set, -Q / r (r the shell's
  // outer edge), and its table m P / sin theta is m / sin theta times Phi's
  // P in the other slot of the same m, so
  //   G_phi[t] = (+1 for t even, -1 for t odd) (m / (r sin theta)) G_Phi[swap t]
  // (sin theta_j' = sin theta_j); slot 0 and the slots past nt are zero.
  const size_t stride = (size_t)a.rows_pad * a.gk;
  uint32_t bmask[NG][2];
  ff_bias_masks<NG>(lane, a.nt, a.bias, bmask);
  __nv_bfloat16 *const Gf = f == 0 ? a.G[0] : f == 1 ? a.G[1] : a.G[2];
  int *const gexp = f == 0 ? a.gexp[0] : f == 1 ? a.gexp[1] : a.gexp[2];
  for (int rr = warp; rr < 32 * R; rr += W) {
    const int sl = rr / R, ri = rr - sl * R;
    const int shell = shell0 + sl, p = pair0 + (ri >> 1);
    if (shell >= a.n_shells || p >= a.half) continue;
    const int j = (ri & 1) ? a.n_theta - 1 - p : p;
    if ((ri & 1) && j == p) continue;                    // the middle row is its own mirror
    const float2 *src = stg + sl * pitch + ri * a.gk;
    float2 v[NG][2];
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int t = 64 * g + 2 * lane + h;
        v[g][h] = t < a.nt ? src[t] : make_float2(0.f, 0.f);
      }
    const size_t row = (size_t)shell * a.n_theta + j;
    const int qe = qe_s[sl];
    ff_row<NG>(v, lane, Gf + row * a.gk, stride, gexp + row, bmask, qe);
    if (f != 0 || !a.gphi) continue;
    const float ch = cphi[sl][ri].x, cl = cphi[sl][ri].y;
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int t = 64 * g + 2 * lane + h;
        float2 w = make_float2(0.f, 0.f);
        if (t >= 1 && t < a.nt) {
          const float2 x = src[(t & 1) ? t + 1 : t - 1];
          const float mf = (float)((t + 1) >> 1);
          const float c0 = __fmul_rn(ch, mf);
          const float c1 = __fmaf_rn(cl, mf, __fmaf_rn(ch, mf, -c0));   // c m = c0 + c1
          const float y = __fmul_rn(x.x, c0);
          const float ye = __fmaf_rn(x.x, c1, __fmaf_rn(x.y, c0, __fmaf_rn(x.x, c0, -y)));
          const float hs = __fadd_rn(y, ye);
          w = make_float2(hs, __fsub_rn(ye, __fsub_rn(hs, y)));
          if (t & 1) w = make_float2(-w.x, -w.y);
        }
        v[g][h] = w;
      }
    ff_row<NG>(v, lane, a.G[3] + row * a.gk, stride, a.gexp[3] + row, bmask, qe);
  }
}

// The polar stage of the analysis in float-float arithmetic (the Ozaki
// path): A[lm] = sum_{j < ceil(n_theta / 2)} T_j[lm] (F_j + s F_j')[t], with
// s = +1 for even l + m and -1 for odd (the cell integrals of P_l^m sin theta
// have the parity of l + m; a middle row enters once), as in k_sep_theta.
// One block per shell: its F rows scaled by a power of two (the shell's
// largest |F| below 1) and split into fp32 pairs, the mirrored sums and
// differences formed in float-float and staged in shared memory, then one
// thread per mode with the pair-split table, both shells' multiply-adds as
// one on the packed fp32 instructions; the result widened to float64 and
// scaled back.
constexpr int kSepFFRegs = 8;    // mirrored (F_j, F_j') pairs per thread held in registers
constexpr int kSepFFShells = 2;  // shells per block: each table value read serves both halves of a pair
static_assert(kSepFFShells == 2, "k_sep_theta_ff packs its two shells into one fp32 pair");

__global__ void __launch_bounds__(512) k_sep_theta_ff(int n_shells, int n_theta, int n_lm, int nt, int nt_pad,
                                                      const float2 *__restrict__ tbf, const double *__restrict__ F,
                                                      double *__restrict__ A) {
  // [2][half][nt_pad]: S, then D, both shells' values as one packed pair
  // (hi of shell 0, hi of shell 1, lo of shell 0, lo of shell 1)
  extern __shared__ float4 sdf[];
  __shared__ unsigned long long red[16];
  __shared__ int qes[kSepFFShells];
  const int half = (n_theta + 1) >> 1;
  const int shell0 = (int)blockIdx.x * kSepFFShells;
  const int tid = (int)threadIdx.x, nthr = (int)blockDim.x;
  const int per_shell = 2 * half * nt_pad;
  // pair e = j nt + t (j < half, t < nt): F_j[t] and F_j'[t], all loads in
  // flight together when the shell fits in registers
  const int n_pairs = half * nt;
  const bool in_regs = n_pairs <= kSepFFRegs * nthr;
  for (int sh = 0; sh < kSepFFShells; ++sh) {
    // shell sh's value of entry e: components sh (hi) and 2 + sh (lo)
    float *sd = reinterpret_cast<float *>(sdf) + sh;
    if (shell0 + sh >= n_shells) {
      for (int e = tid; e < per_shell; e += nthr) sd[4 * e] = sd[4 * e + 2] = 0.f;
      continue;
    }
    const double *Fs = F + (size_t)(shell0 + sh) * n_theta * nt_pad;
    double fa[kSepFFRegs], fb[kSepFFRegs];
    unsigned long long mb = 0ull;
    if (in_regs) {
#pragma unroll
      for (int i = 0; i < kSepFFRegs; ++i) {
        const int e = tid + i * nthr;
        const int j = e / nt, t = e - j * nt, jm = n_theta - 1 - j;
        const bool ok = e < n_pairs;
        fa[i] = ok ? Fs[(size_t)j * nt_pad + t] : 0.0;
        fb[i] = ok && jm != j ? Fs[(size_t)jm * nt_pad + t] : 0.0;
      }
#pragma unroll
      for (int i = 0; i < kSepFFRegs; ++i)
        mb = max(mb, max((unsigned long long)__double_as_longlong(fa[i]) & 0x7FFFFFFFFFFFFFFFull,
                         (unsigned long long)__double_as_longlong(fb[i]) & 0x7FFFFFFFFFFFFFFFull));
    } else {
      for (int e = tid; e < n_pairs; e += nthr) {
        const int j = e / nt, t = e - j * nt, jm = n_theta - 1 - j;
        mb = max(mb, (unsigned long long)__double_as_longlong(Fs[(size_t)j * nt_pad + t]) & 0x7FFFFFFFFFFFFFFFull);
        mb = max(mb, (unsigned long long)__double_as_longlong(Fs[(size_t)jm * nt_pad + t]) & 0x7FFFFFFFFFFFFFFFull);
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, off));
    if ((tid & 31) == 0) red[tid >> 5] = mb;
    __syncthreads();
    mb = 0ull;
    for (int w = 0; w < (nthr >> 5); ++w) mb = max(mb, red[w]);
    const int exm = (int)(mb >> 52);
    const int qe = exm == 0 ? 0 : exm - 1022;              // |F| 2^-qe < 1
    if (tid == 0) qes[sh] = qe;
    if (in_regs) {
#pragma unroll
      for (int i = 0; i < kSepFFRegs; ++i) {
        const int e = tid + i * nthr;
        if (e >= n_pairs) continue;
        const int j = e / nt, t = e - j * nt, jm = n_theta - 1 - j;
        const float2 a = ff_split(fa[i], qe);
        float2 S = a, D = a;
        if (jm != j) {
          const float2 b = ff_split(fb[i], qe);
          S = ff_sum(a, b, 1.f);
          D = ff_sum(a, b, -1.f);
        }
        const int es = j * nt_pad + t, ed = (half + j) * nt_pad + t;
        sd[4 * es] = S.x;
        sd[4 * es + 2] = S.y;
        sd[4 * ed] = D.x;
        sd[4 * ed + 2] = D.y;
      }
    } else {
      for (int e = tid; e < n_pairs; e += nthr) {
        const int j = e / nt, t = e - j * nt, jm = n_theta - 1 - j;
        const float2 a = ff_split(Fs[(size_t)j * nt_pad + t], qe);
        float2 S = a, D = a;
        if (jm != j) {
          const float2 b = ff_split(Fs[(size_t)jm * nt_pad + t], qe);
          S = ff_sum(a, b, 1.f);
          D = ff_sum(a, b, -1.f);
        }
        const int es = j * nt_pad + t, ed = (half + j) * nt_pad + t;
        sd[4 * es] = S.x;
        sd[4 * es + 2] = S.y;
        sd[4 * ed] = D.x;
        sd[4 * ed + 2] = D.y;
      }
    }
    __syncthreads();                                         // red[] is read before the next shell writes it
  }
  for (int idx = tid; idx < n_lm; idx += nthr) {
    const int l = degree_of_mode(idx);
    const int t = idx - l * l;
    const int coff = ((((l + ((t + 1) >> 1)) & 1) != 0) ? half * nt_pad : 0) + t;
    const float2 *p = tbf + idx;
    const ulonglong2 *sq = reinterpret_cast<const ulonglong2 *>(sdf) + coff;
    ffx2 aH = 0ull, aL = 0ull;
#pragma unroll 8
    for (int j = 0; j < half; ++j) {
      const float2 tv = __ldg(p + (size_t)j * n_lm);
      const ulonglong2 q = sq[j * nt_pad];
      ff_fma_x2(q, q.x ^ 0x8000000080000000ull, ff_dup(tv), aH, aL);
    }
    float2 acc[kSepFFShells];
#pragma unroll
    for (int sh = 0; sh < kSepFFShells; ++sh) acc[sh] = make_float2(x2_half(aH, sh), x2_half(aL, sh));
#pragma unroll
    for (int sh = 0; sh < kSepFFShells; ++sh) {
      if (shell0 + sh >= n_shells) break;
      const int qe = qes[sh];
      double v = f32_to_f64(acc[sh].x) + f32_to_f64(acc[sh].y);
      // times 2^qe on the exponent field (a normal result), else by ldexp
      const unsigned long long u = (unsigned long long)__double_as_longlong(v);
      const int ex = (int)((u >> 52) & 0x7FFu);
      if (ex != 0) {
        if (ex + qe > 0 && ex + qe < 2047)
          v = __longlong_as_double((long long)(u + ((unsigned long long)(long long)qe << 52)));
        else
          v = ldexp(v, qe);
      }
      A[(size_t)(shell0 + sh) * n_lm + idx] = v;
    }
  }
}

// threads of k_sep_theta_ff: the modes in as few rounds of at most 512
// threads as possible, whole warps
static int sep_theta_ff_threads(int n_lm) {
  const int rounds = (n_lm + 511) / 512;
  const int per = (n_lm + rounds - 1) / rounds;
  return (per + 31) / 32 * 32;
}

// The other patch's moments in each frame (the combination of the two
// patches, as k_rotate_moments) in float-float arithmetic for the Ozaki path:
//   Atot[p][n][j] = A[p][n][j] + sum_i D^l_ij A[1-p][n][i],  i, j of degree l,
// the sum over the x-reflection parity class of j (the other class of D^l is
// zero).  Per radius and degree, both patches' moments are scaled by one
// power of two (the largest |A| of the degree below 1: D^l maps a degree
// onto itself) and split into fp32 pairs; the rotated sum is widened to
// float64, scaled back and added to the own moment.  One block per (degree,
// kRotRadii radii), the highest degrees first: D^l staged in shared memory
// once, a warp per radius stages the moments (raw, then their pairs in
// place), then a thread per (radius, mode) for both patches.
constexpr int kRotRadii = 4;

__global__ void __launch_bounds__(256) k_rotate_ff(int n_r, int n_lm, int lmax, const float2 *__restrict__ Df,
                                                   const double *__restrict__ A, double *__restrict__ Atot) {
  extern __shared__ float2 rsm[];                          // [w][w] D^l, then [kRotRadii][2 w] moment pairs
  __shared__ int rexp[kRotRadii];
  const int tiles = (n_r + kRotRadii - 1) / kRotRadii;
  const int l = lmax - (int)blockIdx.x / tiles;
  const int n0 = ((int)blockIdx.x % tiles) * kRotRadii;
  const int w = 2 * l + 1, base = l * l;
  const int tid = (int)threadIdx.x, nthr = (int)blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nw = nthr >> 5;
  const float2 *Dl = Df + (size_t)l * (4 * l * l - 1) / 3;
  for (int i = tid; i < w * w; i += nthr) rsm[i] = Dl[i];
  float2 *xs = rsm + w * w;
  for (int r = warp; r < kRotRadii; r += nw) {
    const int n = n0 + r;
    if (n >= n_r) continue;
    const double *a0 = A + (size_t)n * n_lm + base, *a1 = A + ((size_t)n_r + n) * n_lm + base;
    float2 *x = xs + r * 2 * w;
    unsigned long long mb = 0ull;
    for (int i = lane; i < 2 * w; i += 32) {
      const double v = i < w ? a0[i] : a1[i - w];
      mb = max(mb, (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull);
      x[i] = *reinterpret_cast<const float2 *>(&v);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, off));
    const int exm = (int)(mb >> 52);
    const int qe = exm == 0 ? 0 : exm - 1022;
    if (lane == 0) rexp[r] = qe;
    for (int i = lane; i < 2 * w; i += 32) {
      const float2 b = x[i];
      x[i] = ff_split(*reinterpret_cast<const double *>(&b), qe);
    }
  }
  __syncthreads();
  for (int o = tid; o < kRotRadii * w; o += nthr) {
    const int r = o / w, jj = o - r * w, n = n0 + r;
    if (n >= n_r) continue;
    const float2 *x0 = xs + r * 2 * w, *x1 = x0 + w;
    float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);   // into patch 0, into patch 1
    // the class of jj: index 0 and i % 4 in {2, 3} (even), or 1 and i % 4 in {0, 1}
    const bool even = jj == 0 || (jj & 3) >= 2;
    int i = even ? 0 : 1;
    {
      const float2 d = rsm[i * w + jj];
      ff_fma(x1[i], d, s0);
      ff_fma(x0[i], d, s1);
    }
#pragma unroll 2
    for (i = even ? 2 : 4; i < w; i += 4) {
      const float2 d = rsm[i * w + jj];
      ff_fma(x1[i], d, s0);
      ff_fma(x0[i], d, s1);
      if (i + 1 < w) {
        const float2 e = rsm[(i + 1) * w + jj];
        ff_fma(x1[i + 1], e, s0);
        ff_fma(x0[i + 1], e, s1);
      }
    }
    const int qe = rexp[r];
    double rr[2] = {f32_to_f64(s0.x) + f32_to_f64(s0.y), f32_to_f64(s1.x) + f32_to_f64(s1.y)};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      // times 2^qe on the exponent field (a normal result), else by ldexp
      const unsigned long long u = (unsigned long long)__double_as_longlong(rr[k]);
      const int ex = (int)((u >> 52) & 0x7FFu);
      if (ex != 0) {
        if (ex + qe > 0 && ex + qe < 2047)
          rr[k] = __longlong_as_double((long long)(u + ((unsigned long long)(long long)qe << 52)));
        else
          rr[k] = ldexp(rr[k], qe);
      }
    }
    const size_t j0 = (size_t)n * n_lm + base + jj, j1 = ((size_t)n_r + n) * n_lm + base + jj;
    Atot[j0] = A[j0] + rr[0];
    Atot[j1] = A[j1] + rr[1];
  }
}

// The weighted densities of the separable analysis, rho w, as digit rows for
// the analysis: one warp per row (shell, j); lane L takes the pairs
// k = 2 L + 64 c.  rho w is the float64 product of the CUDA-core path; the
// row's scale 2^e from its largest |rho w| (every value below 2^(e - 1)),
// the digits of X = round(|rho w| 2^(48 - e)) taken from the float64 bits,
// and the row exponent of a unit level-6 sum includes the table's scale 2^eb.
struct OzRhoArgs {
  int n_r, n_theta, n_phi, rows, k_pad, rows_pad, eb;
  const double *rho0, *rho1;    // [n_r][n_theta][n_phi] per patch (rho1 NULL on a polar grid)
  const double *w;              // [n_theta][n_phi]
  __nv_bfloat16 *X;             // [6][rows_pad][k_pad]
  int *rexp;                    // [rows_pad]
};

// C: 64-wide pieces of a row held per lane (k_pad <= 64 C).  Two cells'
// digits of one slice go out as one 32-bit store of their bf16 patterns.
template <int C>
__global__ void __launch_bounds__(256) k_rhow_ozaki(OzRhoArgs a) {
  const int row = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (row >= a.rows) return;
  const int shell = row / a.n_theta, j = row % a.n_theta;
  const int p = shell / a.n_r, i = shell % a.n_r;
  const double *rho = (p == 0 ? a.rho0 : a.rho1) + ((size_t)i * a.n_theta + j) * a.n_phi;
  const double *wj = a.w + (size_t)j * a.n_phi;
  unsigned long long bits[C][2];
  unsigned long long mb = 0ull;
  // an even n_phi keeps every row on a 16-byte boundary (the densities are
  // 16-byte aligned): a lane's two cells k, k + 1 in one load of each array
  const bool pairs = (a.n_phi & 1) == 0;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int k = 2 * lane + 64 * c;
    double v[2] = {0.0, 0.0};
    if (pairs) {
      if (k < a.n_phi) {
        const double2 r2 = *reinterpret_cast<const double2 *>(rho + k);
        const double2 w2 = *reinterpret_cast<const double2 *>(wj + k);
        v[0] = r2.x * w2.x;
        v[1] = r2.y * w2.y;
      }
    } else {
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (k + h < a.n_phi) v[h] = rho[k + h] * wj[k + h];
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      bits[c][h] = (unsigned long long)__double_as_longlong(v[h]);
      mb = max(mb, bits[c][h] & 0x7FFFFFFFFFFFFFFFull);
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, off));
  const int exm = (int)(mb >> 52);
  const int e = exm - 1021;
  const size_t stride = (size_t)a.rows_pad * a.k_pad;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int k0 = 2 * lane + 64 * c;
    if (k0 >= a.k_pad) break;
    uint32_t d[2][6];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int ex = (int)((bits[c][h] >> 52) & 0x7FFu);
      const int sh = 1027 - ex + e;
      unsigned long long X = 0;
      if (exm != 0 && ex != 0 && sh < 64)
        X = ((((bits[c][h] & 0xFFFFFFFFFFFFFull) | (1ull << 52)) >> (sh - 1)) + 1ull) >> 1;
      x_digit_bits(X, d[h]);
    }
    // the signs on the bf16 patterns
    const uint32_t sm = ((uint32_t)(bits[c][0] >> 63) << 15) | ((uint32_t)(bits[c][1] >> 63) << 31);
    uint32_t *dst = reinterpret_cast<uint32_t *>(a.X + (size_t)row * a.k_pad + k0);
#pragma unroll
    for (int sl = 0; sl < 6; ++sl) dst[sl * (stride / 2)] = __byte_perm(d[0][sl], d[1][sl], 0x7632) ^ sm;
  }
  if (lane == 0) a.rexp[row] = exm == 0 ? 0 : e + a.eb - 64;
}

}  // namespace yy

struct yy_oz_tables {
  int rows, rows_pad, bn, row_tiles, b_rows_pad, stages, pair_slots;
  int gk;                       // slots of a G row and of a trig digit row: 64 (l_max <= 31) or 128
  int bias;                     // synthesis with biased level sums (one fill): k_oz_synth
  int synth_slots;              // resident clusters of k_oz_synth (0: use k_tc_pair output mode 4)
  yy::OzSynthMaps synth_maps;   // its G maps (those of `maps`) and the trig map with 48-row boxes
  void *G[4];                   // per field: slices [6][rows_pad][64]
  int *gexp[4];                 // per field: [rows_pad]
  double *inv_sin, *inv_r;      // 1 / sin theta_j at the polar cell centres, 1 / r_(n+1) per shell
  int shells_pad;               // shells rounded up to 32 (k_theta_ff's tiles)
  float4 *Qf;                   // [3][n_pm][shells_pad]: scaled coefficients as fp32 pairs (k_q_ff)
  int *qexp;                    // [3][n_shells]: their scales
  float2 *Pf[2];                // [n_theta][n_lm]: P and dP/dtheta as fp32 pairs
  float2 *tbf;                  // [ceil(n_theta / 2)][n_lm]: the analysis table T as fp32 pairs
  float2 *Df;                   // [sum_l (2l+1)^2]: the rotation D^l as fp32 pairs (two patches)
  void *trig;                   // slices of trig / 2: [6][b_rows_pad][64]
  yy::PairMaps maps;
  // analysis (FormOzaki in fills of kFillK): rho w digit rows as operand A, the azimuthal table as operand B
  int an_ok, an_kpad, an_bn, an_row_tiles, an_b_rows_pad, an_stages, an_slots, an_eb;
  void *an_x;                   // [6][rows_pad][an_kpad]
  int *an_exp;                  // [rows_pad]
  void *an_az;                  // [6][an_b_rows_pad][an_kpad]
  yy::PairMaps an_maps;
  int an_slots2;                // resident clusters of k_oz_analysis (0: the pair kernel serves)
  yy::OzAnalysisMaps an_maps2;  // its maps: density digits (box 128 rows), table digits (box 32 rows)
};

namespace yy {

static void free_oz(yy_oz_tables *o) {
  if (!o) return;
  for (int f = 0; f < 4; ++f) {
    if (o->G[f]) cudaFree(o->G[f]);
    if (o->gexp[f]) cudaFree(o->gexp[f]);
  }
  if (o->trig) cudaFree(o->trig);
  if (o->inv_sin) cudaFree(o->inv_sin);
  if (o->inv_r) cudaFree(o->inv_r);
  if (o->Qf) cudaFree(o->Qf);
  if (o->qexp) cudaFree(o->qexp);
  for (int k = 0; k < 2; ++k)
    if (o->Pf[k]) cudaFree(o->Pf[k]);
  if (o->tbf) cudaFree(o->tbf);
  if (o->Df) cudaFree(o->Df);
  if (o->an_x) cudaFree(o->an_x);
  if (o->an_exp) cudaFree(o->an_exp);
  if (o->an_az) cudaFree(o->an_az);
  delete o;
}

void ozaki_free(yy_grid *g) {
  free_oz(g->oz);
  g->oz = nullptr;
}

bool ozaki_ready(const yy_grid *g) { return g->oz != nullptr; }

bool ozaki_analysis_ready(const yy_grid *g) { return g->oz != nullptr && g->oz->an_ok; }

// bf16 bits of a small integer (|v| <= 255: exact, the low 16 bits of the
// fp32 pattern are zero)
static uint16_t bf16_int(int v) {
  const float f = (float)v;
  uint32_t u;
  memcpy(&u, &f, 4);
  return (uint16_t)(u >> 16);
}

// Tables of the analysis by the Ozaki scheme; leaves an_ok = 0 (the float64
// analysis serves) where the rows are longer than four fills.
static yy_status ozaki_prepare_analysis(yy_grid *g, yy_oz_tables *o) {
  typedef FormOzaki F;
  const int nt = 2 * g->lmax + 1;
  if (g->n_phi > F::kFillK * F::kMaxFills || !g->sep_az || !g->sep_F) return YY_OK;
  o->an_kpad = round_up(g->n_phi, kPadK);
  o->an_bn = 32;   // seven level accumulators of bn columns within one 256-column TMEM buffer
  o->an_row_tiles = (nt + o->an_bn - 1) / o->an_bn;
  o->an_b_rows_pad = round_up(nt, kOzAnBN);   // tiles of an_bn (pair kernel) and kOzAnBN (k_oz_analysis)
  o->an_stages = pair_stages<F>(o->an_bn, kEpiStageBytes);
  if (o->an_stages < 2 ||
      cudaFuncSetAttribute(k_tc_pair<F, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit) != cudaSuccess)
    return YY_OK;
  {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg =
        pair_config(64, o->an_stages * pair_stage_bytes<F>(o->an_bn) + kSmemFixed + kEpiStageBytes, 0, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (void *)k_tc_pair<F, 3>, &cfg) != cudaSuccess || n < 1) {
      cudaGetLastError();
      return YY_OK;
    }
    o->an_slots = n;
  }
  cudaError_t e = cudaSuccess;
  auto A = [&](void **ptr, size_t bytes) {
    if (e == cudaSuccess) e = dmalloc(ptr, bytes);
  };
  const size_t x_bytes = (size_t)F::kPA * o->rows_pad * o->an_kpad * F::kElem;
  const size_t b_elems = (size_t)F::kPB * o->an_b_rows_pad * o->an_kpad;
  A(&o->an_x, x_bytes);
  A((void **)&o->an_exp, o->rows_pad * sizeof(int));
  A(&o->an_az, b_elems * F::kElem);
  if (e == cudaSuccess) e = cudaMemset(o->an_x, 0, x_bytes);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? YY_ERR_OOM : YY_ERR_CUDA;
  // the azimuthal table az[k][t] (rows of sep_nt_pad) as operand B, rows t:
  // one scale 2^eb for all of it (every row's largest value is about d_phi)
  const int ntp = g->sep_nt_pad;
  std::vector<double> az((size_t)g->n_phi * ntp);
  std::vector<uint16_t> sl(b_elems, 0);
  if (cudaMemcpy(az.data(), g->sep_az, az.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return YY_ERR_CUDA;
  double mx = 0.0;
  for (int k = 0; k < g->n_phi; ++k)
    for (int t = 0; t < nt; ++t) mx = fmax(mx, fabs(az[(size_t)k * ntp + t]));
  int E2 = 0;
  frexp(mx, &E2);   // mx < 2^E2
  o->an_eb = E2 + 1;
  for (int k = 0; k < g->n_phi && mx > 0.0; ++k)
    for (int t = 0; t < nt; ++t) {
      const double y = ldexp(az[(size_t)k * ntp + t], -o->an_eb);   // |y| < 1/2
      int d[6];
      oz_digits((unsigned long long)floor(ldexp(fabs(y), 48) + 0.5), d);
      for (int s2 = 0; s2 < F::kPB; ++s2)
        sl[((size_t)s2 * o->an_b_rows_pad + t) * o->an_kpad + k] = bf16_int(y < 0 ? -d[s2] : d[s2]);
    }
  if (cudaMemcpy(o->an_az, sl.data(), b_elems * F::kElem, cudaMemcpyHostToDevice) != cudaSuccess) return YY_ERR_CUDA;
  if (!make_map<F>(&o->an_maps.a[0], o->an_x, o->an_kpad, F::kPA * o->rows_pad, kPairRows) ||
      !make_map<F>(&o->an_maps.b[0], o->an_az, o->an_kpad, F::kPB * o->an_b_rows_pad, o->an_bn / 2))
    return YY_ERR_NOT_SUPPORTED;
  o->an_ok = 1;
  // the analysis kernel with all slots in one MMA
  o->an_slots2 = 0;
  if (nt <= kOzAnBN && make_map<F>(&o->an_maps2.a, o->an_x, o->an_kpad, F::kPA * o->rows_pad, kPairRows) &&
      make_map<F>(&o->an_maps2.b, o->an_az, o->an_kpad, F::kPB * o->an_b_rows_pad, kOzAnBN) &&
      cudaFuncSetAttribute(k_oz_analysis, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzAnSmem) == cudaSuccess) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = pair_config(64, kOzAnSmem, 0, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (void *)k_oz_analysis, &cfg) == cudaSuccess && n > 0) o->an_slots2 = n;
  }
  cudaGetLastError();
  return YY_OK;
}

// the polar stage of the analysis after the Ozaki azimuthal stage
static cudaError_t ozaki_theta_analysis(yy_grid *g, cudaStream_t s) {
  const int half = (g->n_theta + 1) / 2;
  const size_t smem = (size_t)kSepFFShells * 2 * half * g->sep_nt_pad * sizeof(float2);
  if (smem > 200 * 1024) return separable_theta_f64(g, s);
  const int shells = grid_rows(g);
  k_sep_theta_ff<<<(unsigned)((shells + kSepFFShells - 1) / kSepFFShells), sep_theta_ff_threads(g->n_lm), smem, s>>>(
      shells, g->n_theta, g->n_lm, 2 * g->lmax + 1, g->sep_nt_pad, g->oz->tbf, g->sep_F, g->A);
  note_launch(g, "k_sep_theta_ff", s);
  return cudaGetLastError();
}

cudaError_t ozaki_analysis(yy_grid *g, const double *ry, const double *rg, cudaStream_t s) {
  typedef FormOzaki F;
  yy_oz_tables *o = g->oz;
  OzRhoArgs ra = {};
  ra.n_r = g->n_r;
  ra.n_theta = g->n_theta;
  ra.n_phi = g->n_phi;
  ra.rows = o->rows;
  ra.k_pad = o->an_kpad;
  ra.rows_pad = o->rows_pad;
  ra.eb = o->an_eb;
  ra.rho0 = ry;
  ra.rho1 = rg;
  ra.w = g->w;
  ra.X = (__nv_bfloat16 *)o->an_x;
  ra.rexp = o->an_exp;
  const unsigned blocks = (unsigned)(((size_t)o->rows * 32 + 255) / 256);
  constexpr int kCmax = FormOzaki::kFillK * FormOzaki::kMaxFills / 64;
  if (o->an_kpad <= 64 * 5)
    k_rhow_ozaki<5><<<blocks, 256, 0, s>>>(ra);
  else
    k_rhow_ozaki<kCmax><<<blocks, 256, 0, s>>>(ra);
  note_launch(g, "k_rhow_ozaki", s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (o->an_slots2 > 0) {
    OzAnalysisArgs z = {};
    z.cells = o->rows;
    z.cell_tiles = o->rows_pad / (2 * kPairRows);
    z.cols = 2 * g->lmax + 1;
    z.kb_total = o->an_kpad * F::kElem / kRowBytes;
    z.kb_fill = F::kFillK * F::kElem / kRowBytes;   // exact level sums per fill; the epilogue adds the fills
    z.a_rows = o->rows_pad;
    z.b_rows = o->an_b_rows_pad;
    z.ldo = g->sep_nt_pad;
    z.out = g->sep_F;
    z.cell_exp = o->an_exp;
    z.err = g->err;
    const int pairs = z.cell_tiles < o->an_slots2 ? z.cell_tiles : o->an_slots2;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = pair_config(pairs, kOzAnSmem, s, attr);
    e = cudaLaunchKernelEx(&cfg, k_oz_analysis, o->an_maps2, z);
    note_launch(g, "k_oz_analysis", s);
    if (e != cudaSuccess) return e;
    return ozaki_theta_analysis(g, s);
  }
  PairArgs a = {};
  a.stages = o->an_stages;
  a.cells = o->rows;
  a.cell_tiles = o->rows_pad / (2 * kPairRows);
  a.rows = 2 * g->lmax + 1;
  a.row_tiles = o->an_row_tiles;
  a.bn = o->an_bn;
  a.kb_total = o->an_kpad * F::kElem / kRowBytes;
  a.kb_chunk = F::kFillK * F::kElem / kRowBytes;   // exact level sums per fill; the epilogue adds the fills
  a.k_splits = 1;
  a.kb_per_split = a.kb_total;
  a.a_rows = o->rows_pad;
  a.b_rows = o->an_b_rows_pad;
  a.out_mode = 3;
  a.out_split = o->rows;
  a.ldo = g->sep_nt_pad;
  a.n_jobs = 1;
  a.err = g->err;
  a.job[0].out0 = g->sep_F;
  a.job[0].out1 = g->sep_F;
  a.job[0].cell_exp = o->an_exp;
  a.job[0].ta = 0;
  a.job[0].tb = 0;
  const int tiles = a.cell_tiles * a.row_tiles;
  const int pairs = tiles < o->an_slots ? tiles : o->an_slots;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg =
      pair_config(pairs, o->an_stages * pair_stage_bytes<F>(o->an_bn) + kSmemFixed + kEpiStageBytes, s, attr);
  e = cudaLaunchKernelEx(&cfg, k_tc_pair<F, 3>, o->an_maps, a);
  note_launch(g, "k_tc_pair<FormOzaki,3>/analysis", s);
  if (e != cudaSuccess) return e;
  return ozaki_theta_analysis(g, s);
}

cudaError_t ozaki_rotate(yy_grid *g, cudaStream_t s) {
  if (g->n_patch == 1) return cudaSuccess;   // polar grid: the scans read A itself
  const int w = 2 * g->lmax + 1;
  const size_t smem = ((size_t)w * w + (size_t)kRotRadii * 2 * w) * sizeof(float2);
  const unsigned blocks = (unsigned)((g->lmax + 1) * ((g->n_r + kRotRadii - 1) / kRotRadii));
  k_rotate_ff<<<blocks, 256, smem, s>>>(g->n_r, g->n_lm, g->lmax, g->oz->Df, g->A, g->Atot);
  note_launch(g, "k_rotate_ff", s);
  return cudaGetLastError();
}

yy_status ozaki_prepare(yy_grid *g) {
  typedef FormOzaki F;
  if (g->oz) return YY_OK;
  const int nt = 2 * g->lmax + 1;
  if (nt > 2 * F::kMaxK || !g->sep_tr || !g->sep_P || !g->sep_dP || !g->sep_Qs) return YY_ERR_NOT_SUPPORTED;
  yy_oz_tables *o = new (std::nothrow) yy_oz_tables();
  if (!o) return YY_ERR_OOM;
  o->gk = nt <= F::kMaxK ? F::kMaxK : 2 * F::kMaxK;   // K of the synthesis contraction: one fill either way
  o->rows = grid_rows(g) * g->n_theta;
  o->rows_pad = round_up(o->rows, 2 * kPairRows);
  o->bn = 32;   // eight accumulators of bn columns fill one 256-column TMEM buffer
  o->row_tiles = (g->n_phi + o->bn - 1) / o->bn;
  // trig rows padded for both synthesis kernels: tiles of bn (k_tc_pair) and
  // of kOzSynthBN (k_oz_synth)
  o->b_rows_pad = round_up(g->n_phi, kOzSynthBN);
  o->stages = pair_stages<F>(o->bn, kEpiStageBytes);
  yy_status st = YY_OK;
  if (o->stages < 2 ||
      cudaFuncSetAttribute(k_tc_pair<F, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit) != cudaSuccess ||
      cudaFuncSetAttribute(k_tc_pair<F, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit) != cudaSuccess)
    st = YY_ERR_NOT_SUPPORTED;
  if (st == YY_OK) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg =
        pair_config(64, o->stages * pair_stage_bytes<F>(o->bn) + kSmemFixed + kEpiStageBytes, 0, attr);
    int n = 0, n4 = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (void *)k_tc_pair<F, 3>, &cfg) != cudaSuccess || n < 1 ||
        cudaOccupancyMaxActiveClusters(&n4, (void *)k_tc_pair<F, 4>, &cfg) != cudaSuccess || n4 < 1) {
      cudaGetLastError();
      st = YY_ERR_NOT_SUPPORTED;
    }
    o->pair_slots = n < n4 ? n : n4;
  }
  cudaError_t e = cudaSuccess;
  auto A = [&](void **ptr, size_t bytes) {
    if (e == cudaSuccess) e = dmalloc(ptr, bytes);
  };
  const size_t g_bytes = (size_t)F::kPA * o->rows_pad * o->gk * F::kElem;
  const size_t t_elems = (size_t)F::kPB * o->b_rows_pad * o->gk;
  if (st == YY_OK) {
    for (int f = 0; f < 4; ++f) {
      A(&o->G[f], g_bytes);
      A((void **)&o->gexp[f], o->rows_pad * sizeof(int));
    }
    A(&o->trig, t_elems * F::kElem);
    A((void **)&o->inv_sin, g->n_theta * sizeof(double));
    A((void **)&o->inv_r, g->n_r * sizeof(double));
    o->shells_pad = round_up(grid_rows(g), 32);
    // four spare rows: k_theta_ff's unconditional loads past a degree-0 row
    A((void **)&o->Qf, ((size_t)3 * n_pm_of(g->lmax) + 4) * o->shells_pad * sizeof(float4));
    A((void **)&o->qexp, (size_t)3 * grid_rows(g) * sizeof(int));
    for (int k = 0; k < 2; ++k) A((void **)&o->Pf[k], (size_t)g->n_theta * g->n_lm * sizeof(float2));
    A((void **)&o->tbf, (size_t)((g->n_theta + 1) / 2) * g->n_lm * sizeof(float2));
    if (g->n_patch == 2) A((void **)&o->Df, rotation_table_size(g->lmax) * sizeof(float2));
    for (int f = 0; f < 4 && e == cudaSuccess; ++f) e = cudaMemset(o->G[f], 0, g_bytes);
    if (e == cudaSuccess) {
      // g_phi's polar factors (k_theta_ff): the same cell centres as the
      // tables and the same 1 / r as the scan coefficients
      std::vector<double> is(g->n_theta), ir(g->n_r), re(g->n_r + 1);
      for (int j = 0; j < g->n_theta; ++j) is[j] = 1.0 / sin(g->th0 + g->dth * (j + 0.5));
      e = cudaMemcpy(re.data(), g->r_edges, re.size() * sizeof(double), cudaMemcpyDeviceToHost);
      for (int n = 0; n < g->n_r; ++n) ir[n] = 1.0 / re[n + 1];
      if (e == cudaSuccess) e = cudaMemcpy(o->inv_sin, is.data(), is.size() * sizeof(double), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(o->inv_r, ir.data(), ir.size() * sizeof(double), cudaMemcpyHostToDevice);
      // the polar tables as fp32 pairs: hi = fl32(x), lo = fl32(x - hi)
      const size_t ne = (size_t)g->n_theta * g->n_lm;
      std::vector<double> tb(ne);
      std::vector<float2> tf(ne);
      const double *tsrc[4] = {g->sep_P, g->sep_dP, g->tbar, g->rot};
      float2 *tdst[4] = {o->Pf[0], o->Pf[1], o->tbf, o->Df};
      const size_t tn[4] = {ne, ne, (size_t)((g->n_theta + 1) / 2) * g->n_lm,
                            g->n_patch == 2 ? (size_t)rotation_table_size(g->lmax) : (size_t)0};
      const size_t tmax = std::max(ne, tn[3]);
      tb.resize(tmax);
      tf.resize(tmax);
      for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
        if (tn[k] == 0) continue;
        e = cudaMemcpy(tb.data(), tsrc[k], tn[k] * sizeof(double), cudaMemcpyDeviceToHost);
        for (size_t i = 0; i < tn[k]; ++i) {
          const float h = (float)tb[i];
          tf[i] = make_float2(h, (float)(tb[i] - (double)h));
        }
        if (e == cudaSuccess) e = cudaMemcpy(tdst[k], tf.data(), tn[k] * sizeof(float2), cudaMemcpyHostToDevice);
      }
      if (e == cudaSuccess)
        e = cudaMemset(o->Qf, 0, ((size_t)3 * n_pm_of(g->lmax) + 4) * o->shells_pad * sizeof(float4));
      // the largest dynamic shared memory of any supported degree (l_max 63),
      // the same for every grid
      const int ff_max = (int)theta_ff_smem(63, 128);
      if (e == cudaSuccess &&
          (cudaFuncSetAttribute(k_theta_ff<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, ff_max) != cudaSuccess ||
           cudaFuncSetAttribute(k_theta_ff<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, ff_max) != cudaSuccess ||
           cudaFuncSetAttribute(k_sep_theta_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess ||
           cudaFuncSetAttribute(k_rotate_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess ||
           cudaFuncSetAttribute(k_q_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kQffOnePassSmem) != cudaSuccess))
        e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) st = e == cudaErrorMemoryAllocation ? YY_ERR_OOM : YY_ERR_CUDA;
  }
  if (st == YY_OK) {
    // trig digits on the host: y = trig / 2, |y| <= 1/2, X = round(|y| 2^48)
    // (exact: |y| 2^48 < 2^52), balanced digits with the sign of y
    std::vector<double> tr((size_t)nt * g->n_phi);
    std::vector<uint16_t> sl(t_elems, 0);
    if (cudaMemcpy(tr.data(), g->sep_tr, tr.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      st = YY_ERR_CUDA;
    // output mode 4 needs two spare K columns and |S_L| < 2^22 for every
    // level and longitude: |S_L| <= 128 sum over the level's products (s, u)
    // of sum_t |trig digit u at t| (G digits are at most 128 in magnitude)
    bool bias = nt + 2 <= o->gk;
    for (int k = 0; k < g->n_phi && st == YY_OK; ++k) {
      long long asum[6] = {0, 0, 0, 0, 0, 0};
      for (int t = 0; t < nt; ++t) {
        const double y = tr[(size_t)t * g->n_phi + k] * 0.5;
        int d[6];
        oz_digits((unsigned long long)floor(ldexp(fabs(y), 48) + 0.5), d);
        for (int s2 = 0; s2 < F::kPB; ++s2) {
          sl[((size_t)s2 * o->b_rows_pad + k) * o->gk + t] = bf16_int(y < 0 ? -d[s2] : d[s2]);
          asum[s2] += d[s2] < 0 ? -d[s2] : d[s2];
        }
      }
      for (int L = 0; L < F::kAccs; ++L) {
        long long b = 0;
        for (int s2 = F::s_lo(L); s2 <= (L < 5 ? L : 5); ++s2) b += asum[L - s2];
        if (128 * b >= (1ll << 22)) bias = false;
      }
    }
    if (bias) {
      // the trig side of the bias columns: 2^11 in every slice at nt, in slice 5 at nt + 1
      const uint16_t two11 = bf16_int(2048);   // a power of two: exact in bf16
      for (int k = 0; k < o->b_rows_pad; ++k) {
        for (int s2 = 0; s2 < F::kPB; ++s2) sl[((size_t)s2 * o->b_rows_pad + k) * o->gk + nt] = two11;
        sl[((size_t)5 * o->b_rows_pad + k) * o->gk + nt + 1] = two11;
      }
    }
    o->bias = bias ? 1 : 0;
    if (st == YY_OK && cudaMemcpy(o->trig, sl.data(), t_elems * F::kElem, cudaMemcpyHostToDevice) != cudaSuccess)
      st = YY_ERR_CUDA;
  }
  if (st == YY_OK) {
    bool ok = make_map<F>(&o->maps.b[0], o->trig, o->gk, F::kPB * o->b_rows_pad, o->bn / 2);
    for (int f = 0; f < 4 && ok; ++f)
      ok = make_map<F>(&o->maps.a[f], o->G[f], o->gk, F::kPA * o->rows_pad, kPairRows);
    if (!ok) st = YY_ERR_NOT_SUPPORTED;
  }
  if (st == YY_OK && o->bias && o->gk == kOzSynthKB * 32) {
    // the synthesis kernel with the G tile resident (falls back to the pair
    // kernel's output mode 4 where it cannot run)
    int n = 0;
    for (int f = 0; f < 4; ++f) o->synth_maps.a[f] = o->maps.a[f];
    if (make_map<F>(&o->synth_maps.b, o->trig, o->gk, F::kPB * o->b_rows_pad, kOzSynthBN / 2) &&
        cudaFuncSetAttribute(k_oz_synth, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSynthSmem) == cudaSuccess) {
      cudaLaunchAttribute attr[1];
      cudaLaunchConfig_t cfg = pair_config(64, kOzSynthSmem, 0, attr);
      if (cudaOccupancyMaxActiveClusters(&n, (void *)k_oz_synth, &cfg) != cudaSuccess) n = 0;
    }
    cudaGetLastError();
    o->synth_slots = n > 0 ? n : 0;
  }
  if (st == YY_OK) st = ozaki_prepare_analysis(g, o);
  if (st != YY_OK) {
    cudaGetLastError();
    free_oz(o);
    return st;
  }
  g->oz = o;
  return YY_OK;
}

cudaError_t ozaki_synthesis(yy_grid *g, double *py, double *pg, double *gy, double *gg, cudaStream_t s) {
  typedef FormOzaki F;
  yy_oz_tables *o = g->oz;
  const int n_jobs = gy ? 4 : 1;
  const int n_shells = grid_rows(g);
  // the coefficients as scaled fp32 pairs, then the polar stage of Phi, g_r
  // and g_theta (Phi's blocks also write g_phi)
  const int n_q = n_jobs == 4 ? 3 : 1;
  OzQffArgs qa = {};
  qa.n_shells = n_shells;
  qa.shells_pad = o->shells_pad;
  qa.lmax = g->lmax;
  qa.n_lm = g->n_lm;
  qa.n_pm = n_pm_of(g->lmax);
  qa.Q = g->Q;
  qa.Qf = o->Qf;
  qa.qexp = o->qexp;
  const size_t qff_smem = (size_t)kQffShells * g->n_lm * sizeof(float2);
  qa.one_pass = qff_smem <= kQffOnePassSmem ? 1 : 0;
  k_q_ff<<<(unsigned)(n_q * (o->shells_pad / kQffShells)), 64 * kQffShells,
           qa.one_pass ? qff_smem : (size_t)kQffChunk * (kQffShells + 1) * sizeof(float2), s>>>(qa);
  note_launch(g, "k_q_ff", s);
  OzThetaFFArgs fa = {};
  fa.n_shells = n_shells;
  fa.shells_pad = o->shells_pad;
  fa.n_theta = g->n_theta;
  fa.half = (g->n_theta + 1) / 2;
  fa.lmax = g->lmax;
  fa.n_lm = g->n_lm;
  fa.n_pm = n_pm_of(g->lmax);
  fa.nt = 2 * g->lmax + 1;
  fa.gphi = n_jobs == 4 ? 1 : 0;
  fa.rows_pad = o->rows_pad;
  fa.gk = o->gk;
  fa.n_r = g->n_r;
  fa.bias = o->bias;
  fa.Qf = o->Qf;
  fa.qexp = o->qexp;
  fa.Pf[0] = o->Pf[0];
  fa.Pf[1] = o->Pf[1];
  fa.inv_sin = o->inv_sin;
  fa.inv_r = o->inv_r;
  for (int f = 0; f < 4; ++f) {
    fa.G[f] = (__nv_bfloat16 *)o->G[f];
    fa.gexp[f] = o->gexp[f];
  }
  const int n_groups = g->lmax / 2 + 1, tp = theta_ff_tp(o->gk);
  const unsigned ff_blocks = (unsigned)(n_q * (o->shells_pad / 32) * ((fa.half + tp - 1) / tp));
  const unsigned ff_threads = (unsigned)(32 * (n_groups < 16 ? n_groups : 16));
  const size_t ff_smem = theta_ff_smem(g->lmax, o->gk);
  if (o->gk == 64)
    k_theta_ff<1><<<ff_blocks, ff_threads, ff_smem, s>>>(fa);
  else
    k_theta_ff<2><<<ff_blocks, ff_threads, ff_smem, s>>>(fa);
  note_launch(g, "k_theta_ff", s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t comp = (size_t)g->n_r * g->n_ang;
  double *o0[4] = {py, gy, gy ? gy + comp : nullptr, gy ? gy + 2 * comp : nullptr};
  double *o1[4] = {pg, gg, gg ? gg + comp : nullptr, gg ? gg + 2 * comp : nullptr};
  if (o->bias && o->synth_slots > 0) {
    OzSynthArgs z = {};
    z.cells = o->rows;
    z.cell_tiles = o->rows_pad / (2 * kPairRows);
    z.cols = g->n_phi;
    z.col_tiles = o->b_rows_pad / kOzSynthBN;
    z.a_rows = o->rows_pad;
    z.b_rows = o->b_rows_pad;
    z.out_split = g->n_r * g->n_theta;
    z.ldo = g->n_phi;
    z.n_jobs = n_jobs;
    z.prefetch = 1;
    z.err = g->err;
    for (int f = 0; f < n_jobs; ++f) {
      z.job[f].out0 = o0[f];
      z.job[f].out1 = o1[f];
      z.job[f].cell_exp = o->gexp[f];
    }
    const int tiles = z.cell_tiles * n_jobs;
    const int pairs = tiles < o->synth_slots ? tiles : o->synth_slots;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = pair_config(pairs, kOzSynthSmem, s, attr);
    e = cudaLaunchKernelEx(&cfg, k_oz_synth, o->synth_maps, z);
    note_launch(g, "k_oz_synth", s);
    return e;
  }
  PairArgs a = {};
  a.stages = o->stages;
  a.cells = o->rows;
  a.cell_tiles = o->rows_pad / (2 * kPairRows);
  a.rows = g->n_phi;
  a.row_tiles = o->row_tiles;
  a.bn = o->bn;
  a.kb_total = o->gk * F::kElem / kRowBytes;   // one fill (level sums below 2^24 up to K = 160)
  a.k_splits = 1;
  a.kb_per_split = a.kb_total;
  a.a_rows = o->rows_pad;
  a.b_rows = o->b_rows_pad;
  a.out_mode = o->bias ? 4 : 3;
  a.out_split = g->n_r * g->n_theta;
  a.ldo = g->n_phi;
  a.n_jobs = n_jobs;
  a.err = g->err;
  for (int f = 0; f < n_jobs; ++f) {
    PairJob &J = a.job[f];
    J.out0 = o0[f];
    J.out1 = o1[f];
    J.cell_exp = o->gexp[f];
    J.ta = f;
    J.tb = 0;
  }
  const int tiles = a.cell_tiles * a.row_tiles * n_jobs;
  const int pairs = tiles < o->pair_slots ? tiles : o->pair_slots;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = pair_config(pairs, o->stages * pair_stage_bytes<F>(o->bn) + kSmemFixed + kEpiStageBytes, s, attr);
  e = o->bias ? cudaLaunchKernelEx(&cfg, k_tc_pair<F, 4>, o->maps, a) : cudaLaunchKernelEx(&cfg, k_tc_pair<F, 3>, o->maps, a);
  note_launch(g, "k_tc_pair<FormOzaki,3>/synthesis", s);
  return e;
}

// ---------------------------------------------------------------------------
// grouped solves: one launch per stage over many fields (batched workload)
// ---------------------------------------------------------------------------
//
// Every field solved densely in a tensor-core form: the density packing, the
// analysis contraction, the split-K sum with the patches' combination, the
// radial scans, the coefficient packing and the synthesis, each one launch
// over all fields.  The per-field arguments are those of the field's own
// solve (the same tiles, K segments, fills and arithmetic, so the results are
// the same bit for bit); they live in one device buffer built here, with the
// fields' tensor maps for the grouped contractions.

struct TcGroup {
  yy_precision prec;
  int n;
  void *dev;                          // every table below
  // density rows: long and even (streamed), other long ones (1024 threads a row), short ones (a warp a row)
  PackArgs *st_jobs, *rho_jobs, *rs_jobs, *cf_jobs;
  uint32_t *st_map;                                        // per row: job << 24 | the job's own row
  uint32_t *rho_map, *rs_map, *cf_map, *rr_map, *sc_map;   // per block: job << 24 | the job's own block
  int st_rows, st_grid, st_smem;
  unsigned char *rho_class, *rs_class, *cf_class;
  PairArgs *an_args, *sy_args;
  PairMaps *an_maps, *sy_maps;
  ReduceRotateArgs *rr;
  ScanGroupField *sc;
  int rho_nblocks, rs_nblocks, cf_nblocks, rr_nblocks, sc_nblocks;
  PairArgs an_top, sy_top;            // kernel arguments of the grouped contractions
  int an_pairs, sy_pairs, an_smem, sy_smem;
};

// blocks of job j, appended to a block map
static void map_blocks(std::vector<uint32_t> &map, int j, int blocks) {
  for (int b = 0; b < blocks; ++b) map.push_back((uint32_t)j << 24 | (uint32_t)b);
}

template <class F>
static yy_status group_build(yy_grid *const *grids, int n, yy_precision prec, const double *const *ry,
                             const double *const *rg, double *const *py, double *const *pg, double *const *gy,
                             double *const *gg, TcGroup *G) {
  if (n > 85) return YY_ERR_NOT_SUPPORTED;   // three coefficient jobs a field within the maps' 8 job bits
  std::vector<PackArgs> stj, rho, rs, cf(3 * (size_t)n);
  std::vector<uint32_t> st_m, rho_m, rs_m, cf_m, rr_m, sc_m;
  int st_kmax = 0;
  std::vector<unsigned char> rho_c, rs_c, cf_c(3 * (size_t)n);
  std::vector<PairArgs> an(n), sy(n);
  std::vector<PairMaps> anm(n), sym(n);
  std::vector<ReduceRotateArgs> rr(n);
  std::vector<ScanGroupField> sc(n);
  int bn_max = 16, an_tiles = 0, sy_tiles = 0;
  for (int i = 0; i < n; ++i) {
    yy_grid *g = grids[i];
    yy_tc_tables *t = g->tc[prec];
    if (!t || g->n_patch != 2 || g->lmax > kReduceRotateLmax) return YY_ERR_NOT_SUPPORTED;
    if ((gy == nullptr) != (gg == nullptr)) return YY_ERR_INVALID_ARG;
    PackArgs pr;
    analysis_args<F>(g, t, ry[i], rg[i], pr, an[i]);
    reduce_rotate_args(g, t, rr[i]);
    if (!scan_group_field(g, false, &sc[i])) return YY_ERR_NOT_SUPPORTED;
    PackArgs c3[3];
    coefficient_args(g, t, c3);
    synthesis_args<F>(g, t, py[i], pg[i], gy ? gy[i] : nullptr, gg ? gg[i] : nullptr, sy[i]);
    // the density rows in the form the field's own solve packs them in:
    // short rows a warp each, long ones a 1024-thread block each
    const bool short_rows = pr.K <= 32 * 64;
    const int rc = pack_class(short_rows ? 32 : 1024, pr.k_pad);
    const int cc = pack_class(32, c3[0].k_pad);
    if (rc < 0 || cc < 0) return YY_ERR_NOT_SUPPORTED;
    const bool stream = !short_rows && ((uintptr_t)pr.src0 % 16) == 0 && ((uintptr_t)pr.src1 % 16) == 0 &&
                        (pr.ld % 2) == 0 && (pr.K % 2) == 0 && pr.K <= kStreamMaxK && pr.k_pad <= kStreamMaxK &&
                        (pr.dot_vec == nullptr || (uintptr_t)pr.dot_vec % 8 == 0);
    if (short_rows) {
      map_blocks(rs_m, (int)rs.size(), (pr.rows_pad + 7) / 8);        // eight rows per 256-thread block
      rs.push_back(pr);
      rs_c.push_back((unsigned char)rc);
    } else if (stream) {
      map_blocks(st_m, (int)stj.size(), pr.rows_pad);                 // the rows themselves
      stj.push_back(pr);
      st_kmax = std::max(st_kmax, pr.K);
    } else {
      map_blocks(rho_m, (int)rho.size(), pr.rows_pad);                // one 1024-thread block per row
      rho.push_back(pr);
      rho_c.push_back((unsigned char)rc);
    }
    for (int c = 0; c < 3; ++c) {
      const int k = 3 * i + c;
      cf[k] = c3[c];
      cf_c[k] = (unsigned char)cc;
      map_blocks(cf_m, k, (c3[c].rows_pad + 7) / 8);
    }
    map_blocks(rr_m, i, g->n_r * ((g->n_lm + 255) / 256));
    map_blocks(sc_m, i, scan_group_blocks(sc[i]));
    anm[i] = t->an_maps;
    sym[i] = t->sy_maps;
    bn_max = std::max(bn_max, t->bn);
    an_tiles += an[i].cell_tiles * an[i].row_tiles * an[i].k_splits * an[i].n_jobs;
    sy_tiles += sy[i].cell_tiles * sy[i].row_tiles * sy[i].k_splits * sy[i].n_jobs;
  }
  // one device buffer, each table on a 128-byte boundary (tensor maps want 64)
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 127) / 128 * 128;
    return o;
  };
  const int n_rho = (int)rho.size(), n_rs = (int)rs.size(), n_st = (int)stj.size();
  const size_t o_anm = take(sizeof(PairMaps) * n), o_sym = take(sizeof(PairMaps) * n);
  const size_t o_an = take(sizeof(PairArgs) * n), o_sy = take(sizeof(PairArgs) * n);
  const size_t o_rho = take(sizeof(PackArgs) * n_rho), o_rs = take(sizeof(PackArgs) * n_rs);
  const size_t o_st = take(sizeof(PackArgs) * n_st), o_stm = take(4 * st_m.size());
  const size_t o_cf = take(sizeof(PackArgs) * 3 * n);
  const size_t o_rr = take(sizeof(ReduceRotateArgs) * n), o_sc = take(sizeof(ScanGroupField) * n);
  const size_t o_rhom = take(4 * rho_m.size()), o_rsm = take(4 * rs_m.size()), o_cfm = take(4 * cf_m.size());
  const size_t o_rrm = take(4 * rr_m.size()), o_scm = take(4 * sc_m.size());
  const size_t o_rhoc = take(n_rho), o_rsc = take(n_rs), o_cfc = take(3 * (size_t)n);
  std::vector<unsigned char> host(off, 0);
  auto put = [&](size_t o, const void *src, size_t bytes) {
    if (bytes > 0) memcpy(host.data() + o, src, bytes);
  };
  put(o_anm, anm.data(), sizeof(PairMaps) * n);
  put(o_sym, sym.data(), sizeof(PairMaps) * n);
  put(o_an, an.data(), sizeof(PairArgs) * n);
  put(o_sy, sy.data(), sizeof(PairArgs) * n);
  put(o_rho, rho.data(), sizeof(PackArgs) * n_rho);
  put(o_rs, rs.data(), sizeof(PackArgs) * n_rs);
  put(o_st, stj.data(), sizeof(PackArgs) * n_st);
  put(o_stm, st_m.data(), 4 * st_m.size());
  put(o_cf, cf.data(), sizeof(PackArgs) * 3 * n);
  put(o_rr, rr.data(), sizeof(ReduceRotateArgs) * n);
  put(o_sc, sc.data(), sizeof(ScanGroupField) * n);
  put(o_rhom, rho_m.data(), 4 * rho_m.size());
  put(o_rsm, rs_m.data(), 4 * rs_m.size());
  put(o_cfm, cf_m.data(), 4 * cf_m.size());
  put(o_rrm, rr_m.data(), 4 * rr_m.size());
  put(o_scm, sc_m.data(), 4 * sc_m.size());
  put(o_rhoc, rho_c.data(), n_rho);
  put(o_rsc, rs_c.data(), n_rs);
  put(o_cfc, cf_c.data(), 3 * (size_t)n);
  uint8_t *d = nullptr;
  cudaError_t e = dmalloc((void **)&d, off);
  if (e == cudaSuccess) e = cudaMemcpy(d, host.data(), off, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (d) cudaFree(d);
    return e == cudaErrorMemoryAllocation ? YY_ERR_OOM : YY_ERR_CUDA;
  }
  G->prec = prec;
  G->n = n;
  G->dev = d;
  G->an_maps = (PairMaps *)(d + o_anm);
  G->sy_maps = (PairMaps *)(d + o_sym);
  G->an_args = (PairArgs *)(d + o_an);
  G->sy_args = (PairArgs *)(d + o_sy);
  G->rho_jobs = (PackArgs *)(d + o_rho);
  G->rs_jobs = (PackArgs *)(d + o_rs);
  G->st_jobs = (PackArgs *)(d + o_st);
  G->st_map = (uint32_t *)(d + o_stm);
  G->st_rows = (int)st_m.size();
  G->st_smem = st_kmax * (int)sizeof(double);
  {
    int dev = 0, n_sm = 1;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm < 1) n_sm = 1;
    G->st_grid = std::min(G->st_rows, n_sm);
  }
  if (G->st_rows > 0 && cudaFuncSetAttribute(k_pack_stream_group<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              kStreamMaxK * (int)sizeof(double)) != cudaSuccess)
    return YY_ERR_NOT_SUPPORTED;
  G->cf_jobs = (PackArgs *)(d + o_cf);
  G->rr = (ReduceRotateArgs *)(d + o_rr);
  G->sc = (ScanGroupField *)(d + o_sc);
  G->rho_map = (uint32_t *)(d + o_rhom);
  G->rs_map = (uint32_t *)(d + o_rsm);
  G->cf_map = (uint32_t *)(d + o_cfm);
  G->rr_map = (uint32_t *)(d + o_rrm);
  G->sc_map = (uint32_t *)(d + o_scm);
  G->rho_class = d + o_rhoc;
  G->rs_class = d + o_rsc;
  G->cf_class = d + o_cfc;
  G->rho_nblocks = (int)rho_m.size();
  G->rs_nblocks = (int)rs_m.size();
  G->cf_nblocks = (int)cf_m.size();
  G->rr_nblocks = (int)rr_m.size();
  G->sc_nblocks = (int)sc_m.size();
  // the grouped contractions: shared-memory stages for the largest field's bn
  const int stages = pair_stages<F>(bn_max);
  const int smem = stages * pair_stage_bytes<F>(bn_max) + kSmemFixed;
  for (int m = 0; m < 2; ++m) {
    PairArgs &top = m == 0 ? G->an_top : G->sy_top;
    top = PairArgs{};
    top.stages = stages;
    top.bn = bn_max;
    top.out_mode = m;
    top.err = grids[0]->err;
    top.group = m == 0 ? G->an_args : G->sy_args;
    top.group_maps = m == 0 ? G->an_maps : G->sy_maps;
    top.n_group = n;
  }
  G->an_smem = G->sy_smem = smem;
  int slots = 0;
  {
    if (cudaFuncSetAttribute(k_tc_pair<F, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_tc_pair<F, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit) !=
            cudaSuccess)
      return YY_ERR_NOT_SUPPORTED;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = pair_config(64, smem, 0, attr);
    if (cudaOccupancyMaxActiveClusters(&slots, (void *)k_tc_pair<F, 1, true>, &cfg) != cudaSuccess || slots < 1) {
      cudaGetLastError();
      return YY_ERR_NOT_SUPPORTED;
    }
  }
  G->an_pairs = std::min(an_tiles, slots);
  G->sy_pairs = std::min(sy_tiles, slots);
  return YY_OK;
}

template <class F>
static cudaError_t group_run(const TcGroup *G, cudaStream_t s) {
  const PairMaps none = {};   // the grouped contractions read each field's maps from G
  if (G->st_rows > 0)
    k_pack_stream_group<F><<<G->st_grid, 1024, G->st_smem, s>>>(G->st_jobs, G->st_map, G->st_rows, G->n > 0 ? G->an_top.err : nullptr);
  if (G->rho_nblocks > 0) k_pack_group<F, 1024><<<G->rho_nblocks, 1024, 0, s>>>(G->rho_jobs, G->rho_map, G->rho_class);
  if (G->rs_nblocks > 0) k_pack_group<F, 32><<<G->rs_nblocks, 256, 0, s>>>(G->rs_jobs, G->rs_map, G->rs_class);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = pair_config(G->an_pairs, G->an_smem, s, attr);
  if ((e = cudaLaunchKernelEx(&cfg, k_tc_pair<F, 0, true>, none, G->an_top)) != cudaSuccess) return e;
  k_reduce_rotate_group<<<G->rr_nblocks, 256, 0, s>>>(G->rr, G->rr_map);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = scan_group_launch(G->sc, G->sc_map, G->sc_nblocks, true, s)) != cudaSuccess) return e;
  k_pack_group<F, 32><<<G->cf_nblocks, 256, 0, s>>>(G->cf_jobs, G->cf_map, G->cf_class);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  cfg = pair_config(G->sy_pairs, G->sy_smem, s, attr);
  return cudaLaunchKernelEx(&cfg, k_tc_pair<F, 1, true>, none, G->sy_top);
}

yy_status tc_group_create(yy_grid *const *grids, int n, yy_precision prec, const double *const *ry,
                          const double *const *rg, double *const *py, double *const *pg, double *const *gy,
                          double *const *gg, TcGroup **out) {
  if (!grids || n < 1 || !out) return YY_ERR_INVALID_ARG;
  TcGroup *G = new (std::nothrow) TcGroup();
  if (!G) return YY_ERR_OOM;
  yy_status st;
  switch (prec) {
    case YY_FP16X2: st = group_build<FormFP16x2>(grids, n, prec, ry, rg, py, pg, gy, gg, G); break;
    case YY_BF16X3: st = group_build<FormBF16x3>(grids, n, prec, ry, rg, py, pg, gy, gg, G); break;
    case YY_TF32: st = group_build<FormTF32>(grids, n, prec, ry, rg, py, pg, gy, gg, G); break;
    default: st = YY_ERR_NOT_SUPPORTED;
  }
  if (st != YY_OK) {
    tc_group_destroy(G);
    return st;
  }
  *out = G;
  return YY_OK;
}

cudaError_t tc_group_run(const TcGroup *G, cudaStream_t s) {
  switch (G->prec) {
    case YY_FP16X2: return group_run<FormFP16x2>(G, s);
    case YY_BF16X3: return group_run<FormBF16x3>(G, s);
    case YY_TF32: return group_run<FormTF32>(G, s);
    default: return cudaErrorInvalidValue;
  }
}

int tc_group_launches(const TcGroup *G) { return 5 + (G->st_rows > 0) + (G->rho_nblocks > 0) + (G->rs_nblocks > 0); }

void tc_group_destroy(TcGroup *G) {
  if (!G) return;
  if (G->dev) cudaFree(G->dev);
  delete G;
}

}  // namespace yy
