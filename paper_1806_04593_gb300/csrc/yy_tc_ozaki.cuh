// The Ozaki forms of the pair kernel: float64 results from exact products of
// bf16 digits (output mode 3 of k_tc_pair), and their epilogue.  Included by
// yy_tc_pair.cuh after the PTX wrappers it uses.
#pragma once

namespace yy {

// Float64 results by the Ozaki scheme: each operand row is scaled by a power
// of two to |x| <= 1/2 and written with six balanced base-256 digits,
// x = sum_s a_s 2^(-8 (s + 1)) + r, integers |a_s| <= 128 (exact in bf16),
// |r| <= 2^-49: the digits of round(|x| 2^48), each taken in [-127, 128]
// with a carry into the next.  The products of digit levels L = s + t <= 6
// (26 of the 36) are kept; the dropped ones add up to below 2^-56.  A
// product sum over K <= 64 is at most 64 * 128^2 = 2^20, and a level has at
// most 6 products, so every level accumulates in one TMEM accumulator below
// 2^23: exact in fp32.  The epilogue combines the seven levels in integers
// and rounds once to float64.  The rounding of the digits makes the
// representation error unbiased, so it does not add up along K.
// Products in level order; level L has s = max(0, L - 5) .. min(L, 5).
struct FormOzaki {
  typedef __nv_bfloat16 elem;
  static constexpr int kKind = KIND_BF16, kElem = 2, kPA = 6, kPB = 6, kPairs = 26, kAccs = 7;
  static constexpr int kMaxK = 64;
  __host__ __device__ static constexpr int s_lo(int L) { return L > 5 ? L - 5 : 0; }
  // first product of level L (levels hold 1, 2, 3, 4, 5, 6, 5 products)
  __host__ __device__ static constexpr int start(int L) {
    return L <= 0 ? 0 : L == 1 ? 1 : L == 2 ? 3 : L == 3 ? 6 : L == 4 ? 10 : L == 5 ? 15 : L == 6 ? 21 : 26;
  }
  __host__ __device__ static constexpr int level(int i) {
    return i < 1 ? 0 : i < 3 ? 1 : i < 6 ? 2 : i < 10 ? 3 : i < 15 ? 4 : i < 21 ? 5 : 6;
  }
  __host__ __device__ static constexpr int pa(int i) { return s_lo(level(i)) + i - start(level(i)); }
  __host__ __device__ static constexpr int pb(int i) { return level(i) - pa(i); }
  __host__ __device__ static constexpr int acc(int i) { return level(i); }
  __host__ __device__ static constexpr bool first(int i) { return i == start(level(i)); }
  // accumulators of level L: acc_base(L) .. + n_acc(L) - 1
  __host__ __device__ static constexpr int acc_base(int L) { return L; }
  __host__ __device__ static constexpr int n_acc(int) { return 1; }
};

// The same digits and products for longer K (up to 320): a product's sum is
// at most K 2^14, so an accumulator takes at most 3 products (3 * 341 * 2^14
// < 2^24) and levels 3-6 use two accumulators each: eleven in all.
struct FormOzakiWide : FormOzaki {
  static constexpr int kAccs = 11, kMaxK = 320;
  __host__ __device__ static constexpr int acc_base(int L) { return L <= 3 ? L : 3 + 2 * (L - 3); }
  __host__ __device__ static constexpr int n_acc(int L) { return L <= 2 ? 1 : 2; }
  __host__ __device__ static constexpr int acc(int i) { return acc_base(level(i)) + (pa(i) - s_lo(level(i))) / 3; }
  __host__ __device__ static constexpr bool first(int i) { return (pa(i) - s_lo(level(i))) % 3 == 0; }
};
static_assert(FormOzakiWide::acc(9) == 4 && FormOzakiWide::acc(25) == 10 && FormOzakiWide::acc(21) == 9 &&
                  FormOzakiWide::first(24) && !FormOzakiWide::first(25) && FormOzakiWide::acc(14) == 6,
              "wide Ozaki product table");
static_assert(FormOzaki::start(7) == 26 && FormOzaki::level(25) == 6 && FormOzaki::pa(25) == 5 &&
                  FormOzaki::pb(25) == 1 && FormOzaki::pa(21) == 1 && FormOzaki::first(21) &&
                  FormOzaki::pa(20) == 5 && FormOzaki::pb(20) == 0 && !FormOzaki::first(20),
              "Ozaki product table");

// v 2^e exactly, for |v| < 2^53 and a result in the normal range (built from
// the bits: the top bit's position gives the exponent, the bits below it the
// fraction); anything else takes ldexp.
__device__ __forceinline__ double i64_ldexp(long long v, int e) {
  if (v == 0) return 0.0;
  const unsigned long long sgn = (unsigned long long)v & 0x8000000000000000ull;
  const unsigned long long u = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  const int lz = __clzll((long long)u);
  const int be = 1086 - lz + e;   // (63 - lz) + 1023 + e
  if (lz < 11 || be <= 0 || be >= 2047) return ldexp((double)v, e);
  const unsigned long long frac = ((u << lz) << 1) >> 12;
  return __longlong_as_double((long long)(sgn | ((unsigned long long)be << 52) | frac));
}

// An accumulator value of the Ozaki forms: an integer below 2^24 held in fp32.
__device__ __forceinline__ int oz_int(uint32_t v) { return __float2int_rn(__uint_as_float(v)); }

// Level sum S_L of 8 columns: the level's accumulators (one or two, bn
// columns apart from tcol onwards) added as integers (below 2^25).
template <class F>
__device__ __forceinline__ void oz_level(uint32_t tcol, int bn, int L, int (&S)[8]) {
  uint32_t v[8];
  tmem_ld8_async(tcol + (uint32_t)(F::acc_base(L) * bn), v);
  tmem_wait_ld();
#pragma unroll
  for (int j = 0; j < 8; ++j) S[j] = oz_int(v[j]);
  if (F::n_acc(L) == 2) {
    tmem_ld8_async(tcol + (uint32_t)((F::acc_base(L) + 1) * bn), v);
    tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < 8; ++j) S[j] += oz_int(v[j]);
  }
}

// Level sum S_L of 8 columns as fp32 (exact for one accumulator; the two of
// a FormOzakiWide level added with one rounding).
template <class F>
__device__ __forceinline__ void oz_level_f(uint32_t tcol, int bn, int L, float (&S)[8]) {
  uint32_t v[8];
  tmem_ld8_async(tcol + (uint32_t)(F::acc_base(L) * bn), v);
  tmem_wait_ld();
#pragma unroll
  for (int j = 0; j < 8; ++j) S[j] = __uint_as_float(v[j]);
  if (F::n_acc(L) == 2) {
    tmem_ld8_async(tcol + (uint32_t)((F::acc_base(L) + 1) * bn), v);
    tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < 8; ++j) S[j] += __uint_as_float(v[j]);
  }
}

// exact float64 of an fp32 value times 2^e (a normal result; zero stays zero)
__device__ __forceinline__ double f32_ldexp(float f, int e) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t ex = (u >> 23) & 0xFFu;
  if (ex == 0u) return 0.0;   // the values here are integer combinations: zero or at least 1
  const int be = (int)ex + 896 + e;
  if (ex == 255u || be <= 0 || be >= 2047) return ldexp((double)f, e);
  const unsigned long long bits = ((unsigned long long)(u & 0x80000000u) << 32) | ((unsigned long long)be << 52) |
                                  ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}

// The 8 float64 values of one epilogue chunk (TMEM column tcol) from the
// level sums S_0 .. S_6:
//   value = 2^ce (hi 2^24 + lo),  hi = S_0 2^24 + S_1 2^16 + S_2 2^8 + S_3  (int64, below 2^49),
//                                  lo = S_4 2^16 + S_5 2^8 + S_6          (fp32).
// hi is exact in int64 and in float64.  lo is formed in fp32 from the
// accumulator values (a unit is 2^-64 of the two rows' scales): |lo| is
// below 2^39 units for FormOzaki and 2^41 for FormOzakiWide, so its rounding
// is at most 2^15 or 2^17 units, under the digits' own error, which is up to
// 2^15 units per product term (2^-49 of the scales) and adds up over the K
// (<= 64 or <= 320) terms.  One more rounding, in the final addition.
template <class F>
__device__ __forceinline__ void ozaki_chunk(uint32_t tcol, int bn, int ce, double *dst) {
  int S[8];
  long long hi[8];
  oz_level<F>(tcol, bn, 0, S);
#pragma unroll
  for (int j = 0; j < 8; ++j) hi[j] = (long long)S[j] << 24;
  oz_level<F>(tcol, bn, 1, S);
#pragma unroll
  for (int j = 0; j < 8; ++j) hi[j] += (long long)S[j] << 16;
  oz_level<F>(tcol, bn, 2, S);
#pragma unroll
  for (int j = 0; j < 8; ++j) hi[j] += (long long)S[j] << 8;
  oz_level<F>(tcol, bn, 3, S);
#pragma unroll
  for (int j = 0; j < 8; ++j) hi[j] += (long long)S[j];
  float lo[8];
  oz_level_f<F>(tcol, bn, 4, lo);
#pragma unroll
  for (int j = 0; j < 8; ++j) lo[j] *= 65536.0f;
  float t[8];
  oz_level_f<F>(tcol, bn, 5, t);
#pragma unroll
  for (int j = 0; j < 8; ++j) lo[j] = fmaf(t[j], 256.0f, lo[j]);
  oz_level_f<F>(tcol, bn, 6, t);
#pragma unroll
  for (int j = 0; j < 8; ++j) dst[j] = i64_ldexp(hi[j], ce + 24) + f32_ldexp(lo[j] + t[j], ce);
}

}  // namespace yy
