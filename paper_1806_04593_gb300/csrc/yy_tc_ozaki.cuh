// The Ozaki forms of the pair kernel: float64 results from exact products of
// bf16 digits (output modes 3 and 4 of k_tc_pair), and their epilogues.  Included by
// yy_tc_pair.cuh after the PTX wrappers it uses.
#pragma once

namespace yy {

// Float64 results by the Ozaki scheme: each operand row is scaled by a power
// of two to |x| <= 1/2 and written with six balanced base-256 digits,
// x = sum_s a_s 2^(-8 (s + 1)) + r, integers |a_s| <= 128 (exact in bf16),
// |r| <= 2^-49: the digits of round(|x| 2^48), each taken in [-127, 128]
// with a carry into the next.  The products of digit levels L = s + t <= 6
// (26 of the 36) are kept; the dropped ones add up to below 2^-56.  A
// product sum over K <= 160 is at most 160 * 128^2 < 2^21.4, and a level has
// at most 6 products, so every level accumulates in one TMEM accumulator
// below 2^24 over a fill of up to 160: exact in fp32.  Longer K runs in
// several fills, which the epilogue adds.  The epilogue combines levels 0-3
// in int64 and the three lowest in fp32, and rounds once to float64.  The
// digits are rounded to nearest, so their representation errors take either
// sign and grow like sqrt(K) along K rather than like K.
// Products in level order; level L has s = max(0, L - 5) .. min(L, 5).
struct FormOzaki {
  typedef __nv_bfloat16 elem;
  static constexpr int kKind = KIND_BF16, kElem = 2, kPA = 6, kPB = 6, kPairs = 26, kAccs = 7;
  // K per accumulator fill (a level sum stays below 6 * 160 * 2^14 < 2^24), and
  // the longest K taken: the epilogue adds up to four fills in int64 / fp32
  static constexpr int kFillK = 160, kMaxFills = 4;
  static constexpr int kMaxK = 64;   // K of the synthesis (2 l_max + 1, one fill)
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
};

static_assert(FormOzaki::start(7) == 26 && FormOzaki::level(25) == 6 && FormOzaki::pa(25) == 5 &&
                  FormOzaki::pb(25) == 1 && FormOzaki::pa(21) == 1 && FormOzaki::first(21) &&
                  FormOzaki::pa(20) == 5 && FormOzaki::pb(20) == 0 && !FormOzaki::first(20),
              "Ozaki product table");

// v 2^e exactly, for |v| < 2^53 and a result in the normal range, built
// from the bits: |v| shifted so that its top bit lands on bit 52 (the
// implicit one), then the biased exponent less one added above it (the
// implicit one carries it up by one) and the sign bit set; anything else
// takes ldexp.
__device__ __forceinline__ double i64_ldexp(long long v, int e) {
  const unsigned long long s = (unsigned long long)(v >> 63);          // 0 or all ones
  const unsigned long long u = ((unsigned long long)v ^ s) - s;        // |v|
  const int lz = __clzll((long long)u);                                // 64 for v = 0
  const int be = 1086 - lz + e;                                        // (63 - lz) + 1023 + e
  if (lz < 11 || lz == 64 || be <= 0 || be >= 2047) return lz == 64 ? 0.0 : ldexp((double)v, e);
  const unsigned long long m = u << (lz - 11);
  return __longlong_as_double((long long)((m + ((unsigned long long)(be - 1) << 52)) | (s << 63)));
}

// i64_ldexp for callers that checked e once per row: |v| < 2^53 and
// e in [-1022, 971] keep every nonzero result normal, so the range checks go.
__device__ __forceinline__ bool i64_ldexp_row_ok(int e) { return e >= -1022 && e <= 971; }
__device__ __forceinline__ double i64_ldexp_row(long long v, int e) {
  const unsigned long long s = (unsigned long long)(v >> 63);
  const unsigned long long u = ((unsigned long long)v ^ s) - s;
  const int lz = __clzll((long long)u);
  const unsigned long long m = u << ((lz - 11) & 63);
  const unsigned long long b = (m + ((unsigned long long)(1085 - lz + e) << 52)) | (s << 63);
  return __longlong_as_double((long long)(u == 0ull ? 0ull : b));
}

// The same through the float64 pipe's conversion (exact: |v| < 2^53) and an
// exponent add: a few issue slots instead of the integer formatting, for
// callers that spread their values over both pipes.
__device__ __forceinline__ double i64_ldexp_row_cvt(long long v, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(__ll2double_rn(v));
  return __longlong_as_double((long long)(v == 0 ? 0ull : b + ((unsigned long long)(long long)e << 52)));
}

// An accumulator value of the Ozaki forms: an integer below 2^24 held in fp32.
__device__ __forceinline__ int oz_int(uint32_t v) { return __float2int_rn(__uint_as_float(v)); }

// Level sum S_L of 8 columns (accumulator L, bn columns apart from tcol
// onwards), as an integer and as the fp32 value itself.
__device__ __forceinline__ void oz_level(uint32_t tcol, int bn, int L, int (&S)[8]) {
  uint32_t v[8];
  tmem_ld8_async(tcol + (uint32_t)(L * bn), v);
  tmem_wait_ld();
#pragma unroll
  for (int j = 0; j < 8; ++j) S[j] = oz_int(v[j]);
}

__device__ __forceinline__ void oz_level_f(uint32_t tcol, int bn, int L, float (&S)[8]) {
  uint32_t v[8];
  tmem_ld8_async(tcol + (uint32_t)(L * bn), v);
  tmem_wait_ld();
#pragma unroll
  for (int j = 0; j < 8; ++j) S[j] = __uint_as_float(v[j]);
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

// One fill's level sums S_0 .. S_6 of 8 columns (TMEM column tcol) added to
// the chunk's running value 2^ce (hi 2^24 + lo):
//   hi += S_0 2^24 + S_1 2^16 + S_2 2^8 + S_3   (int64: below 2^48 per fill)
//   lo += S_4 2^16 + S_5 2^8 + S_6             (fp32)
// hi stays exact (below 2^50 over four fills, exact in float64 too).  lo is
// formed in fp32 from the accumulator values (a unit is 2^-64 of the two
// rows' scales): below 2^40 units per fill, so its rounding stays under 2^18
// units over four fills, below the digits' own error, which is up to 2^15
// units per product term (2^-49 of the scales) and adds up over the K terms.
__device__ __forceinline__ void ozaki_accumulate(uint32_t tcol, int bn, long long (&hi)[8], float (&lo)[8]) {
  int S[8];
  oz_level(tcol, bn, 0, S);
#pragma unroll
  for (int j = 0; j < 8; ++j) hi[j] += (long long)S[j] << 24;
  oz_level(tcol, bn, 1, S);
#pragma unroll
  for (int j = 0; j < 8; ++j) hi[j] += (long long)S[j] << 16;
  oz_level(tcol, bn, 2, S);
#pragma unroll
  for (int j = 0; j < 8; ++j) hi[j] += (long long)S[j] << 8;
  oz_level(tcol, bn, 3, S);
#pragma unroll
  for (int j = 0; j < 8; ++j) hi[j] += (long long)S[j];
  float u[8], w[8];
  oz_level_f(tcol, bn, 4, u);
  oz_level_f(tcol, bn, 5, w);
#pragma unroll
  for (int j = 0; j < 8; ++j) u[j] = fmaf(w[j], 256.0f, u[j] * 65536.0f);
  oz_level_f(tcol, bn, 6, w);
#pragma unroll
  for (int j = 0; j < 8; ++j) lo[j] += u[j] + w[j];
}

// ---- the biased single-fill epilogue (output mode 4) ----------------------
//
// Two spare columns of the K padding carry a constant product into every
// level accumulator: column nt holds the digit 6144 = 3 2^11 in slice 0 of
// each G row and 2048 = 2^11 in all six slices of the trig table, column
// nt + 1 holds 6144 in slice 1 of each G row and 2048 in slice 5 of the trig
// table.  Of the kept products (s, t) exactly one per level meets a non-zero
// pair there -- (0, L) for L <= 5 in column nt, (1, 5) for L = 6 in column
// nt + 1 -- so every level sum becomes 3 2^22 + S_L.  The host checks, from
// the trig digits and |G digit| <= 128, that |S_L| < 2^22 for every column;
// the accumulator then lies in [2^23, 2^24), where fp32 steps by exactly 1,
// and its bit pattern minus that of 3 2^22 is S_L as an integer: no float to
// integer conversions.
constexpr uint32_t kOzBiasBits = 0x4B400000u;        // fp32 bits of 3 2^22
constexpr float kOzBiasG = 6144.0f, kOzBiasT = 2048.0f;
// a 2^8 + b of two biased levels minus the biases' share (mod 2^32)
constexpr uint32_t kOzBias2 = (kOzBiasBits << 8) + kOzBiasBits;

// Float64 values of 8 columns (TMEM column tcol, accumulator L at + L bn) of
// a single fill, rows scaled by 2^ce per unit level-6 sum.  In units of a
// level-4 sum, V = S_0 2^32 + S_1 2^24 + S_2 2^16 + S_3 2^8 + S_4 +
// round((S_5 2^8 + S_6) / 2^16): an integer below 2^53 in magnitude (|S_0| <=
// 2^14 K with K <= 64), so its conversion is exact and the only rounding is
// that of the two lowest levels, at most half a level-4 unit (2^-49 of the
// rows' scales, below the digits' own representation error).
__device__ __forceinline__ void ozaki_biased8(uint32_t tcol, int bn, int ce, double *dst) {
  uint32_t u[7][8];
#pragma unroll
  for (int L = 0; L < 7; ++L) tmem_ld8_async(tcol + (uint32_t)(L * bn), u[L]);
  tmem_wait_ld();
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int t56 = (int)((u[5][j] << 8) + u[6][j] - kOzBias2);          // S_5 2^8 + S_6
    const int lo = (int)((u[3][j] << 8) + u[4][j] - kOzBias2) + ((t56 + 32768) >> 16);
    const int mid = (int)((u[1][j] << 8) + u[2][j] - kOzBias2);          // S_1 2^8 + S_2
    const int hi = (int)(u[0][j] - kOzBiasBits);                          // S_0
    const long long V = ((long long)hi << 32) + ((long long)mid << 16) + (long long)lo;
    dst[j] = i64_ldexp(V, ce + 16);
  }
}

// The chunk's float64 values: one rounding, in the final addition.
__device__ __forceinline__ void ozaki_finish(const long long (&hi)[8], const float (&lo)[8], int ce, double *dst) {
#pragma unroll
  for (int j = 0; j < 8; ++j) dst[j] = i64_ldexp(hi[j], ce + 24) + f32_ldexp(lo[j], ce);
}

}  // namespace yy
