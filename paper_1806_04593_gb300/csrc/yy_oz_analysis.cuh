// k_oz_analysis: the azimuthal stage of the float64 analysis by the Ozaki
// scheme.
//
//   F[row][t] = sum_k (rho w)[row][k] az[k][t]     rows (shell, theta row), t = 0 .. 2 l_max
//
// with the weighted densities (rho w) and the azimuthal table az written as
// FormOzaki's six bf16 digit slices (k_rhow_ozaki, ozaki_prepare_analysis).
// K = n_phi is long (up to 640), so it runs in fills of kFillK = 160 whose
// level sums stay exact in fp32 (below 2^24), and the epilogue adds the fills
// in integers (ozaki_accumulate) before the one rounding to float64.
//
// Schedule: each stage of a three-stage ring holds one 32-wide K block of
// both operands: the six digit slices of 128 density rows (48 KiB) and three
// slices of the table, all 64 slot rows (12 KiB) -- the even slices in the
// even CTA, the odd ones in the odd CTA, at the same offsets.  (Keeping the
// table resident, 120 KiB at K = 320, left room for two density stages
// only, and the loads of one stage did not hide behind the MMAs of the
// other.)  The table is re-read from L2 for every row tile.
//
// Two digit products per MMA: an MMA of N = 128 takes its B columns 0-63
// from the even CTA and 64-127 from the odd one, so with A = density slice s
// and the table slot holding slices u (even CTA) and u + 1 (odd CTA) it adds
// the products (s, u) and (s, u + 1) into the accumulators of levels s + u
// and s + u + 1, which lie side by side (level L at TMEM columns 64 L).  The
// 26 products of levels <= 6 take 14 MMAs per 16-wide K step instead of 26
// (two of them also add a level-7 product into a spare accumulator that is
// never read), and an MMA's fixed cost -- reading its 4 KiB A tile from
// shared memory -- buys four times the work of the 32-column tiles of the
// pair kernel.  Since one MMA starts two accumulators that other MMAs
// continue, the MMAs always accumulate and the epilogue clears the
// accumulators (TMEM stores of zeros) after reading each fill, and once
// before the first.  The eight level accumulators of 64 columns (all 512
// TMEM columns) have one buffer: each fill's MMAs wait until the epilogue
// has read and cleared the previous fill, a small part of a fill's MMA time.
//   warp 0  lane 0: TMA producer
//   warp 1  TMEM allocation; in the even CTA lane 0 issues MMAs and commits
//   warps 2-17: epilogue, 16 slots x 32 rows each, results stored straight
//               from registers (128 contiguous bytes per row)
// Every wait is bounded (~2 s): on expiry the device error word gets
// YY_DEVERR_TIMEOUT and the CTA winds down, releasing TMEM.
#pragma once

namespace yy {

constexpr int kOzAnBN = 64;                   // slots of a row tile
constexpr int kOzAnStages = 3;
constexpr int kOzAnSlotA = kPairRows * kRowBytes;                    // 8 KiB
constexpr int kOzAnSlotB = kOzAnBN * kRowBytes;                      // 4 KiB: one table slice, all slots
constexpr int kOzAnStageA = FormOzaki::kPA * kOzAnSlotA;             // 48 KiB
constexpr int kOzAnKBlockB = (FormOzaki::kPB / 2) * kOzAnSlotB;      // 12 KiB per K block (three slices)
constexpr int kOzAnLevels = FormOzaki::kAccs + 1;                    // levels 0..6 and the spare level 7
static_assert(kOzAnLevels * kOzAnBN <= kPairTmemCols, "k_oz_analysis accumulators");
static_assert(FormOzaki::kPA == 6 && FormOzaki::kPB == 6, "k_oz_analysis pairs slices u, u + 1 of six");

// The paired products of one K step: density slice s with table slices
// u, u + 1 (u = 0, 2, 4), for s + u <= 6; 14 pairs cover the 26 products of
// levels <= 6 (and (2, 5), (4, 3) of level 7).
__host__ __device__ constexpr int oz_an_pairs() { return 14; }
__host__ __device__ constexpr int oz_an_s(int i) { return i < 6 ? i : (i < 11 ? i - 6 : i - 11); }
__host__ __device__ constexpr int oz_an_u(int i) { return i < 6 ? 0 : (i < 11 ? 2 : 4); }

constexpr int kOzAnStage = kOzAnStageA + kOzAnKBlockB;               // 60 KiB
constexpr int kOzAnSmem = 1024 + kOzAnStages * kOzAnStage + 512;
static_assert(kOzAnSmem <= kSmemLimit, "k_oz_analysis shared memory");

struct OzAnalysisArgs {
  int cells, cell_tiles;        // valid density rows; tiles of 256 rows (pairs of 128)
  int cols;                     // valid slots (2 l_max + 1)
  int kb_total, kb_fill;        // K blocks; K blocks per accumulator fill
  int a_rows, b_rows;           // rows of one slice in the stacked operands
  long long ldo;                // output row stride (doubles)
  double *out;                  // [cells][ldo]
  const int *cell_exp;          // per row: power of two of a unit level-6 sum
  int *err;
};

struct OzAnalysisMaps {
  CUtensorMap a, b;             // density digits (box 32 x 128), table digits (box 32 x 64)
};

__global__ void __launch_bounds__(kThreads, 1)
k_oz_analysis(const __grid_constant__ OzAnalysisMaps maps, const __grid_constant__ OzAnalysisArgs a) {
  typedef FormOzaki F;
  constexpr int KSTEPS = kRowBytes / 32;
  constexpr int S = kOzAnStages;

  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *ring = smem;                                      // [stage]{[slice][128 rows][64 B], [slice][32 rows][64 B]}
  uint64_t *bars = (uint64_t *)(ring + S * kOzAnStage);
  uint64_t *full = bars, *empty = full + S;
  uint64_t *tfull = empty + S, *tempty = tfull + 1;          // one accumulator set; tempty counted in the even CTA
  uint32_t *tmem_slot = (uint32_t *)(tempty + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rank = (int)cluster_rank();
  const int pair = (int)blockIdx.x >> 1, n_pairs = (int)gridDim.x >> 1;
  const int total = a.cell_tiles;
  const int fills = (a.kb_total + a.kb_fill - 1) / a.kb_fill;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, 2 * kEpiWarps);
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc_pair(tmem_slot, kPairTmemCols);
    tc_fence_before();
  }
  __syncthreads();
  cluster_sync();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      const uint32_t tx = 2u * (uint32_t)kOzAnStage;
      int gk = 0, s = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int t = pair; t < total && ok; t += n_pairs) {
        const int arow = (2 * t + rank) * kPairRows;
        for (int kb = 0; kb < a.kb_total; ++kb, ++gk) {
          if (gk >= S && !mbar_wait(&empty[s], ph ^ 1, a.err)) {
            ok = false;
            break;
          }
          if (rank == 0) mbar_expect_tx(&full[s], tx);
          const uint32_t fbar = mapa_rank(smem_u32(&full[s]), 0);
          uint8_t *st = ring + s * kOzAnStage;
#pragma unroll
          for (int p = 0; p < F::kPA; ++p)
            tma_load_2d_pair(&maps.a, smem_u32(st + p * kOzAnSlotA), fbar, kb * 32, p * a.a_rows + arow);
          // this CTA's three table slices (rank, rank + 2, rank + 4), all slots
#pragma unroll
          for (int p = 0; p < F::kPB / 2; ++p)
            tma_load_2d_pair(&maps.b, smem_u32(st + kOzAnStageA + p * kOzAnSlotB), fbar, kb * 32,
                             (2 * p + rank) * a.b_rows);
          if (++s == S) {
            s = 0;
            ph ^= 1;
          }
        }
      }
      if (ok)
        for (int i = max(0, gk - S); i < gk; ++i)
          if (!mbar_wait(&empty[i % S], (i / S) & 1, a.err)) break;
    }
  } else if (warp == 1) {
    if (rank == 0 && lane == 0) {
      const uint32_t idesc = instr_desc_pair<F>(2 * kOzAnBN);
      int gk = 0, it = 0, s = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int t = pair; t < total && ok; t += n_pairs) {
        for (int c0 = 0; c0 < a.kb_total && ok; c0 += a.kb_fill, ++it) {
          // the epilogue has read the previous fill out of the accumulators
          // and cleared them (or cleared them before the first)
          if (!mbar_wait_cluster(tempty, it & 1, a.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const int c1 = min(a.kb_total, c0 + a.kb_fill);
          for (int kb = c0; kb < c1; ++kb, ++gk) {
            if (!mbar_wait_cluster(&full[s], ph, a.err)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(ring + s * kOzAnStage);
            const uint32_t sb = sa + kOzAnStageA;
#pragma unroll
            for (int q = 0; q < oz_an_pairs(); ++q) {
              const int s_a = oz_an_s(q), u = oz_an_u(q);
              const uint32_t dq = tmem_base + (uint32_t)((s_a + u) * kOzAnBN);
#pragma unroll
              for (int kk = 0; kk < KSTEPS; ++kk) {
                const uint64_t da = smem_desc(sa + s_a * kOzAnSlotA + kk * 32);
                const uint64_t db = smem_desc(sb + (u / 2) * kOzAnSlotB + kk * 32);
                mma_pair<F>(dq, da, db, idesc, 1u);
              }
            }
            mma_commit_pair(&empty[s]);
            if (++s == S) {
              s = 0;
              ph ^= 1;
            }
          }
          if (ok) mma_commit_pair(tfull);
        }
      }
    }
  } else {
    // epilogue: lane quarter `quarter` (32 rows), slots 16 sub .. 16 sub + 15
    const int quarter = warp & 3;
    const int sub = (warp - 2) >> 2;
    const uint32_t tempty_even = mapa_rank(smem_u32(tempty), 0);
    const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(sub * 16);
    // clear this warp's columns of every level accumulator, then release them
    auto clear_levels = [&]() {
#pragma unroll
      for (int L = 0; L < kOzAnLevels; ++L) tmem_zero16(tbase + (uint32_t)(L * kOzAnBN));
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster_relaxed(tempty_even);
    };
    clear_levels();
    int it = 0;
    bool ok = true;
    for (int t = pair; t < total && ok; t += n_pairs) {
      const int cell = (2 * t + rank) * kPairRows + quarter * 32 + lane;
      const bool cell_ok = cell < a.cells;
      const int ce = cell_ok ? a.cell_exp[cell] : 0;
      long long hi[2][8];
      float lo[2][8];
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          hi[h][j] = 0;
          lo[h][j] = 0.0f;
        }
      for (int f = 0; f < fills; ++f, ++it) {
        if (!mbar_wait_cluster(tfull, it & 1, a.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        ozaki_accumulate(tbase, kOzAnBN, hi[0], lo[0]);
        ozaki_accumulate(tbase + 8u, kOzAnBN, hi[1], lo[1]);
        clear_levels();
      }
      if (!ok) break;
      if (cell_ok) {
        double v[16];
        ozaki_finish(hi[0], lo[0], ce, v);
        ozaki_finish(hi[1], lo[1], ce, v + 8);
        double *orow = a.out + (size_t)cell * a.ldo;
        const int c0 = sub * 16;
        if ((a.ldo & 1) == 0 && c0 + 16 <= a.cols) {
#pragma unroll
          for (int j = 0; j < 16; j += 2) *reinterpret_cast<double2 *>(orow + c0 + j) = make_double2(v[j], v[j + 1]);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (c0 + j < a.cols) orow[c0 + j] = v[j];
        }
      }
    }
  }
  __syncthreads();
  cluster_sync();   // no CTA leaves while its peer may still reach its barriers or TMEM
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc_pair(tmem_base, kPairTmemCols);
  }
}

}  // namespace yy
