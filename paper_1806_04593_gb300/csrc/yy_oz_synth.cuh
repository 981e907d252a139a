// k_oz_synth: the azimuthal stage of the float64 synthesis by the Ozaki
// scheme, digit levels in pairs.
//
//   out[row][k] = sum_t G[row][t] trig[t][k]     rows (shell, theta row), k = phi_k
//
// for up to four fields (Phi, g_r, g_theta, g_phi), K = 2 l_max + 1 <= 62 in
// one accumulator fill (two 32-wide K blocks).  The operands are FormOzaki's
// six bf16 digit slices; the level sums carry the bias of ozaki_biased8 (two
// spare K columns add 3 2^22 to every level sum), so each level sum S_L is
// the accumulator's bit pattern minus that of 3 2^22.
//
// Levels in pairs, lowest first: the 26 digit products of a tile are issued
// as four passes -- levels (6, 5), (4, 3), (2, 1) and 0 -- each level into
// its own accumulator of N = 96 columns, the two accumulators of a pass side
// by side, two passes in TMEM at a time.  Holding all seven levels of a tile
// at once would limit N to 32 columns (7 x 32, double-buffered, in 512 TMEM
// columns), and an MMA re-reads its 4 KiB A tile from shared memory whatever
// its N, so N = 32 spends most of the tensor core's time on that read.  The
// epilogue keeps two 32-bit integers per output across the passes -- from
// the low end, lo = S_3 2^8 + S_4 + round((S_5 2^8 + S_6) / 2^16), then
// mid = S_1 2^8 + S_2 -- and with S_0 forms the exact integer
// V = S_0 2^32 + mid 2^16 + lo (|V| < 2^53, a level-4 unit) and its float64.
//
// Schedule: a CTA pair (cluster of two, cta_group::2, M = 256 rows) takes a
// cell tile of 256 rows of one field, loads its G digits once (both K blocks,
// all six slices: 96 KiB per CTA) and then runs every longitude tile of
// N = 96 columns against it; the trig digits of each longitude tile (36 KiB
// per CTA) come through a two-stage ring.  While a cell tile runs, the
// producer asks L2 for the next one's G digits.
//   warp 0  lane 0: TMA producer (G tile, then the trig ring)
//   warp 1  TMEM allocation; in the even CTA lane 0 issues MMAs and commits
//   warps 2-17: epilogue, 24 columns x 32 rows each (lane quarter, column
//               group), values staged in shared memory 8 columns at a time so
//               that each store instruction writes 64-byte row runs
// Every wait is bounded (~2 s): on expiry the device error word gets
// YY_DEVERR_TIMEOUT and the CTA winds down, releasing TMEM.
#pragma once

namespace yy {

constexpr int kOzSynthKB = 2;                 // K blocks of 32 digits (K <= 64)
constexpr int kOzSynthBN = 96;                // longitude columns per tile (N of the MMA)
constexpr int kOzSynthNBuf = 2;               // passes in TMEM at a time (256 columns apart, a level at + 0 / + 128)
constexpr int kOzSynthPasses = 4;             // level pairs (6, 5), (4, 3), (2, 1), (0)
constexpr int kOzSynthStages = 2;             // trig ring stages (one longitude tile each)
constexpr int kOzSynthCols = kOzSynthBN / kEpiPerQuarter;           // 24 columns per epilogue warp
constexpr int kOzSlotA = kPairRows * kRowBytes;                      // one slice, one K block: 8 KiB
constexpr int kOzSlotB = (kOzSynthBN / 2) * kRowBytes;               // 3 KiB
constexpr int kOzTileA = kOzSynthKB * FormOzaki::kPA * kOzSlotA;     // 96 KiB
constexpr int kOzStageB = kOzSynthKB * FormOzaki::kPB * kOzSlotB;    // 36 KiB
constexpr int kOzEpiPad = 8 + 2;                                     // staged row: 8 values + 2 pad
constexpr int kOzEpiWarpBytes = 32 * kOzEpiPad * 8 + 32 * 8;         // values + row pointers
constexpr int kOzSynthSmem =
    1024 + kOzTileA + kOzSynthStages * kOzStageB + kEpiWarps * kOzEpiWarpBytes + 512;
static_assert(kOzSynthSmem <= kSmemLimit, "k_oz_synth shared memory");
static_assert(kOzSynthCols % 8 == 0, "epilogue columns in groups of 8");


struct OzSynthJob {
  double *out0, *out1;          // rows r < out_split -> out0 + r ldo, else out1 + (r - out_split) ldo
  const int *cell_exp;          // per row: power of two of a unit level-6 sum
};

struct OzSynthArgs {
  int cells, cell_tiles;        // valid G rows; tiles of 256 rows (pairs of 128)
  int cols, col_tiles;          // valid output columns (n_phi); tiles of kOzSynthBN
  int a_rows, b_rows;           // rows of one slice in the stacked G / trig operands
  int out_split;
  long long ldo;
  int n_jobs;
  int prefetch;                 // ask L2 for the next cell tile's G digits
  OzSynthJob job[4];
  int *err;
};

struct OzSynthMaps {
  CUtensorMap a[4], b;          // G digits per field (box 32 x 128), trig digits (box 32 x 48)
};

__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap *map, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"((uint64_t)map), "r"(x),
               "r"(y)
               : "memory");
}

__global__ void __launch_bounds__(kThreads, 1)
k_oz_synth(const __grid_constant__ OzSynthMaps maps, const __grid_constant__ OzSynthArgs a) {
  typedef FormOzaki F;
  constexpr int KSTEPS = kRowBytes / 32;        // MMAs of K = 16 per K block
  constexpr int BH = kOzSynthBN / 2;            // trig rows per CTA and tile
  constexpr int S = kOzSynthStages;
  constexpr int NB = kOzSynthNBuf;
  constexpr int NC = kOzSynthCols;

  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *tileA = smem;                                     // [kb][slice][128 rows][64 B]
  uint8_t *ringB = smem + kOzTileA;                          // [stage][kb][slice][48 rows][64 B]
  uint8_t *epi = ringB + S * kOzStageB;                      // epilogue staging
  uint64_t *bars = (uint64_t *)(epi + kEpiWarps * kOzEpiWarpBytes);
  uint64_t *a_full = bars, *a_empty = bars + 1;
  uint64_t *b_full = bars + 2, *b_empty = b_full + S;
  uint64_t *tfull = b_empty + S, *tempty = tfull + NB;       // [NB] each, tempty counted in the even CTA
  uint32_t *tmem_slot = (uint32_t *)(tempty + NB);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rank = (int)cluster_rank();
  const int pair = (int)blockIdx.x >> 1, n_pairs = (int)gridDim.x >> 1;
  const int total = a.cell_tiles * a.n_jobs;     // job-major cell tiles

  if (threadIdx.x == 0) {
    mbar_init(a_full, 1);
    mbar_init(a_empty, 1);
    for (int s = 0; s < S; ++s) {
      mbar_init(&b_full[s], 1);
      mbar_init(&b_empty[s], 1);
    }
    for (int b = 0; b < NB; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 2 * kEpiWarps);
    }
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
      const uint32_t a_tx = 2u * (uint32_t)kOzTileA;
      const uint32_t b_tx = 2u * (uint32_t)kOzStageB;
      const uint32_t a_bar = mapa_rank(smem_u32(a_full), 0);
      int gs = 0, s = 0, n_tiles = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int t = pair; t < total && ok; t += n_pairs, ++n_tiles) {
        const int jb = t / a.cell_tiles, ct = t % a.cell_tiles;
        const int arow = (2 * ct + rank) * kPairRows;
        const CUtensorMap *tmA = &maps.a[jb];
        // the previous cell tile's MMAs have all completed before its G tile is replaced
        if (n_tiles > 0 && !mbar_wait(a_empty, (n_tiles - 1) & 1, a.err)) {
          ok = false;
          break;
        }
        if (rank == 0) mbar_expect_tx(a_full, a_tx);
#pragma unroll
        for (int kb = 0; kb < kOzSynthKB; ++kb)
#pragma unroll
          for (int p = 0; p < F::kPA; ++p)
            tma_load_2d_pair(tmA, smem_u32(tileA + (kb * F::kPA + p) * kOzSlotA), a_bar, kb * 32,
                             p * a.a_rows + arow);
        if (a.prefetch && t + n_pairs < total) {
          const int tn = t + n_pairs;
          const CUtensorMap *tmN = &maps.a[tn / a.cell_tiles];
          const int nrow = (2 * (tn % a.cell_tiles) + rank) * kPairRows;
#pragma unroll
          for (int kb = 0; kb < kOzSynthKB; ++kb)
#pragma unroll
            for (int p = 0; p < F::kPA; ++p) tma_prefetch_2d(tmN, kb * 32, p * a.a_rows + nrow);
        }
        for (int ctile = 0; ctile < a.col_tiles; ++ctile, ++gs) {
          if (gs >= S && !mbar_wait(&b_empty[s], ph ^ 1, a.err)) {
            ok = false;
            break;
          }
          if (rank == 0) mbar_expect_tx(&b_full[s], b_tx);
          const uint32_t fbar = mapa_rank(smem_u32(&b_full[s]), 0);
          const uint32_t base = smem_u32(ringB + s * kOzStageB);
          const int brow = ctile * kOzSynthBN + rank * BH;
#pragma unroll
          for (int kb = 0; kb < kOzSynthKB; ++kb)
#pragma unroll
            for (int p = 0; p < F::kPB; ++p)
              tma_load_2d_pair(&maps.b, base + (kb * F::kPB + p) * kOzSlotB, fbar, kb * 32, p * a.b_rows + brow);
          if (++s == S) {
            s = 0;
            ph ^= 1;
          }
        }
      }
      // every load has been consumed before this CTA leaves: the last
      // stages of the ring and the last G tile
      if (ok) {
        for (int i = max(0, gs - S); i < gs; ++i)
          if (!mbar_wait(&b_empty[i % S], (i / S) & 1, a.err)) break;
        if (n_tiles > 0) mbar_wait(a_empty, (n_tiles - 1) & 1, a.err);
      }
    }
  } else if (warp == 1) {
    if (rank == 0 && lane == 0) {
      const uint32_t idesc = instr_desc_pair<F>(kOzSynthBN);
      int gs = 0, it = 0, s = 0, n_tiles = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int t = pair; t < total && ok; t += n_pairs, ++n_tiles) {
        if (!mbar_wait_cluster(a_full, n_tiles & 1, a.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        for (int ctile = 0; ctile < a.col_tiles && ok; ++ctile, ++gs) {
          if (!mbar_wait_cluster(&b_full[s], ph, a.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sb = smem_u32(ringB + s * kOzStageB);
          // the passes of this tile: levels (6, 5), (4, 3), (2, 1), 0, each
          // pass into the next accumulator pair of the rotation
#pragma unroll 1
          for (int pass = 0; pass < kOzSynthPasses; ++pass, ++it) {
            const int b = it % NB;
            if (it >= NB) {
              if (!mbar_wait_cluster(&tempty[b], ((it / NB) & 1) ^ 1, a.err)) {
                ok = false;
                break;
              }
              tc_fence_after();
            }
            const int Lhi = 6 - 2 * pass;                  // 6, 4, 2, 0; its partner Lhi - 1 (none for 0)
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
              const int L = Lhi - h;
              if (L < 0) break;
              const uint32_t dacc = tmem_base + (uint32_t)(b * 256 + h * 128);
              const int s0 = F::s_lo(L), s1 = L < 5 ? L : 5;
              for (int sa = s0; sa <= s1; ++sa) {
#pragma unroll
                for (int kb = 0; kb < kOzSynthKB; ++kb) {
#pragma unroll
                  for (int kk = 0; kk < KSTEPS; ++kk) {
                    const uint64_t da = smem_desc(smem_u32(tileA + (kb * F::kPA + sa) * kOzSlotA) + kk * 32);
                    const uint64_t db = smem_desc(sb + (kb * F::kPB + (L - sa)) * kOzSlotB + kk * 32);
                    mma_pair<F>(dacc, da, db, idesc, (sa != s0 || kb != 0 || kk != 0) ? 1u : 0u);
                  }
                }
              }
            }
            mma_commit_pair(&tfull[b]);
          }
          if (!ok) break;
          mma_commit_pair(&b_empty[s]);   // the trig stage is free once this tile's MMAs complete
          if (++s == S) {
            s = 0;
            ph ^= 1;
          }
        }
        // the G tile is free once every MMA issued so far has completed
        if (ok) mma_commit_pair(a_empty);
      }
    }
  } else {
    // epilogue: lane quarter `quarter` of the TMEM lanes (32 rows), column
    // group `sub` (NC columns) of each longitude tile
    const int quarter = warp & 3;
    const int sub = (warp - 2) >> 2;
    const uint32_t tempty_even = mapa_rank(smem_u32(&tempty[0]), 0);
    uint8_t *wbuf = epi + (size_t)(warp - 2) * kOzEpiWarpBytes;
    double *ebuf = reinterpret_cast<double *>(wbuf);                            // [32][kOzEpiPad]
    double **rowp = reinterpret_cast<double **>(wbuf + 32 * kOzEpiPad * 8);     // [32] output rows
    const bool vec = (a.ldo & 1) == 0;
    int it = 0;
    bool ok = true;
    for (int t = pair; t < total && ok; t += n_pairs) {
      const OzSynthJob &J = a.job[t / a.cell_tiles];
      const int ct = t % a.cell_tiles;
      const int cell = (2 * ct + rank) * kPairRows + quarter * 32 + lane;
      const bool cell_ok = cell < a.cells;
      const int ce = cell_ok ? J.cell_exp[cell] : 0;
      const bool row_ok = i64_ldexp_row_ok(ce + 16);
      __syncwarp();   // the previous tile's row pointers are no longer read
      rowp[lane] = !cell_ok ? nullptr
                   : (cell < a.out_split) ? J.out0 + (size_t)cell * a.ldo
                                          : J.out1 + (size_t)(cell - a.out_split) * a.ldo;
      for (int ctile = 0; ctile < a.col_tiles && ok; ++ctile) {
        // per output, from the low levels up: lo, then mid (see above)
        int lo[NC], mid[NC];
        const int col_base = ctile * kOzSynthBN + sub * NC;
#pragma unroll 1
        for (int pass = 0; pass < kOzSynthPasses; ++pass, ++it) {
          const int b = it % NB;
          if (!mbar_wait_cluster(&tfull[b], (it / NB) & 1, a.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t tcol = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 256 + sub * NC);
          if (pass < kOzSynthPasses - 1) {
#pragma unroll
            for (int c = 0; c < NC; c += 8) {
              uint32_t uh[8], ul[8];                     // levels 6 - 2 pass and 5 - 2 pass
              tmem_ld8_async(tcol + (uint32_t)c, uh);
              tmem_ld8_async(tcol + 128u + (uint32_t)c, ul);
              tmem_wait_ld();
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                // S_(L-1) 2^8 + S_L of the pair (exact in 32 bits), from the biased patterns
                const int w = (int)((ul[j] << 8) + uh[j] - kOzBias2);
                if (pass == 0)
                  lo[c + j] = (w + 32768) >> 16;               // round((S_5 2^8 + S_6) / 2^16)
                else if (pass == 1)
                  lo[c + j] += w;                              // + S_3 2^8 + S_4
                else
                  mid[c + j] = w;                              // S_1 2^8 + S_2
              }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster_relaxed(tempty_even + (uint32_t)(b * sizeof(uint64_t)));
            continue;
          }
          // level 0: the values 2^(ce + 16) V, staged 8 columns at a time and
          // stored as row runs
#pragma unroll
          for (int c0 = 0; c0 < NC; c0 += 8) {
            uint32_t u0[8];
            tmem_ld8_async(tcol + (uint32_t)c0, u0);
            tmem_wait_ld();
            if (c0 + 8 >= NC) {
              // the accumulators are no longer needed
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive_cluster_relaxed(tempty_even + (uint32_t)(b * sizeof(uint64_t)));
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const long long V = ((long long)(int)(u0[j] - kOzBiasBits) << 32) +
                                  ((long long)mid[c0 + j] << 16) + (long long)lo[c0 + j];
              // the even columns through the float64 pipe's conversion, the
              // odd ones by integer formatting: the epilogue's issue slots are
              // its limit and the float64 pipe is otherwise idle (three of
              // eight: 526 -> 515 us, four: 511, six: 510, the pipe near full)
              ebuf[lane * kOzEpiPad + j] = !row_ok       ? i64_ldexp(V, ce + 16)
                                           : (j % 2 == 0) ? i64_ldexp_row_cvt(V, ce + 16)
                                                          : i64_ldexp_row(V, ce + 16);
            }
            __syncwarp();
            const int col0 = col_base + c0;
            if (vec && col0 + 8 <= a.cols) {
              // the whole run inside the row; lanes 4 c' + e: row 8 q + c', values
              // 2 e and 2 e + 1 of the run
              const int e = lane & 3, col = col0 + 2 * e;
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const int r = 8 * q + (lane >> 2);
                double *orow = rowp[r];
                const double2 val = *reinterpret_cast<const double2 *>(ebuf + r * kOzEpiPad + 2 * e);
                if (orow != nullptr) *reinterpret_cast<double2 *>(orow + col) = val;
              }
            } else if (vec) {
              const int e = lane & 3, col = col0 + 2 * e;
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const int r = 8 * q + (lane >> 2);
                double *orow = rowp[r];
                const double2 val = *reinterpret_cast<const double2 *>(ebuf + r * kOzEpiPad + 2 * e);
                if (orow != nullptr) {
                  if (col + 1 < a.cols)
                    *reinterpret_cast<double2 *>(orow + col) = val;
                  else if (col < a.cols)
                    orow[col] = val.x;
                }
              }
            } else {
              const int e = lane & 7, col = col0 + e;
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                const int r = 4 * q + (lane >> 3);
                double *orow = rowp[r];
                if (orow != nullptr && col < a.cols) orow[col] = ebuf[r * kOzEpiPad + e];
              }
            }
            __syncwarp();   // the staged values are read before the next group overwrites them
          }
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
