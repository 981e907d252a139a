// The tensor-core (tcgen05) pair kernel k_tc_pair and what it is built from:
// the precision forms, the tile constants, the PTX wrappers (mbarrier, TMA,
// TMEM, MMA) and the exact fp32 <-> float64 conversions.  Included by
// yy_tc.cu only (the packing, tables and launches).
//
// The two contractions of the solver:
//   analysis   A[2 n_r][n_lm]    = rho . B_an^T   (§3 Eqs. ac/as with the §4 weights)
//   synthesis  Phi[2 n_r][n_ang] = Q . Y^T        (§4 sum of the four potentials,
//                                                  with combined coefficients)
//
// Operands are float64 on entry.  Each is split into pieces of a narrower
// type with a power-of-two scale per row:
//   FP16X2  x = s (h + l), h, l fp16;        products h.h + h.l + l.h
//   BF16X3  x = s (h + m + l), bf16;         products hh hm mh hl lh mm
//   TF32    x = s t, t tf32 (round to nearest);  one product
// The products run on tcgen05.mma (kind::f16 / kind::tf32) from shared memory
// tiles loaded by TMA (64-byte swizzle, K-major), accumulating in fp32 in
// tensor memory; the epilogue warps read TMEM and apply the scales.  The
// analysis is split over K and its fp32 partial sums are added in a fixed
// order.  The monopole (l = 0) column of each contraction is taken out of
// the tensor-core product and done in float64 (it dominates Phi and A;
// keeping it exact keeps the error of the narrow products relative to the
// small l >= 1 part), and the analysis runs on rho minus its row mean, the
// mean's contribution being added back in float64.
//
// The FP64 pipe of this chip retires about two operations per clock per SM,
// so the packing, reduction and epilogue code uses fp32 arithmetic and
// exact integer conversions between fp32 and float64.
//
// Both contractions run on one persistent kernel over pairs of CTAs
// (clusters of two, one CTA per SM, M = 256 per MMA, cta_group::2):
//   warp 0  lane 0: TMA producer over a ring of shared-memory stages
//   warp 1  allocates TMEM (both CTAs); in the even CTA lane 0 issues the
//           MMAs and the commits
//   warps 2-17: epilogue, TMEM lanes 32 (w % 4) .. + 31, 16-column chunks
// Every mbarrier wait gives up after ~2 s, sets the device error word and
// lets the CTA finish (TMEM is always released).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>

#include "yy_internal.h"

namespace yy {


// ---------------------------------------------------------------------------
// precision forms
// ---------------------------------------------------------------------------

enum { KIND_F16 = 0, KIND_BF16 = 1, KIND_TF32 = 2 };

// A form lists its piece products q = 0 .. kPairs - 1 (pieces pa(q) of A and
// pb(q) of B) and the TMEM accumulator acc(q) each goes to; first(q) marks
// the first product of its accumulator in a fill.  The split forms sum every
// product in one accumulator.
struct FormFP16x2 {
  typedef __half elem;
  static constexpr int kKind = KIND_F16, kElem = 2, kPA = 2, kPB = 2, kPairs = 3, kAccs = 1;
  __host__ __device__ static constexpr int pa(int i) { return i == 2 ? 1 : 0; }
  __host__ __device__ static constexpr int pb(int i) { return i == 1 ? 1 : 0; }
  __host__ __device__ static constexpr int acc(int) { return 0; }
  __host__ __device__ static constexpr bool first(int i) { return i == 0; }
};

struct FormBF16x3 {
  typedef __nv_bfloat16 elem;
  static constexpr int kKind = KIND_BF16, kElem = 2, kPA = 3, kPB = 3, kPairs = 6, kAccs = 1;
  // (0,0) (0,1) (1,0) (0,2) (2,0) (1,1)
  __host__ __device__ static constexpr int pa(int i) { return i == 2 ? 1 : (i == 4 ? 2 : (i == 5 ? 1 : 0)); }
  __host__ __device__ static constexpr int pb(int i) { return i == 1 ? 1 : (i == 3 ? 2 : (i == 5 ? 1 : 0)); }
  __host__ __device__ static constexpr int acc(int) { return 0; }
  __host__ __device__ static constexpr bool first(int i) { return i == 0; }
};

struct FormTF32 {
  typedef float elem;
  static constexpr int kKind = KIND_TF32, kElem = 4, kPA = 1, kPB = 1, kPairs = 1, kAccs = 1;
  __host__ __device__ static constexpr int pa(int) { return 0; }
  __host__ __device__ static constexpr int pb(int) { return 0; }
  __host__ __device__ static constexpr int acc(int) { return 0; }
  __host__ __device__ static constexpr bool first(int i) { return i == 0; }
};

constexpr int kRowBytes = 64;        // K bytes per tile row and stage: one 64-byte swizzle atom
constexpr int kPadK = 64;            // K padding (elements) of every packed operand
constexpr double kY00 = 0.28209479177387814347403972578039;   // K_00 P_0^0 = 1/sqrt(4 pi)

constexpr int kEpiWarps = 16;        // four epilogue warps per TMEM lane quarter
constexpr int kEpiPerQuarter = kEpiWarps / 4;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kEpiCols = 16;         // columns per TMEM load
// K elements per accumulator fill of the analysis: the fp32 accumulation error
// of a chain grows with its length times the size of its partial sums, and a
// fill of 256 keeps it near 1e-7 of the moments at K = 24300 (1 degree cells)
constexpr int kAnalysisFill = 256;

// CTA-pair kernel: per CTA and stage, the form's pieces of 128 rows of A and of
// bn / 2 rows of B, each piece one 64-byte-wide swizzled slot.  As many stages
// as the shared memory holds (at most kMaxStages).
constexpr int kPairRows = 128;
constexpr int kPairTmemCols = 512;   // two accumulators of up to 256 columns
// out_mode 2 stages each epilogue warp's 32 x 16 results in shared memory
// (rows padded to 18 doubles: 16-byte accesses without bank conflicts) plus
// its 32 output-row pointers, so that the float64 stores run along the rows
constexpr int kEpiPad = kEpiCols + 2;
constexpr int kEpiWarpBytes = 32 * kEpiPad * 8 + 32 * 8;
constexpr int kEpiStageBytes = kEpiWarps * kEpiWarpBytes;
constexpr int kMaxStages = 16;
constexpr int kSmemLimit = 232448;   // dynamic shared memory of one CTA
constexpr int kSmemFixed = 1024 /*alignment*/ + 512 /*barriers, TMEM address*/;

template <class F>
constexpr int pair_stage_bytes(int bn) {
  return (F::kPA * kPairRows + F::kPB * (bn / 2)) * kRowBytes;
}
template <class F>
int pair_stages(int bn, int reserve = 0) {
  const int s = (kSmemLimit - kSmemFixed - reserve) / pair_stage_bytes<F>(bn);
  return s < kMaxStages ? s : kMaxStages;
}

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait: ~2 s of wall time, then the error word gets YY_DEVERR_TIMEOUT.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err) {
  const uint32_t addr = smem_u32(bar);
  for (int i = 0; i < 256; ++i)
    if (mbar_try_wait(addr, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (true) {
    if (mbar_try_wait(addr, parity)) return true;
    if (globaltimer() - t0 > 2000000000ull) {
      atomicOr(err, YY_DEVERR_TIMEOUT);
      return false;
    }
  }
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 64-byte swizzle (layout type 4),
// 8-row groups 512 bytes apart (stride byte offset), descriptor version 1.
// The tile base must be 512-byte aligned; advancing K by 32 bytes inside the
// swizzle atom advances the start address.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

// 16 columns of this warp's 32 TMEM lanes, without waiting (tmem_wait_ld).
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld8_async(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Zeros into 16 columns of this warp's 32 TMEM lanes, and the wait for a
// thread's TMEM stores.
__device__ __forceinline__ void tmem_zero16(uint32_t taddr) {
  const uint32_t z = 0u;
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr),
      "r"(z)
      : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ---- CTA-pair (cta_group::2) forms -------------------------------------
//
// Two CTAs of a cluster share one MMA of M = 256: the even CTA issues it; each
// CTA holds 128 rows of A and half the columns of B in its own shared memory
// and 128 lanes of the accumulator in its own TMEM.

// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa_rank(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

// Bounded wait with cluster-scope acquire (arrivals may come from the peer).
__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_cluster(uint64_t *bar, uint32_t parity, int *err) {
  const uint32_t addr = smem_u32(bar);
  for (int i = 0; i < 256; ++i)
    if (mbar_try_wait_cluster(addr, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (true) {
    if (mbar_try_wait_cluster(addr, parity)) return true;
    if (globaltimer() - t0 > 2000000000ull) {
      atomicOr(err, YY_DEVERR_TIMEOUT);
      return false;
    }
  }
}

// Arrive on a barrier given by its shared::cluster address (own or peer CTA).
// Release of a TMEM accumulator by an epilogue warp.  Its tcgen05.ld have
// completed (tcgen05.wait::ld) and are fenced (tcgen05.fence::before_thread_sync)
// before this arrive, so the MMAs that follow the barrier cannot disturb
// them; nothing else needs ordering, in particular not the warp's global
// stores, which a release arrive would wait for.
__device__ __forceinline__ void mbar_arrive_cluster_relaxed(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

// TMA load into this CTA's shared memory that completes on a barrier of
// either CTA of the pair (cluster address).
__device__ __forceinline__ void tma_load_2d_pair(const CUtensorMap *map, uint32_t dst, uint32_t bar_cluster, int x,
                                                 int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"((uint64_t)map), "r"(bar_cluster), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tmem_alloc_pair(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc_pair(uint32_t base, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols) : "memory");
}

template <class F>
__device__ __forceinline__ void mma_pair(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (F::kKind == KIND_TF32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  }
}

// Arrive on the barrier at this offset in both CTAs of the pair once the
// MMAs issued before it have completed.
__device__ __forceinline__ void mma_commit_pair(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"((uint16_t)3)
      : "memory");
}

// Instruction descriptor of the pair MMA: M = 256, N = n (multiple of 16, <= 256).
template <class F>
__host__ __device__ constexpr uint32_t instr_desc_pair(int n) {
  return (1u << 4) | ((uint32_t)F::kKind << 7) | ((uint32_t)F::kKind << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(256 >> 4) << 24);
}

// fp32 <-> float64 with integer operations only: exact widening, and
// round-to-nearest-even narrowing (the same result as the conversion
// instruction); zero / subnormal / overflow / NaN take the instruction.
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t ex = (u >> 23) & 0xFFu;
  if (ex == 0u || ex == 255u) {
    if ((u << 1) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
    return (double)f;
  }
  const uint32_t hi = (u & 0x80000000u) | ((ex + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}

__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(u >> 32);
  const int ex = (int)((hi >> 20) & 0x7FFu);
  const int e32 = ex - 1023 + 127;
  if (e32 <= 0 || e32 >= 255) {
    if ((u << 1) == 0ull) return __uint_as_float(hi & 0x80000000u);
    return (float)x;
  }
  const unsigned long long man = u & 0xFFFFFFFFFFFFFull;
  const uint32_t m23 = (uint32_t)(man >> 29);
  const uint32_t rem = (uint32_t)(man & 0x1FFFFFFFull);
  const uint32_t up = (rem > 0x10000000u || (rem == 0x10000000u && (m23 & 1u))) ? 1u : 0u;
  return __uint_as_float((hi & 0x80000000u) | (((uint32_t)e32 << 23) + m23 + up));
}

}  // namespace yy

// the Ozaki forms (float64 results from exact bf16 digit products) and their
// epilogue, for out_mode 3
#include "yy_tc_ozaki.cuh"

namespace yy {

// ---------------------------------------------------------------------------
// the synthesis kernel: CTA pairs, M = 256 cells x N = bn coefficient rows
// ---------------------------------------------------------------------------
//
// out[row][cell] = (sum_k Y[cell][k] Q[row][k]) cell_scale[cell] row_scale[row] + row_add[row]
// with Y a packed table (operand A, one row per cell) and Q packed
// coefficients (operand B), for up to four jobs (Phi, g_r, g_theta, g_phi)
// in one launch.  The analysis uses the same kernel with the analysis table
// as A (one row per mode), the densities as B, K split over tiles, and raw
// fp32 partial sums as output (out_mode 0).  Clusters of two CTAs; pair p handles tiles p, p + #pairs,
// ... of the job-major tile list (coefficient-row tiles fastest, so the
// pairs working at the same time share table tiles in L2).  Per stage each CTA loads its 128
// table rows and its bn / 2 coefficient rows; both CTAs' loads complete on
// the even CTA's "full" barrier, whose thread 32 issues the M = 256 MMAs and
// releases each stage in both CTAs with a multicast commit.  Each CTA's TMEM
// holds its 128 cells x bn accumulator (double-buffered), so a lane of an
// epilogue warp owns one cell and a 16-column TMEM load gives it 16 rows:
// every store is 32 consecutive cells of one output row.  The epilogue warps
// of both CTAs release a buffer on the even CTA's "tempty" barrier.
struct PairJob {
  double *out0, *out1;          // row r < out_split -> out0 + r ldo, else out1 + (r - out_split) ldo
                                // (out_mode 2: cell c < out_split -> out0 + c ldo, ...)
  const float *cell_scale, *row_scale, *row_add;
  const float *cell_add;        // out_mode 2: added to every value of the cell
  const int *cell_exp;          // out_mode 3: power of two of a unit level-6 sum in the cell's row
  int ta, tb;                   // operand maps of this job
};

struct PairArgs {
  int stages;                   // shared-memory stages (pair_stages)
  int cells, cell_tiles;        // valid A rows ("cells"); tiles of 256
  int rows, row_tiles, bn;      // valid B rows; tiles of bn rows (multiple of 16, <= 256)
  int kb_total;                 // K blocks (kRowBytes per row)
  int k_splits, kb_per_split;   // K split of every tile
  int kb_chunk;                 // K blocks per accumulator fill; mode 0 adds the fills in registers
  int k_segs, segs_per_split;   // mode 0: K segments (0: none) -- segment z starts at K block
                                // floor(z kb_total / k_segs), a split takes segs_per_split whole
                                // segments, fills restart at every segment and each segment's
                                // sums go out as one partial
  int a_rows, b_rows;           // rows of one piece in the stacked A / B operands
  int out_mode;                 // 1: scaled float64 job outputs; 0: raw fp32 partial sums;
                                // 2: scaled float64 outputs stored along the rows of each cell;
                                // 3: as 2, from the exact level sums of FormOzaki;
                                // 4: as 3 with one fill and biased level sums
  float *part;                  // mode 0: part[(segment rows + row) part_ld + cell]
  int part_ld;
  int out_split;
  long long ldo;
  int n_jobs;
  PairJob job[4];
  int *err;
  // grouped launch (k_tc_pair<F, MODE, true>): the fields' own arguments and
  // tensor maps in global memory; this struct then gives only the stage count,
  // the largest field's bn (the shared-memory layout) and the error word
  const struct PairArgs *group;
  const struct PairMaps *group_maps;
  int n_group;
};

struct PairMaps {
  CUtensorMap a[4], b[3];       // tables (operand A), coefficient sets (operand B)
};

// First K block of segment z (of k_segs) of the K axis.
__device__ __forceinline__ int seg_start(const PairArgs &a, int z) {
  return (int)(((long long)z * a.kb_total) / a.k_segs);
}

// The K blocks of split z of a tile, [kb0, kb0 + nkb), walked in fills of
// `chunk` blocks that restart at every segment start.  seg is the current
// segment (the split's own index when K has no segments), seg_end its end
// relative to kb0.
struct TileFills {
  int kb0, nkb, seg, seg_end;
  __device__ __forceinline__ TileFills(const PairArgs &a, int z) {
    if (a.k_segs > 0) {
      seg = z * a.segs_per_split;
      kb0 = seg_start(a, seg);
      nkb = seg_start(a, min(a.k_segs, seg + a.segs_per_split)) - kb0;
      seg_end = seg_start(a, seg + 1) - kb0;
    } else {
      seg = z;
      kb0 = z * a.kb_per_split;
      nkb = min(a.kb_total, kb0 + a.kb_per_split) - kb0;
      seg_end = nkb;
    }
  }
  // end (relative to kb0) of the fill that starts at c0
  __device__ __forceinline__ int fill_end(int c0, int chunk) const { return min(c0 + chunk, seg_end); }
  // after the fill ending at c1: whether it closed segment `seg`; if so, and
  // more follow, move on to the next (the caller reads seg first)
  __device__ __forceinline__ bool closes(int c1) const { return c1 == seg_end; }
  __device__ __forceinline__ void advance(const PairArgs &a, int c1) {
    if (c1 == seg_end && c1 < nkb) {
      ++seg;
      seg_end = seg_start(a, seg + 1) - kb0;
    }
  }
};

// The tiles of one launch in order: field by field (one field unless the
// launch is grouped), each field's tiles as its own launch would order them.
// Pair p takes the tiles p, p + #pairs, ... of the whole sequence: from
// (field f, its tile t) this moves on to the next such tile, crossing into
// later fields; false past the last field.  base: tiles of the fields before f.
template <bool GROUPED>
__device__ __forceinline__ bool pair_tile_next(const PairArgs &a0, int pair, int n_pairs, int &f, int &base, int &t) {
  const int nf = GROUPED ? a0.n_group : 1;
  while (f < nf) {
    const PairArgs &a = GROUPED ? a0.group[f] : a0;
    const int total = a.cell_tiles * a.row_tiles * a.k_splits * a.n_jobs;
    if (t < total) return true;
    base += total;
    ++f;
    t = ((pair - base) % n_pairs + n_pairs) % n_pairs;
  }
  return false;
}

template <class F, int OUT_MODE, bool GROUPED = false>
__global__ void __launch_bounds__(kThreads, 1)
k_tc_pair(const __grid_constant__ PairMaps maps0, const __grid_constant__ PairArgs a0) {
  constexpr int A_SLOT = kPairRows * kRowBytes;
  constexpr int KSTEP_BYTES = 32;
  constexpr int KSTEPS = kRowBytes / KSTEP_BYTES;
  constexpr int BK = kRowBytes / F::kElem;

  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int S = a0.stages;
  // B slots sized for a0.bn (grouped: the largest field's); a field's tiles fill their first bn / 2 rows
  const int B_SLOT = (a0.bn >> 1) * kRowBytes;       // a multiple of 512 bytes (bn / 2 % 8 == 0)
  const int STAGE = F::kPA * A_SLOT + F::kPB * B_SLOT;
  uint64_t *full = (uint64_t *)(smem + S * STAGE);
  uint64_t *empty = full + S;
  uint64_t *tfull = empty + S;      // [2]
  uint64_t *tempty = tfull + 2;     // [2], counted in the even CTA
  uint32_t *tmem_slot = (uint32_t *)(tempty + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rank = (int)cluster_rank();
  const int pair = (int)blockIdx.x >> 1, n_pairs = (int)gridDim.x >> 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
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
  cluster_sync();   // both CTAs' barriers and TMEM exist before any remote use
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int gk = 0, s = 0;
      uint32_t ph = 0;   // phase of stage s in the ring (gk / S) & 1
      bool ok = true;
      for (int f_ = 0, base_ = 0, t = pair; ok && pair_tile_next<GROUPED>(a0, pair, n_pairs, f_, base_, t);
           t += n_pairs) {
        const PairArgs &a = GROUPED ? a0.group[f_] : a0;
        const PairMaps &maps = GROUPED ? a0.group_maps[f_] : maps0;
        const int per_job = a.cell_tiles * a.row_tiles * a.k_splits;
        const int bh = a.bn >> 1;
        const uint32_t tx_bytes = 2u * (uint32_t)(F::kPA * kPairRows + F::kPB * bh) * kRowBytes;
        const int jb = t / per_job, tl = t % per_job;
        const int rt = tl % a.row_tiles, ct = (tl / a.row_tiles) % a.cell_tiles;
        const TileFills tf(a, tl / (a.row_tiles * a.cell_tiles));
        const int kb0 = tf.kb0, nkb = tf.nkb;
        const int arow = (2 * ct + rank) * kPairRows;
        const int brow = rt * a.bn + rank * bh;
        const CUtensorMap *tmA = &maps.a[a.job[jb].ta];
        const CUtensorMap *tmB = &maps.b[a.job[jb].tb];
        if constexpr (GROUPED) {
          // the field's tensor maps live in device memory (written before the launch)
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmA) : "memory");
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmB) : "memory");
          asm volatile("prefetch.tensormap [%0];" ::"l"(tmA) : "memory");
          asm volatile("prefetch.tensormap [%0];" ::"l"(tmB) : "memory");
        }
        for (int i = 0; i < nkb; ++i, ++gk) {
          if (gk >= S && !mbar_wait(&empty[s], ph ^ 1, a.err)) {
            ok = false;
            break;
          }
          if (rank == 0) mbar_expect_tx(&full[s], tx_bytes);
          const uint32_t fbar = mapa_rank(smem_u32(&full[s]), 0);
          const uint32_t base = smem_u32(smem + s * STAGE);
          const int kx = (kb0 + i) * BK;
#pragma unroll
          for (int p = 0; p < F::kPA; ++p) tma_load_2d_pair(tmA, base + p * A_SLOT, fbar, kx, p * a.a_rows + arow);
#pragma unroll
          for (int p = 0; p < F::kPB; ++p)
            tma_load_2d_pair(tmB, base + F::kPA * A_SLOT + p * B_SLOT, fbar, kx, p * a.b_rows + brow);
          if (++s == S) {
            s = 0;
            ph ^= 1;
          }
        }
      }
      // the last uses of every stage must be complete before this CTA leaves
      if (ok)
        for (int i = max(0, gk - S); i < gk; ++i)
          if (!mbar_wait(&empty[i % S], (i / S) & 1, a0.err)) break;
    }
  } else if (warp == 1) {
    if (rank == 0 && lane == 0) {
      int gk = 0, it = 0, s = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int f_ = 0, base_ = 0, t = pair; ok && pair_tile_next<GROUPED>(a0, pair, n_pairs, f_, base_, t);
           t += n_pairs) {
        const PairArgs &a = GROUPED ? a0.group[f_] : a0;
        const int per_job = a.cell_tiles * a.row_tiles * a.k_splits;
        // K blocks per accumulator fill (modes 0 and 3 add the fills in the epilogue)
        const int chunk = ((OUT_MODE == 0 || OUT_MODE == 3) && a.kb_chunk > 0) ? a.kb_chunk : a.kb_total;
        const uint32_t idesc = instr_desc_pair<F>(a.bn);
        const int tl = t % per_job;
        TileFills tf(a, tl / (a.row_tiles * a.cell_tiles));
        const int nkb = tf.nkb;
        // the tile's K blocks in fills of kb_chunk, alternating between the two accumulators
        for (int c0 = 0, c1 = 0; c0 < nkb && ok; c0 = c1, ++it) {
          c1 = tf.fill_end(c0, chunk);
          tf.advance(a, c1);
          const int b = it & 1;
          if (it >= 2) {
            if (!mbar_wait_cluster(&tempty[b], ((it >> 1) & 1) ^ 1, a.err)) {
              ok = false;
              break;
            }
            tc_fence_after();
          }
          const uint32_t dacc = tmem_base + (uint32_t)(b * 256);   // accumulator a at + a bn
          for (int i = c0; i < c1; ++i, ++gk) {
            if (!mbar_wait_cluster(&full[s], ph, a.err)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + s * STAGE);
            const uint32_t sb = sa + F::kPA * A_SLOT;
#pragma unroll
            for (int q = 0; q < F::kPairs; ++q) {
              const uint32_t dq = dacc + (uint32_t)(F::acc(q) * a.bn);
#pragma unroll
              for (int kk = 0; kk < KSTEPS; ++kk) {
                const uint64_t da = smem_desc(sa + F::pa(q) * A_SLOT + kk * KSTEP_BYTES);
                const uint64_t db = smem_desc(sb + F::pb(q) * B_SLOT + kk * KSTEP_BYTES);
                mma_pair<F>(dq, da, db, idesc, (((i - c0) | kk) != 0 || !F::first(q)) ? 1u : 0u);
              }
            }
            mma_commit_pair(&empty[s]);
            if (++s == S) {
              s = 0;
              ph ^= 1;
            }
          }
          if (ok) mma_commit_pair(&tfull[b]);
        }
      }
    }
  } else {
    // Lane quarter of this warp's TMEM lanes; the warps of a quarter take
    // 16-column chunks sub, sub + kEpiPerQuarter, ...  The 16 rows of a chunk are one aligned run (row0 is a multiple
    // of 16 and the scale arrays are padded to whole tiles), so their scales
    // arrive as warp-uniform vector loads and their output rows follow from
    // one base pointer (unless the run crosses from Yin into Yang).
    const int quarter = warp & 3;
    const int sub = (warp - 2) >> 2;    // 0 .. kEpiPerQuarter - 1 within the lane quarter
    const uint32_t tempty_even = mapa_rank(smem_u32(&tempty[0]), 0);
    constexpr bool scaled = OUT_MODE == 1;
    int it = 0;
    if constexpr (OUT_MODE == 0) {
      // Segment partial sums: the tile's accumulator fills (kb_chunk K blocks
      // each) are added here in fp32 registers, so no fp32 accumulation chain
      // in the tensor core runs longer than one fill, and each K segment
      // (k_segs of them, fixed by the sizes; a split takes whole segments and
      // fills restart at each) goes out as its own partial: the same fills
      // are added in the same order whatever the split.  This warp owns 16-column chunks sub,
      // sub + kEpiPerQuarter, ... (at most kMaxOwn of them).
      constexpr int kMaxOwn = 256 / kEpiCols / kEpiPerQuarter;
      for (int f_ = 0, base_ = 0, t = pair; pair_tile_next<GROUPED>(a0, pair, n_pairs, f_, base_, t); t += n_pairs) {
        const PairArgs &a = GROUPED ? a0.group[f_] : a0;
        const int per_job = a.cell_tiles * a.row_tiles * a.k_splits;
        // K blocks per accumulator fill (modes 0 and 3 add the fills in the epilogue)
        const int chunk = ((OUT_MODE == 0 || OUT_MODE == 3) && a.kb_chunk > 0) ? a.kb_chunk : a.kb_total;
        const int n_chunks = a.bn / kEpiCols;
        const int tl = t % per_job;
        const int rt = tl % a.row_tiles, ct = (tl / a.row_tiles) % a.cell_tiles;
        TileFills tf(a, tl / (a.row_tiles * a.cell_tiles));
        const int nkb = tf.nkb;
        const int cell = (2 * ct + rank) * kPairRows + quarter * 32 + lane;
        float acc[kMaxOwn][kEpiCols];
#pragma unroll
        for (int o = 0; o < kMaxOwn; ++o)
#pragma unroll
          for (int j = 0; j < kEpiCols; ++j) acc[o][j] = 0.0f;
        bool ok = true;
        for (int c0 = 0, c1 = 0; c0 < nkb; c0 = c1, ++it) {
          c1 = tf.fill_end(c0, chunk);
          const int b = it & 1;
          if (!mbar_wait_cluster(&tfull[b], (it >> 1) & 1, a.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 256);
#pragma unroll
          for (int o = 0; o < kMaxOwn; ++o) {
            const int k = sub + o * kEpiPerQuarter;
            if (k < n_chunks) {
              uint32_t v[16];
              tmem_ld16_async(tbase + (uint32_t)(k * kEpiCols), v);
              tmem_wait_ld();
#pragma unroll
              for (int j = 0; j < kEpiCols; ++j) acc[o][j] += __uint_as_float(v[j]);
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive_cluster_relaxed(tempty_even + (uint32_t)(b * sizeof(uint64_t)));
          if (!tf.closes(c1)) continue;
          // the end of a segment: its partial sums go out
          const size_t zs = (size_t)tf.seg;
          tf.advance(a, c1);
          const int rows_v = a.rows, bn = a.bn, part_ld = a.part_ld;
          float *const part = a.part;
          const bool cell_ok = cell < a.cells;
#pragma unroll
          for (int o = 0; o < kMaxOwn; ++o) {
            const int k = sub + o * kEpiPerQuarter;
            if (k < n_chunks && cell_ok) {
#pragma unroll
              for (int j = 0; j < kEpiCols; ++j) {
                const int row = rt * bn + k * kEpiCols + j;
                if (row < rows_v) part[(zs * rows_v + row) * part_ld + cell] = acc[o][j];
              }
            }
#pragma unroll
            for (int j = 0; j < kEpiCols; ++j) acc[o][j] = 0.0f;
          }
        }
        if (!ok) break;
      }
    } else if constexpr (OUT_MODE == 2 || OUT_MODE == 3 || OUT_MODE == 4) {
      // Cells are rows of the output arrays (stride ldo) and the accumulator
      // columns run along them: each lane holds 16 consecutive values of its
      // cell's row.  They go through this warp's shared-memory block, and the
      // warp then writes two cells' 16-value runs per store instruction.
      // Mode 3 forms the values from FormOzaki's level accumulators.
      static_assert(!GROUPED, "grouped launches take output modes 0 and 1");
      const PairArgs &a = a0;
      const int per_job = a.cell_tiles * a.row_tiles * a.k_splits;
      const int total = per_job * a.n_jobs;
      const int chunk = (OUT_MODE == 3 && a.kb_chunk > 0) ? a.kb_chunk : a.kb_total;
      const int n_chunks = a.bn / kEpiCols;
      uint8_t *wbuf = smem + S * STAGE + 512 + (size_t)(warp - 2) * kEpiWarpBytes;
      double *ebuf = reinterpret_cast<double *>(wbuf);                          // [32][kEpiPad]
      double **rowp = reinterpret_cast<double **>(wbuf + 32 * kEpiPad * 8);     // [32] output rows
      const bool vec = (a.ldo & 1) == 0;   // rows start on 16-byte boundaries (with 16-byte aligned bases)
      if constexpr (OUT_MODE == 3 || OUT_MODE == 4) {
        // FormOzaki: the tile's fills (kb_chunk K blocks each) are added in
        // registers, level by level; this warp owns the 8-column chunk sub
        // (bn <= 8 kEpiPerQuarter), and the values are formed after the last fill.
        // Mode 4 has one fill with biased level sums (ozaki_biased8) and forms
        // the values straight from the accumulator.
        const int k = sub;
        const bool mine = k < a.bn / 8;
        for (int t = pair; t < total; t += n_pairs) {
          const PairJob &J = a.job[t / per_job];
          const int tl = t % per_job;
          const int rt = tl % a.row_tiles, ct = (tl / a.row_tiles) % a.cell_tiles;
          TileFills tf(a, tl / (a.row_tiles * a.cell_tiles));
          const int nkb = tf.nkb;
          const int cell = (2 * ct + rank) * kPairRows + quarter * 32 + lane;
          const bool cell_ok = cell < a.cells;
          const int ce = cell_ok ? J.cell_exp[cell] : 0;
          __syncwarp();   // the previous tile's row pointers are no longer read
          rowp[lane] = !cell_ok ? nullptr
                       : (cell < a.out_split) ? J.out0 + (size_t)cell * a.ldo
                                              : J.out1 + (size_t)(cell - a.out_split) * a.ldo;
          long long hi[8];
          float lo[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            hi[j] = 0;
            lo[j] = 0.0f;
          }
          bool ok = true;
          for (int c0 = 0, c1 = 0; c0 < nkb; c0 = c1, ++it) {
            c1 = tf.fill_end(c0, chunk);
            tf.advance(a, c1);
            const int b = it & 1;
            if (!mbar_wait_cluster(&tfull[b], (it >> 1) & 1, a.err)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 256);
            if (mine) {
              if constexpr (OUT_MODE == 4)
                ozaki_biased8(tbase + (uint32_t)(k * 8), a.bn, ce, ebuf + lane * kEpiPad);
              else
                ozaki_accumulate(tbase + (uint32_t)(k * 8), a.bn, hi, lo);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster_relaxed(tempty_even + (uint32_t)(b * sizeof(uint64_t)));
          }
          if (!ok) break;
          if (mine) {
            const int row0 = rt * a.bn + k * 8;
            if constexpr (OUT_MODE == 3) ozaki_finish(hi, lo, ce, ebuf + lane * kEpiPad);
            __syncwarp();
            if (vec) {
              // lanes 4 c' + e: cell 8 q + c', values 2 e and 2 e + 1 of the run
              const int e = lane & 3, row = row0 + 2 * e;
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const int c = 8 * q + (lane >> 2);
                double *orow = rowp[c];
                const double2 val = *reinterpret_cast<const double2 *>(ebuf + c * kEpiPad + 2 * e);
                if (orow != nullptr) {
                  if (row + 1 < a.rows)
                    *reinterpret_cast<double2 *>(orow + row) = val;
                  else if (row < a.rows)
                    orow[row] = val.x;
                }
              }
            } else {
              const int e = lane & 7, row = row0 + e;
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                const int c = 4 * q + (lane >> 3);
                double *orow = rowp[c];
                if (orow != nullptr && row < a.rows) orow[row] = ebuf[c * kEpiPad + e];
              }
            }
            __syncwarp();
          }
        }
      } else
      for (int t = pair; t < total; t += n_pairs, ++it) {
        const int b = it & 1;
        const PairJob &J = a.job[t / per_job];
        const int tl = t % per_job;
        const int rt = tl % a.row_tiles, ct = (tl / a.row_tiles) % a.cell_tiles;
        const int cell0 = (2 * ct + rank) * kPairRows + quarter * 32;
        const int cell = cell0 + lane;
        const bool cell_ok = cell < a.cells;
        const float cs = cell_ok ? J.cell_scale[cell] : 0.0f;
        const float ca = cell_ok ? J.cell_add[cell] : 0.0f;
        __syncwarp();   // the previous tile's row pointers are no longer read
        rowp[lane] = !cell_ok ? nullptr
                     : (cell < a.out_split) ? J.out0 + (size_t)cell * a.ldo
                                            : J.out1 + (size_t)(cell - a.out_split) * a.ldo;
        if (!mbar_wait_cluster(&tfull[b], (it >> 1) & 1, a.err)) break;
        tc_fence_after();
        const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 256);
        {
#pragma unroll 1
        for (int k = sub; k < n_chunks; k += kEpiPerQuarter) {
          const int row0 = rt * a.bn + k * kEpiCols;
          {
            uint32_t v[16];
            tmem_ld16_async(tbase + (uint32_t)(k * kEpiCols), v);
            float4 rs4[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) rs4[q] = reinterpret_cast<const float4 *>(J.row_scale + row0)[q];
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < kEpiCols; j += 2) {
              const float4 r4 = rs4[j >> 2];
              const float ra = (j & 2) ? r4.z : r4.x, rb = (j & 2) ? r4.w : r4.y;
              *reinterpret_cast<double2 *>(ebuf + lane * kEpiPad + j) =
                  make_double2(f32_to_f64(fmaf(__uint_as_float(v[j]) * cs, ra, ca)),
                               f32_to_f64(fmaf(__uint_as_float(v[j + 1]) * cs, rb, ca)));
            }
          }
          __syncwarp();
          if (vec) {
            // lanes 8 c' + e: cell 4 q + c', values 2 e and 2 e + 1 of the run
            const int e = lane & 7, row = row0 + 2 * e;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int c = 4 * q + (lane >> 3);
              double *orow = rowp[c];
              const double2 val = *reinterpret_cast<const double2 *>(ebuf + c * kEpiPad + 2 * e);
              if (orow != nullptr) {
                if (row + 1 < a.rows)
                  *reinterpret_cast<double2 *>(orow + row) = val;
                else if (row < a.rows)
                  orow[row] = val.x;
              }
            }
          } else {
            const int e = lane & 15, row = row0 + e;
#pragma unroll 4
            for (int q = 0; q < 16; ++q) {
              const int c = 2 * q + (lane >> 4);
              double *orow = rowp[c];
              if (orow != nullptr && row < a.rows) orow[row] = ebuf[c * kEpiPad + e];
            }
          }
          __syncwarp();
        }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster_relaxed(tempty_even + (uint32_t)(b * sizeof(uint64_t)));
      }
    } else
    for (int f_ = 0, base_ = 0, t = pair; pair_tile_next<GROUPED>(a0, pair, n_pairs, f_, base_, t); t += n_pairs, ++it) {
      const PairArgs &a = GROUPED ? a0.group[f_] : a0;
      const int per_job = a.cell_tiles * a.row_tiles * a.k_splits;
      const int n_chunks = a.bn / kEpiCols;
      const int b = it & 1;
      const PairJob &J = a.job[t / per_job];
      const int tl = t % per_job;
      const int rt = tl % a.row_tiles, ct = (tl / a.row_tiles) % a.cell_tiles;
      const int cell = (2 * ct + rank) * kPairRows + quarter * 32 + lane;
      const bool cell_ok = cell < a.cells;
      const float cs = (cell_ok && scaled) ? J.cell_scale[cell] : 0.0f;
      // the tile's arguments in registers (the output stores could otherwise
      // alias them in a grouped launch, whose arguments are in device memory)
      const int rows_v = a.rows, out_split = a.out_split, bn = a.bn;
      const long long ldo = a.ldo;
      double *const out0 = J.out0, *const out1 = J.out1;
      const float *const row_scale = J.row_scale, *const row_add = J.row_add;
      if (!mbar_wait_cluster(&tfull[b], (it >> 1) & 1, a.err)) break;
      tc_fence_after();
      const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 256);
#pragma unroll 1
      for (int k = sub; k < n_chunks; k += kEpiPerQuarter) {
        const int row0 = rt * bn + k * kEpiCols;
        uint32_t v[16];
        tmem_ld16_async(tbase + (uint32_t)(k * kEpiCols), v);
        if constexpr (scaled) {
          float4 rs4[4], ra4[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            rs4[q] = reinterpret_cast<const float4 *>(row_scale + row0)[q];
            ra4[q] = reinterpret_cast<const float4 *>(row_add + row0)[q];
          }
          const bool cross = row0 < out_split && row0 + kEpiCols > out_split;
          double *base = (row0 < out_split) ? out0 + (size_t)row0 * ldo : out1 + (size_t)(row0 - out_split) * ldo;
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < kEpiCols; ++j) {
            const float4 r4 = rs4[j >> 2], a4 = ra4[j >> 2];
            const float rs = (j & 3) == 0 ? r4.x : (j & 3) == 1 ? r4.y : (j & 3) == 2 ? r4.z : r4.w;
            const float ra = (j & 3) == 0 ? a4.x : (j & 3) == 1 ? a4.y : (j & 3) == 2 ? a4.z : a4.w;
            const int row = row0 + j;
            double *orow = base + (size_t)j * ldo;
            if (cross) orow = (row < out_split) ? out0 + (size_t)row * ldo : out1 + (size_t)(row - out_split) * ldo;
            if (row < rows_v && cell_ok) orow[cell] = f32_to_f64(fmaf(__uint_as_float(v[j]) * cs, rs, ra));
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster_relaxed(tempty_even + (uint32_t)(b * sizeof(uint64_t)));
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
