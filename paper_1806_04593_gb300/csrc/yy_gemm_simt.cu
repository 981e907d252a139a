// CUDA-core contractions of the solver: float64 (DFMA) and float32 (FFMA).
//
//  analysis   A[2 n_r][n_lm]  = rho[2 n_r][n_ang] . B_an^T      (§3 Eqs. ac/as, §4 weights)
//  synthesis  Phi[2 n_r][n_ang] = Q[2 n_r][n_lm] . Ysyn^T   (§4 sum of four potentials, with
//             the other patch's moments already rotated into each patch's frame)
//
// Both operands are K-major (row m of A and row n of B are contiguous in k),
// rows of A may come from two arrays (Yin rows then Yang rows) and rows of C
// may go to two arrays, so the caller's per-patch buffers are used in place.
// The analysis cuts K into fixed segments (set by the grid's sizes alone) and
// writes one float64 partial per segment, which a second kernel sums in
// segment order; blockIdx.z takes one or more whole segments, so the moments
// are bitwise the same for every K split (deterministic, no atomics).
#include <algorithm>

#include "yy_internal.h"

namespace yy {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4, NT = 256;

template <typename T, typename Acc, bool PARTIAL>
__global__ void __launch_bounds__(NT)
k_gemm_tn(int M, int N, int K, int k_chunk, int seg,
          const T *__restrict__ A0, const T *__restrict__ A1, int a_split, long long lda,
          const T *__restrict__ B, long long ldb,
          double *__restrict__ C0, double *__restrict__ C1, int c_split, long long ldc) {
  __shared__ T As[2][BK][BM + 4];
  __shared__ T Bs[2][BK][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int bm = blockIdx.y * BM, bn = blockIdx.x * BN;
  const int kz0 = blockIdx.z * k_chunk;
  const int kz1 = min(K, kz0 + k_chunk);
  const int lr = tid >> 2, lk = (tid & 3) * 4;
  const int am = bm + lr;
  const T *arow = nullptr;
  if (am < M) arow = (am < a_split) ? A0 + (long long)am * lda : A1 + (long long)(am - a_split) * lda;
  const int bnr = bn + lr;
  const T *brow = (bnr < N) ? B + (long long)bnr * ldb : nullptr;

  Acc acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = Acc(0);

  T ra[4], rb[4];
  auto load = [&](int k0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = k0 + lk + i;
      ra[i] = (arow != nullptr && k < kz1) ? arow[k] : T(0);
      rb[i] = (brow != nullptr && k < kz1) ? brow[k] : T(0);
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      As[buf][lk + i][lr] = ra[i];
      Bs[buf][lk + i][lr] = rb[i];
    }
  };

  const int nk = (kz1 > kz0) ? (kz1 - kz0 + BK - 1) / BK : 0;
  if (nk > 0) {
    load(kz0);
    store(0);
  }
  __syncthreads();
  for (int t = 0; t < nk; ++t) {
    const int buf = t & 1;
    if (t + 1 < nk) load(kz0 + (t + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma((Acc)a[i], (Acc)b[j], acc[i][j]);
    }
    if (PARTIAL) {
      // the end of a K segment (seg is a multiple of BK): its partial goes out
      const int k_next = kz0 + (t + 1) * BK;
      if (k_next % seg == 0 || t + 1 == nk) {
        const size_t zs = (size_t)((kz0 + t * BK) / seg);   // the segment this step belongs to
#pragma unroll
        for (int i = 0; i < TM; ++i) {
          const int m = bm + ty * TM + i;
          if (m < M) {
            double *crow = C0 + zs * M * ldc + (size_t)m * ldc;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
              const int n = bn + tx * TN + j;
              if (n < N) crow[n] = (double)acc[i][j];
            }
          }
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = Acc(0);
        }
      }
    }
    if (t + 1 < nk) store(buf ^ 1);
    __syncthreads();
  }
  if constexpr (!PARTIAL) {
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int m = bm + ty * TM + i;
      if (m >= M) continue;
      double *crow = (m < c_split) ? C0 + (size_t)m * ldc : C1 + (size_t)(m - c_split) * ldc;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int n = bn + tx * TN + j;
        if (n < N) crow[n] = (double)acc[i][j];
      }
    }
  }
}

// out[e] = sum_z part[z][e], z ascending.
__global__ void k_sum_partials(size_t count, int splits, const double *__restrict__ part,
                               double *__restrict__ out) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  double s = 0.0;
  for (int z = 0; z < splits; ++z) s += part[(size_t)z * count + e];
  out[e] = s;
}

__global__ void k_to_f32(size_t count, const double *__restrict__ src, float *__restrict__ dst) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) dst[e] = (float)src[e];
}

__global__ void k_rho_to_f32(size_t per_patch, const double *__restrict__ a, const double *__restrict__ b,
                             float *__restrict__ dst) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < per_patch) {
    dst[e] = (float)a[e];
    if (b) dst[per_patch + e] = (float)b[e];   // no second patch on a polar grid
  }
}

// K in n_seg segments of seg elements (n_seg 1: one unsplit pass writing C0 / C1),
// taken `splits` ways: each z block takes ceil(n_seg / splits) whole segments.
template <typename T, typename Acc>
cudaError_t launch_gemm(int M, int N, int K, int seg, int n_seg, int splits, const T *A0, const T *A1,
                        int a_split, long long lda, const T *B, long long ldb, double *C0, double *C1,
                        int c_split, long long ldc, cudaStream_t s) {
  if (n_seg > 1) {
    const int per = (n_seg + splits - 1) / splits;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, (n_seg + per - 1) / per);
    k_gemm_tn<T, Acc, true><<<grid, NT, 0, s>>>(M, N, K, per * seg, seg, A0, A1, a_split, lda, B, ldb, C0, C1,
                                                c_split, ldc);
  } else {
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, 1);
    k_gemm_tn<T, Acc, false><<<grid, NT, 0, s>>>(M, N, K, K, K, A0, A1, a_split, lda, B, ldb, C0, C1, c_split,
                                                 ldc);
  }
  return cudaGetLastError();
}

}  // namespace

// K segments of the float64 / float32 dense analysis, from the sizes alone:
// about eight blocks per SM at the full split, segments of at least 512.
void simt_segments(int M, int N, int K, int *seg, int *n_seg) {
  const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  int s = (8 * 152 + tiles - 1) / tiles;
  s = std::max(1, std::min(std::min(s, std::max(1, K / 512)), 64));
  const int len = ((K + s - 1) / s + BK - 1) / BK * BK;
  *seg = len;
  *n_seg = (K + len - 1) / len;
}

cudaError_t analysis_simt(yy_grid *g, const double *rho_yin, const double *rho_yang, bool fp32,
                          cudaStream_t s) {
  const int M = grid_rows(g), N = g->n_lm, K = g->n_ang;
  const int n_seg = g->split_k, splits = g->simt_splits;
  double *out = (n_seg > 1) ? g->part : g->A;
  cudaError_t err;
  if (fp32) {
    const size_t pp = (size_t)g->n_r * g->n_ang;
    k_rho_to_f32<<<(unsigned)((pp + 255) / 256), 256, 0, s>>>(pp, rho_yin, rho_yang, g->rho32);
    note_launch(g, "k_rho_to_f32", s);
    err = launch_gemm<float, float>(M, N, K, g->seg_k, n_seg, splits, g->rho32, g->rho32 + pp, g->n_r, K, g->ban32, K,
                                    out, out, M, N, s);
  } else {
    err = launch_gemm<double, double>(M, N, K, g->seg_k, n_seg, splits, rho_yin, rho_yang, g->n_r, K, g->ban, K, out,
                                      out, M, N, s);
  }
  if (err != cudaSuccess) return err;
  note_launch(g, "k_gemm_tn/analysis", s);
  if (n_seg > 1) {
    const size_t count = (size_t)M * N;
    k_sum_partials<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(count, n_seg, g->part, g->A);
    note_launch(g, "k_sum_partials", s);
    err = cudaGetLastError();
  }
  return err;
}

cudaError_t synthesis_simt(yy_grid *g, double *phi_yin, double *phi_yang, double *grad_yin,
                           double *grad_yang, bool fp32, cudaStream_t s) {
  const int M = grid_rows(g), N = g->n_ang, K = g->n_lm;
  const size_t qsz = (size_t)M * K;
  const size_t comp = (size_t)g->n_r * g->n_ang;
  cudaError_t err;
  // Phi = Q . Y ; g_r = Q_r . Y ; g_theta = Q_t . Y_t ; g_phi = Q_t . Y_p
  struct Job {
    int q;
    int table;
    double *c0, *c1;
  } jobs[4] = {{0, 0, phi_yin, phi_yang},
               {1, 0, grad_yin, grad_yang},
               {2, 1, grad_yin ? grad_yin + comp : nullptr, grad_yang ? grad_yang + comp : nullptr},
               {2, 2, grad_yin ? grad_yin + 2 * comp : nullptr, grad_yang ? grad_yang + 2 * comp : nullptr}};
  const int n_jobs = grad_yin ? 4 : 1;
  for (int t = 0; t < n_jobs; ++t) {
    const Job &jb = jobs[t];
    if (fp32) {
      const float *tabs[3] = {g->ysyn32, g->ysyn_t32, g->ysyn_p32};
      const float *Aq = g->Q32 + jb.q * qsz;
      err = launch_gemm<float, float>(M, N, K, K, 1, 1, Aq, Aq, M, K, tabs[jb.table], K, jb.c0, jb.c1,
                                      g->n_r, N, s);
    } else {
      const double *tabs[3] = {g->ysyn, g->ysyn_t, g->ysyn_p};
      const double *Aq = g->Q + jb.q * qsz;
      err = launch_gemm<double, double>(M, N, K, K, 1, 1, Aq, Aq, M, K, tabs[jb.table], K, jb.c0, jb.c1,
                                        g->n_r, N, s);
    }
    if (err != cudaSuccess) return err;
    note_launch(g, "k_gemm_tn/synthesis", s);
  }
  return cudaSuccess;
}

cudaError_t convert_tables_f32(yy_grid *g) {
  const size_t n_ban = (size_t)g->n_lm * g->n_ang;
  const size_t n_syn = (size_t)g->n_ang * g->n_lm;
  cudaError_t err;
  if ((err = dmalloc((void **)&g->ban32, n_ban * sizeof(float))) != cudaSuccess) return err;
  if ((err = dmalloc((void **)&g->ysyn32, n_syn * sizeof(float))) != cudaSuccess) return err;
  if ((err = dmalloc((void **)&g->ysyn_t32, n_syn * sizeof(float))) != cudaSuccess) return err;
  if ((err = dmalloc((void **)&g->ysyn_p32, n_syn * sizeof(float))) != cudaSuccess) return err;
  if ((err = dmalloc((void **)&g->rho32, (size_t)grid_rows(g) * g->n_ang * sizeof(float))) != cudaSuccess)
    return err;
  if ((err = dmalloc((void **)&g->Q32, 3 * (size_t)grid_rows(g) * g->n_lm * sizeof(float))) != cudaSuccess)
    return err;
  k_to_f32<<<(unsigned)((n_ban + 255) / 256), 256>>>(n_ban, g->ban, g->ban32);
  k_to_f32<<<(unsigned)((n_syn + 255) / 256), 256>>>(n_syn, g->ysyn, g->ysyn32);
  k_to_f32<<<(unsigned)((n_syn + 255) / 256), 256>>>(n_syn, g->ysyn_t, g->ysyn_t32);
  k_to_f32<<<(unsigned)((n_syn + 255) / 256), 256>>>(n_syn, g->ysyn_p, g->ysyn_p32);
  return cudaGetLastError();
}

}  // namespace yy
