// Allocation-free variant of the radial scan kernel: yy_radial_scan_static.
//
// Some callers cannot allocate device memory at the point where they need the
// radial sums: applications whose device memory is handed out entirely by
// their own pool or arena (an allocation outside it fails or breaks their
// accounting), hosts that load this code as a plugin and forbid it to touch
// the allocator, and time-critical loops where cudaMalloc / cudaFree, which
// may synchronise the device, are not allowed.  This entry point needs no
// handle and allocates nothing: its only scratch (the inner-scan values kept
// between the two passes) lives in the file-scope array below, which every
// GPU that loads the library holds until the process exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "yy_internal.h"

namespace {

// Scratch capacity in float64 values: 2 * n_r * (l_max + 1)^2 must fit.
constexpr size_t kScanScratchDoubles = size_t(1) << 21;   // 16 MiB per device
constexpr int kMaxDevices = 64;
constexpr double kFourPi = 12.566370614359172953850573533118;

__device__ __align__(256) double yy_scan_scratch[kScanScratchDoubles];

// Device address of yy_scan_scratch, resolved at set-up once per device and
// per CUDA context on it: a new primary context (after cudaDeviceReset, say)
// loads the module again, and the array may then sit elsewhere, so the cache
// is keyed on the context's unique id as well as the device.
struct ScratchSlot {
  unsigned long long ctx_id;
  double *addr;
  bool shared_ok;   // k_radial_scan_static_shared may use kSharedZones zones of shared memory
};
ScratchSlot g_scratch[kMaxDevices];
std::mutex g_setup_mutex;

PFN_cuCtxGetCurrent_v4000 g_ctx_current = nullptr;
PFN_cuCtxGetId_v12000 g_ctx_id = nullptr;

bool driver_entry_points() {
  if (g_ctx_current && g_ctx_id) return true;
  cudaDriverEntryPointQueryResult q;
  void *p = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return false;
  g_ctx_current = (PFN_cuCtxGetCurrent_v4000)p;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return false;
  g_ctx_id = (PFN_cuCtxGetId_v12000)p;
  return true;
}

// Zone factors of the scaled recurrences (the formulas of the per-grid scan
// table, computed here on the fly): inner c_n = a c_{n-1} + b A_n, with
// a = (r_n^- / r_n^+)^(l+1) and b = (r_n^+)^2 (1 - (r_n^- / r_n^+)^(l+3)) / (l+3);
// outer d_n = e d_{n+1} + f A_{n+1}, with e = (r_n^+ / r_{n+1}^+)^l and
// f = (r_n^+)^2 ((r_{n+1}^+ / r_n^+)^(2-l) - 1) / (2 - l) (log for l = 2).
__device__ __forceinline__ void inner_factors(int n, int l, const double *__restrict__ r, double &a, double &b) {
  const double r0 = r[n], r1 = r[n + 1];
  const double lq = (r0 > 0.0) ? log(r0 / r1) : -INFINITY;
  a = exp((l + 1.0) * lq);
  b = r1 * r1 * (-expm1((l + 3.0) * lq)) / (l + 3.0);
}

__device__ __forceinline__ void outer_factors(int n, int l, int n_r, const double *__restrict__ r, double &e,
                                              double &f) {
  e = 0.0;
  f = 0.0;
  if (n + 1 < n_r) {
    const double r1 = r[n + 1];
    const double lu = log(r[n + 2] / r1);
    e = exp(-(double)l * lu);
    f = (l == 2) ? r1 * r1 * lu : r1 * r1 * expm1((2.0 - l) * lu) / (2.0 - l);
  }
}

// One warp per (patch, mode): lane L owns radii L*CH .. L*CH + CH - 1, the
// affine maps of its stretch are composed across lanes by shuffles, and each
// lane then applies its incoming value along its stretch.  The inner scan
// runs upward, the outer one downward.  `cin` is the static scratch: every
// element is written by the inner pass of the lane that later reads it, so
// nothing needs clearing between calls.
__global__ void __launch_bounds__(256)
k_radial_scan_static(int n_r, int lmax, int n_lm, double G, const double *__restrict__ r,
                     const double *__restrict__ A, double *__restrict__ cin, double *__restrict__ Q) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= 2 * n_lm) return;
  const int p = warp / n_lm, idx = warp % n_lm;
  int l = (int)sqrtf((float)idx);   // corrected below; exact for idx < 2^24
  while (l * l > idx) --l;
  while ((l + 1) * (l + 1) <= idx) ++l;
  const int CH = (n_r + 31) / 32;
  const int n0 = min(n_r, lane * CH), n1 = min(n_r, n0 + CH);
  const double *Ap = A + (size_t)p * n_r * n_lm + idx;
  double *Cp = cin + (size_t)p * n_r * n_lm + idx;
  double a, b, e, f;

  double al = 1.0, be = 0.0;
  for (int n = n0; n < n1; ++n) {
    inner_factors(n, l, r, a, b);
    be = fma(a, be, b * Ap[(size_t)n * n_lm]);
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
  for (int n = n0; n < n1; ++n) {
    inner_factors(n, l, r, a, b);
    x = fma(a, x, b * Ap[(size_t)n * n_lm]);
    Cp[(size_t)n * n_lm] = x;
  }

  al = 1.0;
  be = 0.0;
  for (int n = n1 - 1; n >= n0; --n) {
    outer_factors(n, l, n_r, r, e, f);
    const double an = (n + 1 < n_r) ? Ap[(size_t)(n + 1) * n_lm] : 0.0;
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
  const double f_phi = -G * kFourPi / (2.0 * l + 1.0);
  const size_t qsz = (size_t)2 * n_r * n_lm;
  for (int n = n1 - 1; n >= n0; --n) {
    outer_factors(n, l, n_r, r, e, f);
    const double an = (n + 1 < n_r) ? Ap[(size_t)(n + 1) * n_lm] : 0.0;
    y = fma(e, y, f * an);
    const double cn = Cp[(size_t)n * n_lm];
    const double inv_r = 1.0 / r[n + 1];
    const double q = f_phi * (cn + y);
    const double qr = -f_phi * (-(l + 1.0) * cn + l * y) * inv_r;
    const double qt = -q * inv_r;
    const size_t o = (size_t)(p * n_r + n) * n_lm + idx;
    Q[o] = q;
    Q[qsz + o] = qr;
    Q[2 * qsz + o] = qt;
  }
}

// The same scan with the zone factors shared: block (l, g) takes the items
// 8 g .. 8 g + 7 of degree l (item i: patch i / (2l+1), mode l^2 + i % (2l+1)),
// and its threads first compute the four factors of every zone for degree l
// once into shared memory (n_r <= kSharedZones), where the per-warp kernel
// above recomputes them in each of its four passes.
constexpr int kSharedZones = 6144;   // 4 float64 factors per zone: 192 KiB

__global__ void __launch_bounds__(256)
k_radial_scan_static_shared(int n_r, int lmax, int n_lm, double G, const double *__restrict__ r,
                            const double *__restrict__ A, double *__restrict__ cin, double *__restrict__ Q) {
  extern __shared__ double fz[];   // [4][n_r]: a, b, e, f
  // block -> (degree l, group g): degree l has ceil(2 (2l + 1) / 8) groups
  int l = 0, g = (int)blockIdx.x;
  while (l <= lmax && g >= (4 * l + 2 + 7) / 8) {
    g -= (4 * l + 2 + 7) / 8;
    ++l;
  }
  if (l > lmax) return;
  double *fa = fz, *fb = fz + n_r, *fe = fz + 2 * n_r, *ff = fz + 3 * n_r;
  for (int n = threadIdx.x; n < n_r; n += blockDim.x) {
    inner_factors(n, l, r, fa[n], fb[n]);
    outer_factors(n, l, n_r, r, fe[n], ff[n]);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = 8 * g + warp;
  if (item >= 2 * (2 * l + 1)) return;
  const int p = item / (2 * l + 1), idx = l * l + item % (2 * l + 1);
  const int CH = (n_r + 31) / 32;
  const int n0 = min(n_r, lane * CH), n1 = min(n_r, n0 + CH);
  const double *Ap = A + (size_t)p * n_r * n_lm + idx;
  double *Cp = cin + (size_t)p * n_r * n_lm + idx;

  double al = 1.0, be = 0.0;
  for (int n = n0; n < n1; ++n) {
    be = fma(fa[n], be, fb[n] * Ap[(size_t)n * n_lm]);
    al *= fa[n];
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
  for (int n = n0; n < n1; ++n) {
    x = fma(fa[n], x, fb[n] * Ap[(size_t)n * n_lm]);
    Cp[(size_t)n * n_lm] = x;
  }

  al = 1.0;
  be = 0.0;
  for (int n = n1 - 1; n >= n0; --n) {
    const double an = (n + 1 < n_r) ? Ap[(size_t)(n + 1) * n_lm] : 0.0;
    be = fma(fe[n], be, ff[n] * an);
    al *= fe[n];
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
  const double f_phi = -G * kFourPi / (2.0 * l + 1.0);
  const size_t qsz = (size_t)2 * n_r * n_lm;
  for (int n = n1 - 1; n >= n0; --n) {
    const double an = (n + 1 < n_r) ? Ap[(size_t)(n + 1) * n_lm] : 0.0;
    y = fma(fe[n], y, ff[n] * an);
    const double cn = Cp[(size_t)n * n_lm];
    const double inv_r = 1.0 / r[n + 1];
    const double q = f_phi * (cn + y);
    const double qr = -f_phi * (-(l + 1.0) * cn + l * y) * inv_r;
    const double qt = -q * inv_r;
    const size_t o = (size_t)(p * n_r + n) * n_lm + idx;
    Q[o] = q;
    Q[qsz + o] = qr;
    Q[2 * qsz + o] = qt;
  }
}

bool aligned8(const void *p) { return ((uintptr_t)p & 7u) == 0; }

}  // namespace

extern "C" yy_status yy_radial_scan_static(const double *r_edges, int n_r, int l_max, double G,
                                           const double *moments, double *coeff, void *cuda_stream) {
  if (!r_edges || !moments || !coeff || !aligned8(r_edges) || !aligned8(moments) || !aligned8(coeff))
    return YY_ERR_INVALID_ARG;
  if (n_r < 1 || l_max < 0 || l_max > YY_LMAX_CAP || !isfinite(G)) return YY_ERR_INVALID_ARG;
  const size_t n_lm = (size_t)(l_max + 1) * (l_max + 1);
  if (2 * (size_t)n_r * n_lm > kScanScratchDoubles) return YY_ERR_INVALID_ARG;   // beyond the static scratch

  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return YY_ERR_CUDA;
  double *scratch = nullptr;
  bool shared_ok = false;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    // the calling thread's current context; none yet if this is the first
    // runtime call that touches the device (the symbol lookup below then
    // makes the device's primary context current)
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!driver_entry_points()) return YY_ERR_CUDA;
    bool have_id = g_ctx_current(&ctx) == CUDA_SUCCESS && ctx != nullptr && g_ctx_id(ctx, &id) == CUDA_SUCCESS;
    if (!have_id || g_scratch[dev].addr == nullptr || g_scratch[dev].ctx_id != id) {
      // Set-up on this device (and context): resolve the array's device
      // address.  In host code yy_scan_scratch is only a stand-in for the
      // device symbol and must never reach a kernel.
      double *p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress((void **)&p, yy_scan_scratch);
      if (e != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return YY_ERR_CUDA;
      }
      // the symbol lookup made the device's primary context current if none was
      if (!have_id)
        have_id = g_ctx_current(&ctx) == CUDA_SUCCESS && ctx != nullptr && g_ctx_id(ctx, &id) == CUDA_SUCCESS;
      if (!have_id) return YY_ERR_CUDA;
      g_scratch[dev].addr = p;
      g_scratch[dev].ctx_id = id;
      // the shared-factor kernel needs more than the default 48 KiB
      g_scratch[dev].shared_ok =
          cudaFuncSetAttribute(k_radial_scan_static_shared, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(4 * kSharedZones * sizeof(double))) == cudaSuccess;
      cudaGetLastError();
    }
    scratch = g_scratch[dev].addr;
    shared_ok = g_scratch[dev].shared_ok;
  }

  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (shared_ok && n_r <= kSharedZones) {
    int blocks = 0;
    for (int l = 0; l <= l_max; ++l) blocks += (4 * l + 2 + 7) / 8;
    k_radial_scan_static_shared<<<blocks, 256, 4 * (size_t)n_r * sizeof(double), s>>>(
        n_r, l_max, (int)n_lm, G, r_edges, moments, scratch, coeff);
  } else {
    const int warps = 2 * (int)n_lm;
    const int blocks = (warps * 32 + 255) / 256;
    k_radial_scan_static<<<blocks, 256, 0, s>>>(n_r, l_max, (int)n_lm, G, r_edges, moments, scratch, coeff);
  }
  return cudaGetLastError() == cudaSuccess ? YY_OK : YY_ERR_CUDA;
}
