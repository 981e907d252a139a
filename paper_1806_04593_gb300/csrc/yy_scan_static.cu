// Allocation-free variant of the radial scan kernel: yy_radial_scan_static.
//
// Some callers cannot allocate device memory at the point where they need the
// radial sums: code that runs while a CUDA graph is being captured (device
// allocation is not a capturable operation), applications whose device memory
// is handed out entirely by their own pool or arena, and time-critical loops
// that must not enter the driver's allocator.  This entry point needs no
// handle and allocates nothing: its only scratch (the inner-scan values kept
// between the two passes) lives in the file-scope array below, which every
// GPU that loads the library holds until the process exits.
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "yy.h"

namespace {

// Scratch capacity in float64 values: 2 * n_r * (l_max + 1)^2 must fit.
constexpr size_t kScanScratchDoubles = size_t(1) << 21;   // 16 MiB per device
constexpr int kMaxDevices = 64;
constexpr double kFourPi = 12.566370614359172953850573533118;

__device__ __align__(256) double yy_scan_scratch[kScanScratchDoubles];

// Device address of yy_scan_scratch per device, looked up once per device.
double *g_scratch_addr[kMaxDevices];
std::mutex g_setup_mutex;

// Zone factors of the scaled recurrences (same formulas as the per-grid
// table): inner c_n = a c_{n-1} + b A_n, outer d_n = e d_{n+1} + f A_{n+1}.
__device__ __forceinline__ void zone_factors(int n, int l, int n_r, const double *__restrict__ r,
                                             double &a, double &b, double &e, double &f) {
  const double r0 = r[n], r1 = r[n + 1];
  const double lq = (r0 > 0.0) ? log(r0 / r1) : -INFINITY;
  a = exp((l + 1.0) * lq);
  b = r1 * r1 * (-expm1((l + 3.0) * lq)) / (l + 3.0);
  e = 0.0;
  f = 0.0;
  if (n + 1 < n_r) {
    const double lu = log(r[n + 2] / r1);
    e = exp(-(double)l * lu);
    f = (l == 2) ? r1 * r1 * lu : r1 * r1 * expm1((2.0 - l) * lu) / (2.0 - l);
  }
}

// One warp per (patch, mode); see the per-grid scan kernel for the method.
// `cin` is the static scratch: every element is written by the inner pass of
// the lane that later reads it, so nothing needs clearing between calls.
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
    zone_factors(n, l, n_r, r, a, b, e, f);
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
    zone_factors(n, l, n_r, r, a, b, e, f);
    x = fma(a, x, b * Ap[(size_t)n * n_lm]);
    Cp[(size_t)n * n_lm] = x;
  }

  al = 1.0;
  be = 0.0;
  for (int n = n1 - 1; n >= n0; --n) {
    zone_factors(n, l, n_r, r, a, b, e, f);
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
    zone_factors(n, l, n_r, r, a, b, e, f);
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

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

extern "C" yy_status yy_radial_scan_static(const double *r_edges, int n_r, int l_max, double G,
                                           const double *moments, double *coeff, void *cuda_stream) {
  if (!r_edges || !moments || !coeff || !aligned16(r_edges) || !aligned16(moments) || !aligned16(coeff))
    return YY_ERR_INVALID_ARG;
  if (n_r < 1 || l_max < 0 || l_max > 80 || !isfinite(G)) return YY_ERR_INVALID_ARG;
  const size_t n_lm = (size_t)(l_max + 1) * (l_max + 1);
  if (2 * (size_t)n_r * n_lm > kScanScratchDoubles) return YY_ERR_INVALID_ARG;   // beyond the static scratch

  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return YY_ERR_CUDA;
  double *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_scratch_addr[dev] == nullptr) {
      // First call on this device: resolve the array's device address (the
      // host-side symbol is only a stand-in and must not reach a kernel).
      double *p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress((void **)&p, yy_scan_scratch);
      if (e != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return YY_ERR_CUDA;
      }
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
  }

  const int warps = 2 * (int)n_lm;
  const int blocks = (warps * 32 + 255) / 256;
  k_radial_scan_static<<<blocks, 256, 0, (cudaStream_t)cuda_stream>>>(n_r, l_max, (int)n_lm, G, r_edges,
                                                                       moments, scratch, coeff);
  return cudaGetLastError() == cudaSuccess ? YY_OK : YY_ERR_CUDA;
}
