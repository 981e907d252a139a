// Batched solves: many independent density fields of uneven shape (radial
// zones, angular resolution, l_max) in one CUDA graph.
//
// Each field keeps its own grid handle (tables built once).  yy_batch_potential
// records every field's solve into one graph by stream capture, the fields
// spread over kBranches parallel branches (fork / join through events) so that
// the short kernels of one field overlap the long ones of another, and then
// replays the instantiated graph on the caller's stream.  Graphs are cached
// per (precision, gradient, buffer pointers): a replay costs one launch.
// yy_batch_tune is the autotuner: for every field it times both evaluations
// (dense contractions, separable stages) on scratch buffers and records the
// faster for that precision; the capture applies it.
#include <string.h>

#include <new>
#include <vector>

#include "yy_internal.h"

namespace {

constexpr int kBranches = 4;
constexpr int kCacheSize = 4;
constexpr int kPrecisions = YY_FP16X2 + 1;

struct GraphEntry {
  int prec, grad;
  std::vector<const void *> ptrs;
  cudaGraphExec_t exec;
};

}  // namespace

struct yy_batch {
  int n;
  int device;
  std::vector<yy_grid *> grids;
  std::vector<int> method;          // [field][precision]: analysis evaluation recorded for it
  cudaStream_t cap;                 // capture origin
  cudaStream_t branch[kBranches];
  cudaEvent_t fork, join[kBranches];
  std::vector<GraphEntry> cache;
  int launches;                     // kernels in the last captured graph
};

namespace {

yy_status to_status(cudaError_t e) {
  if (e == cudaSuccess) return YY_OK;
  if (e == cudaErrorMemoryAllocation) return YY_ERR_OOM;
  return YY_ERR_CUDA;
}

void drop_cache(yy_batch *b) {
  for (GraphEntry &g : b->cache) cudaGraphExecDestroy(g.exec);
  b->cache.clear();
}

void free_batch(yy_batch *b) {
  drop_cache(b);
  for (yy_grid *g : b->grids) yy_destroy(g);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (int k = 0; k < kBranches; ++k) {
    if (b->branch[k]) cudaStreamDestroy(b->branch[k]);
    if (b->join[k]) cudaEventDestroy(b->join[k]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
}

}  // namespace

extern "C" {

yy_status yy_batch_create(const yy_field_desc *fields, int n_fields, yy_batch **out) {
  if (!out) return YY_ERR_INVALID_ARG;
  *out = nullptr;
  if (!fields || n_fields < 1 || n_fields > (1 << 16)) return YY_ERR_INVALID_ARG;
  yy_batch *b = new (std::nothrow) yy_batch();
  if (!b) return YY_ERR_OOM;
  b->n = n_fields;
  b->method.assign((size_t)n_fields * kPrecisions, (int)YY_ANALYSIS_AUTO);
  cudaGetDevice(&b->device);
  yy_status st = YY_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  for (int k = 0; k < kBranches && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&b->branch[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e != cudaSuccess) st = to_status(e);
  for (int i = 0; i < n_fields && st == YY_OK; ++i) {
    const yy_field_desc &f = fields[i];
    yy_grid *g = nullptr;
    st = yy_grid_create(f.r_edges, f.n_r, f.n_theta, f.n_phi, f.delta_theta, f.delta_phi, f.l_max, f.G, &g);
    if (st == YY_OK) b->grids.push_back(g);
  }
  if (st != YY_OK) {
    free_batch(b);
    delete b;
    return st;
  }
  *out = b;
  return YY_OK;
}

yy_status yy_batch_prepare(yy_batch *b, yy_precision prec) {
  if (!b) return YY_ERR_INVALID_ARG;
  for (yy_grid *g : b->grids) {
    const yy_status st = yy_grid_prepare(g, prec);
    if (st != YY_OK) return st;
  }
  return YY_OK;
}

yy_status yy_batch_set_analysis(yy_batch *b, int field, yy_analysis method) {
  if (!b || field < 0 || field >= b->n) return YY_ERR_INVALID_ARG;
  const yy_status st = yy_grid_set_analysis(b->grids[field], method);   // validates method
  if (st != YY_OK) return st;
  for (int p = 0; p < kPrecisions; ++p) b->method[(size_t)field * kPrecisions + p] = (int)method;
  drop_cache(b);
  return YY_OK;
}

yy_grid *yy_batch_grid(yy_batch *b, int field) {
  if (!b || field < 0 || field >= b->n) return nullptr;
  return b->grids[field];
}

yy_status yy_batch_tune(yy_batch *b, yy_precision prec, int with_gradient, int reps, int *chosen) {
  if (!b || reps < 1 || (int)prec < 0 || (int)prec >= kPrecisions) return YY_ERR_INVALID_ARG;
  yy_status st = yy_batch_prepare(b, prec);
  if (st != YY_OK) return st;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) return to_status(ce);
  const yy_analysis cands[2] = {YY_ANALYSIS_DENSE, YY_ANALYSIS_SEPARABLE};
  for (int i = 0; i < b->n && st == YY_OK; ++i) {
    yy_grid *g = b->grids[i];
    const size_t field = ((size_t)g->n_r * g->n_ang + 1) & ~(size_t)1;   // even: every part 16-byte aligned
    double *buf = nullptr;   // rho (2 fields), phi (2), gradient (6)
    ce = cudaMalloc((void **)&buf, (with_gradient ? 10 : 4) * field * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMemset(buf, 0, 2 * field * sizeof(double));
    if (ce != cudaSuccess) {
      st = to_status(ce);
      break;
    }
    double *gy = with_gradient ? buf + 4 * field : nullptr, *gg = with_gradient ? buf + 7 * field : nullptr;
    float best = 1e30f;
    int pick = 0;
    for (int c = 0; c < 2 && st == YY_OK; ++c) {
      yy_grid_set_analysis(g, cands[c]);
      st = yy_potential(g, buf, buf + field, buf + 2 * field, buf + 3 * field, gy, gg, prec, b->cap);   // warm-up
      if (st != YY_OK) break;
      cudaEventRecord(e0, b->cap);
      for (int r = 0; r < reps && st == YY_OK; ++r)
        st = yy_potential(g, buf, buf + field, buf + 2 * field, buf + 3 * field, gy, gg, prec, b->cap);
      cudaEventRecord(e1, b->cap);
      ce = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
      if (ce != cudaSuccess) st = to_status(ce);
      if (ms < best) {
        best = ms;
        pick = c;
      }
    }
    cudaFree(buf);
    yy_grid_set_analysis(g, YY_ANALYSIS_AUTO);
    b->method[(size_t)i * kPrecisions + prec] = (int)cands[pick];
    if (chosen) chosen[i] = (int)cands[pick];
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  drop_cache(b);
  return st;
}

yy_status yy_batch_potential(yy_batch *b, const double *const *rho_yin, const double *const *rho_yang,
                             double *const *phi_yin, double *const *phi_yang, double *const *grad_yin,
                             double *const *grad_yang, yy_precision prec, void *cuda_stream) {
  if (!b || !rho_yin || !rho_yang || !phi_yin || !phi_yang) return YY_ERR_INVALID_ARG;
  if ((grad_yin == nullptr) != (grad_yang == nullptr)) return YY_ERR_INVALID_ARG;
  if ((int)prec < 0 || (int)prec >= kPrecisions) return YY_ERR_INVALID_ARG;
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != b->device) return YY_ERR_INVALID_ARG;
  const int grad = grad_yin != nullptr;
  std::vector<const void *> key;
  key.reserve((size_t)b->n * 6);
  for (int i = 0; i < b->n; ++i) {
    key.push_back(rho_yin[i]);
    key.push_back(rho_yang[i]);
    key.push_back(phi_yin[i]);
    key.push_back(phi_yang[i]);
    key.push_back(grad ? grad_yin[i] : nullptr);
    key.push_back(grad ? grad_yang[i] : nullptr);
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  for (GraphEntry &ge : b->cache)
    if (ge.prec == (int)prec && ge.grad == grad && ge.ptrs == key) return to_status(cudaGraphLaunch(ge.exec, s));

  // first use of this set of buffers: capture every field's solve
  for (yy_grid *g : b->grids) {
    if (g->profiling) yy_grid_set_profiling(g, 0);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return to_status(e);
  yy_status st = YY_OK;
  if ((e = cudaEventRecord(b->fork, b->cap)) != cudaSuccess) st = to_status(e);
  for (int k = 0; k < kBranches && st == YY_OK; ++k)
    if ((e = cudaStreamWaitEvent(b->branch[k], b->fork, 0)) != cudaSuccess) st = to_status(e);
  int launches = 0;
  for (int i = 0; i < b->n && st == YY_OK; ++i) {
    yy_grid *g = b->grids[i];
    yy_grid_set_analysis(g, (yy_analysis)b->method[(size_t)i * kPrecisions + prec]);
    st = yy_potential(g, rho_yin[i], rho_yang[i], phi_yin[i], phi_yang[i], grad ? grad_yin[i] : nullptr,
                      grad ? grad_yang[i] : nullptr, prec, b->branch[i % kBranches]);
    launches += g->launches;
  }
  for (int k = 0; k < kBranches && st == YY_OK; ++k) {
    if ((e = cudaEventRecord(b->join[k], b->branch[k])) == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->join[k], 0);
    if (e != cudaSuccess) st = to_status(e);
  }
  e = cudaStreamEndCapture(b->cap, &graph);
  if (st == YY_OK && e != cudaSuccess) st = to_status(e);
  if (st != YY_OK) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return st;
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return to_status(e);
  if ((int)b->cache.size() >= kCacheSize) {
    cudaGraphExecDestroy(b->cache.front().exec);
    b->cache.erase(b->cache.begin());
  }
  b->cache.push_back(GraphEntry{(int)prec, grad, key, exec});
  b->launches = launches;
  return to_status(cudaGraphLaunch(exec, s));
}

int yy_batch_last_launch_count(const yy_batch *b) { return b ? b->launches : -1; }

yy_status yy_batch_last_device_status(yy_batch *b) {
  if (!b) return YY_ERR_INVALID_ARG;
  yy_status worst = YY_OK;
  for (yy_grid *g : b->grids) {
    const yy_status st = yy_last_device_status(g);
    if (st != YY_OK && worst == YY_OK) worst = st;
  }
  return worst;
}

void yy_batch_destroy(yy_batch *b) {
  if (!b) return;
  cudaDeviceSynchronize();
  free_batch(b);
  delete b;
}

}  // extern "C"
