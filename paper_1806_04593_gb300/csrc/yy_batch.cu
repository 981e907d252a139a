// Batched solves: many independent density fields of uneven shape (radial
// zones, angular resolution, l_max) in one CUDA graph.
//
// Each field keeps its own grid handle (tables built once).  yy_batch_potential
// records every field's solve into one graph by stream capture, the fields
// spread over parallel branches (fork / join through events) so that the
// short kernels of one field overlap the long ones of another, and then
// replays the instantiated graph on the caller's stream.  Graphs are cached
// per (precision, gradient, buffer pointers): a replay costs one launch.
//
// yy_batch_tune is the autotuner.  Per field it times both evaluations
// (dense contractions, separable stages) and, for a dense tensor-core
// analysis, the K split of the contraction (the rule's count and half of it;
// the moments are the same at every split), on scratch buffers, and records
// the fastest for that precision.
// The first capture after tuning also times the whole graph with 1, 2, 4, 8
// and 16 branches on the caller's buffers and keeps the fastest.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "yy_internal.h"

namespace {

constexpr int kBranchesMax = 16;
constexpr int kBranchesDefault = 4;
constexpr int kCacheSize = 4;
constexpr int kPrecisions = YY_FP64_OZAKI + 1;

struct GraphEntry {
  int prec, grad;
  std::vector<const void *> ptrs;
  cudaGraphExec_t exec;
  std::vector<yy::TcGroup *> groups;   // the grouped solves' argument tables (empty: per-field graph)
  int launches;
};

}  // namespace

struct yy_batch {
  int n;
  int device;
  std::vector<yy_grid *> grids;
  std::vector<int> method;          // [field][precision]: analysis evaluation recorded for it
  std::vector<int> splits;          // [field][precision]: K split of the dense analysis (0: the rule's)
  int branches;                     // parallel branches of the graph
  int tune_branches;                // time the branch counts at the next capture
  cudaStream_t cap;                 // capture origin
  cudaStream_t branch[kBranchesMax];
  cudaEvent_t fork, join[kBranchesMax];
  std::vector<GraphEntry> cache;
  int launches;                     // kernels in the last captured graph
  int grouping;                     // tensor-core forms: one launch per stage over all fields when they allow
  int n_groups;                     // concurrent groups of fields (each its own launch per stage)
  int tune_groups;                  // time 1, 2 and 4 groups at the next grouped capture
};

namespace {

yy_status to_status(cudaError_t e) {
  if (e == cudaSuccess) return YY_OK;
  if (e == cudaErrorMemoryAllocation) return YY_ERR_OOM;
  return YY_ERR_CUDA;
}

bool tensor_form(yy_precision p) { return p == YY_TF32 || p == YY_BF16X3 || p == YY_FP16X2; }

void drop_groups(std::vector<yy::TcGroup *> &groups) {
  for (yy::TcGroup *grp : groups) yy::tc_group_destroy(grp);
  groups.clear();
}

void drop_entry(GraphEntry &g) {
  cudaGraphExecDestroy(g.exec);
  drop_groups(g.groups);
}

void drop_cache(yy_batch *b) {
  for (GraphEntry &g : b->cache) drop_entry(g);
  b->cache.clear();
}

void free_batch(yy_batch *b) {
  drop_cache(b);
  for (yy_grid *g : b->grids) yy_destroy(g);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (int k = 0; k < kBranchesMax; ++k) {
    if (b->branch[k]) cudaStreamDestroy(b->branch[k]);
    if (b->join[k]) cudaEventDestroy(b->join[k]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
}

// the field's recorded evaluation and K split for this precision
yy_status apply_field_setting(yy_batch *b, int i, yy_precision prec) {
  yy_grid *g = b->grids[i];
  yy_grid_set_analysis(g, (yy_analysis)b->method[(size_t)i * kPrecisions + prec]);
  if (!tensor_form(prec)) return YY_OK;
  int rule = 0;
  if (yy::tc_analysis_splits(g, prec, &rule, nullptr) == 0) return YY_OK;   // not prepared: yy_potential reports it
  const int s = b->splits[(size_t)i * kPrecisions + prec];
  return yy::tc_set_analysis_splits(g, prec, s > 0 ? s : rule);
}

struct Buffers {
  const double *const *rho_yin, *const *rho_yang;
  double *const *phi_yin, *const *phi_yang, *const *grad_yin, *const *grad_yang;
};

// The fields in `ng` groups of about equal work (largest first, each to the
// group with the least so far; the synthesis, n_r n_ang (l_max + 1)^2, leads),
// each group's argument tables built; NOT_SUPPORTED if a field does not fit.
yy_status build_groups(yy_batch *b, const Buffers &io, yy_precision prec, int ng,
                       std::vector<yy::TcGroup *> *out) {
  std::vector<int> order(b->n);
  std::vector<double> work(b->n);
  for (int i = 0; i < b->n; ++i) {
    const yy_grid *g = b->grids[i];
    order[i] = i;
    work[i] = (double)g->n_r * g->n_ang * (double)g->n_lm;
  }
  std::sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
  std::vector<std::vector<int>> members(ng);
  std::vector<double> load(ng, 0.0);
  for (int i : order) {
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    members[k].push_back(i);
    load[k] += work[i];
  }
  const bool grad = io.grad_yin != nullptr;
  for (int k = 0; k < ng; ++k) {
    if (members[k].empty()) continue;
    std::sort(members[k].begin(), members[k].end());
    std::vector<yy_grid *> gs;
    std::vector<const double *> ry, rg;
    std::vector<double *> py, pg, gy, gg;
    for (int i : members[k]) {
      gs.push_back(b->grids[i]);
      ry.push_back(io.rho_yin[i]);
      rg.push_back(io.rho_yang[i]);
      py.push_back(io.phi_yin[i]);
      pg.push_back(io.phi_yang[i]);
      gy.push_back(grad ? io.grad_yin[i] : nullptr);
      gg.push_back(grad ? io.grad_yang[i] : nullptr);
    }
    yy::TcGroup *grp = nullptr;
    const yy_status st = yy::tc_group_create(gs.data(), (int)gs.size(), prec, ry.data(), rg.data(), py.data(),
                                             pg.data(), grad ? gy.data() : nullptr, grad ? gg.data() : nullptr, &grp);
    if (st != YY_OK) {
      drop_groups(*out);
      return st;
    }
    out->push_back(grp);
  }
  return YY_OK;
}

// record the grouped solves into a graph: each group's launches on its own
// branch, the groups running side by side
yy_status capture_groups(yy_batch *b, const std::vector<yy::TcGroup *> &groups, cudaGraphExec_t *out,
                         int *launches) {
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return to_status(e);
  cudaError_t run = cudaEventRecord(b->fork, b->cap);
  int n = 0;
  for (size_t k = 0; k < groups.size() && run == cudaSuccess; ++k) {
    run = cudaStreamWaitEvent(b->branch[k], b->fork, 0);
    if (run == cudaSuccess) run = yy::tc_group_run(groups[k], b->branch[k]);
    if (run == cudaSuccess) run = cudaEventRecord(b->join[k], b->branch[k]);
    if (run == cudaSuccess) run = cudaStreamWaitEvent(b->cap, b->join[k], 0);
    n += yy::tc_group_launches(groups[k]);
  }
  e = cudaStreamEndCapture(b->cap, &graph);
  if (run != cudaSuccess || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return to_status(run != cudaSuccess ? run : e);
  }
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  *launches = n;
  return to_status(e);
}

// record every field's solve on `branches` parallel branches into a graph
yy_status capture(yy_batch *b, const Buffers &io, yy_precision prec, int branches, cudaGraphExec_t *out,
                  int *launches) {
  const bool grad = io.grad_yin != nullptr;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return to_status(e);
  yy_status st = YY_OK;
  if ((e = cudaEventRecord(b->fork, b->cap)) != cudaSuccess) st = to_status(e);
  for (int k = 0; k < branches && st == YY_OK; ++k)
    if ((e = cudaStreamWaitEvent(b->branch[k], b->fork, 0)) != cudaSuccess) st = to_status(e);
  int n_launch = 0;
  for (int i = 0; i < b->n && st == YY_OK; ++i) {
    yy_grid *g = b->grids[i];
    st = apply_field_setting(b, i, prec);
    if (st == YY_OK)
      st = yy_potential(g, io.rho_yin[i], io.rho_yang[i], io.phi_yin[i], io.phi_yang[i],
                        grad ? io.grad_yin[i] : nullptr, grad ? io.grad_yang[i] : nullptr, prec,
                        b->branch[i % branches]);
    n_launch += g->launches;
  }
  for (int k = 0; k < branches && st == YY_OK; ++k) {
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
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return to_status(e);
  *launches = n_launch;
  return YY_OK;
}

// time one graph replay on stream s (after one untimed replay)
yy_status time_graph(cudaGraphExec_t exec, cudaStream_t s, float *ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return to_status(e);
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
  b->splits.assign((size_t)n_fields * kPrecisions, 0);
  b->branches = kBranchesDefault;
  b->grouping = 1;
  b->n_groups = 2;
  cudaGetDevice(&b->device);
  yy_status st = YY_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  for (int k = 0; k < kBranchesMax && e == cudaSuccess; ++k) {
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
    // candidates: (evaluation, K split of the dense tensor-core analysis; 0 = not applicable)
    int rule = 0, cap = 0;
    const bool tc = tensor_form(prec) && yy::tc_analysis_splits(g, prec, &rule, &cap) > 0;
    struct Cand {
      yy_analysis method;
      int splits;
    } cands[6];
    int n_cand = 0;
    cands[n_cand++] = {YY_ANALYSIS_SEPARABLE, 0};
    if (tc) {
      const int opts[2] = {rule / 2, rule};   // rule: one K segment per tile, the finest split
      for (int o : opts) {
        bool dup = o < 1 || o > cap;
        for (int q = 0; q < n_cand && !dup; ++q) dup = cands[q].splits == o;
        if (!dup) cands[n_cand++] = {YY_ANALYSIS_DENSE, o};
      }
    } else {
      cands[n_cand++] = {YY_ANALYSIS_DENSE, 0};
    }
    float best = 1e30f;
    int pick = 0;
    for (int c = 0; c < n_cand && st == YY_OK; ++c) {
      if (yy_grid_set_analysis(g, cands[c].method) != YY_OK) {   // its tables could not be built
        cudaGetLastError();
        if (c == pick) pick = c + 1;
        continue;
      }
      if (tc) st = yy::tc_set_analysis_splits(g, prec, cands[c].splits > 0 ? cands[c].splits : rule);
      if (st == YY_OK)   // warm-up
        st = yy_potential(g, buf, buf + field, buf + 2 * field, buf + 3 * field, gy, gg, prec, b->cap);
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
    if (tc) yy::tc_set_analysis_splits(g, prec, rule);
    if (cands[pick].method != YY_ANALYSIS_SEPARABLE) yy::tc_release_separable(g, prec);
    b->method[(size_t)i * kPrecisions + prec] = (int)cands[pick].method;
    b->splits[(size_t)i * kPrecisions + prec] = cands[pick].splits;
    if (chosen) chosen[i] = (int)cands[pick].method;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  drop_cache(b);
  if (st == YY_OK) b->tune_branches = b->tune_groups = 1;
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
    if (ge.prec == (int)prec && ge.grad == grad && ge.ptrs == key) {
      b->launches = ge.launches;
      return to_status(cudaGraphLaunch(ge.exec, s));
    }

  // first use of this set of buffers: capture every field's solve.  Tables a
  // field's evaluation needs are built here, before the capture begins.
  for (int i = 0; i < b->n; ++i) {
    yy_grid *g = b->grids[i];
    if (g->profiling) yy_grid_set_profiling(g, 0);
    const yy_status st = yy_grid_set_analysis(g, (yy_analysis)b->method[(size_t)i * kPrecisions + prec]);
    if (st != YY_OK) return st;
  }
  const Buffers io = {rho_yin, rho_yang, phi_yin, phi_yang, grad_yin, grad_yang};
  cudaGraphExec_t exec = nullptr;
  std::vector<yy::TcGroup *> groups;
  int launches = 0;
  yy_status st = YY_OK;
  bool timing = false;   // after tuning: time the grouped and the per-field graphs
  float best_grouped = 1e30f;
  if (b->grouping && tensor_form(prec)) {
    timing = b->tune_groups != 0;
    // every field dense: one launch per stage over the fields of a group,
    // the groups side by side (their number timed once after tuning)
    bool dense = true;
    for (int i = 0; i < b->n && dense; ++i) dense = b->method[(size_t)i * kPrecisions + prec] != YY_ANALYSIS_SEPARABLE;
    for (int i = 0; i < b->n && dense && st == YY_OK; ++i) st = apply_field_setting(b, i, prec);
    if (st != YY_OK) return st;
    const int trials[3] = {1, 2, 4};
    float best = 1e30f;
    for (int q = 0; q < 3 && dense; ++q) {
      const int ng = b->tune_groups ? trials[q] : b->n_groups;
      if (!b->tune_groups && q > 0) break;
      if (ng > b->n || ng > kBranchesMax) continue;
      std::vector<yy::TcGroup *> trial_groups;
      st = build_groups(b, io, prec, ng, &trial_groups);
      if (st == YY_ERR_NOT_SUPPORTED) {   // a field does not fit: per-field graphs
        st = YY_OK;
        break;
      }
      if (st != YY_OK) break;
      cudaGraphExec_t trial = nullptr;
      int n_launch = 0;
      float ms = 0.0f;
      st = capture_groups(b, trial_groups, &trial, &n_launch);
      if (st == YY_OK && b->tune_groups) st = time_graph(trial, s, &ms);
      if (st == YY_OK && ms < best) {
        best = ms;
        if (exec) cudaGraphExecDestroy(exec);
        drop_groups(groups);
        exec = trial;
        groups = trial_groups;
        launches = n_launch;
        b->n_groups = ng;
      } else {
        if (trial) cudaGraphExecDestroy(trial);
        drop_groups(trial_groups);
      }
      if (st != YY_OK) break;
    }
    if (st != YY_OK) {
      if (exec) cudaGraphExecDestroy(exec);
      drop_groups(groups);
      return st;
    }
    best_grouped = best;
  }
  if (!exec || timing) {
    // the per-field graph: when nothing was grouped, or to compare with the grouped one
    cudaGraphExec_t fexec = nullptr;
    int flaunch = 0;
    float fbest = 1e30f;
    if (b->tune_branches) {
      // time the graph with each branch count on these buffers (every trial
      // leaves the same results in them) and keep the fastest
      for (int nb = 1; nb <= kBranchesMax && st == YY_OK; nb *= 2) {
        cudaGraphExec_t trial = nullptr;
        int n_launch = 0;
        float ms = 0.0f;
        st = capture(b, io, prec, nb, &trial, &n_launch);
        if (st == YY_OK) st = time_graph(trial, s, &ms);
        if (st == YY_OK && ms < fbest) {
          fbest = ms;
          if (fexec) cudaGraphExecDestroy(fexec);
          fexec = trial;
          flaunch = n_launch;
          b->branches = nb;
        } else if (trial) {
          cudaGraphExecDestroy(trial);
        }
      }
      if (st == YY_OK) b->tune_branches = 0;
    } else {
      st = capture(b, io, prec, b->branches, &fexec, &flaunch);
      if (st == YY_OK && exec) st = time_graph(fexec, s, &fbest);
    }
    if (st != YY_OK) {
      if (fexec) cudaGraphExecDestroy(fexec);
      if (exec) cudaGraphExecDestroy(exec);
      drop_groups(groups);
      return st;
    }
    if (!exec || fbest < best_grouped) {
      // the per-field graph it is (the tuner keeps to it for this batch)
      if (exec) {
        cudaGraphExecDestroy(exec);
        drop_groups(groups);
        b->grouping = 0;
      }
      exec = fexec;
      launches = flaunch;
    } else {
      cudaGraphExecDestroy(fexec);
    }
  }
  if (timing) b->tune_groups = 0;
  if ((int)b->cache.size() >= kCacheSize) {
    drop_entry(b->cache.front());
    b->cache.erase(b->cache.begin());
  }
  b->cache.push_back(GraphEntry{(int)prec, grad, key, exec, groups, launches});
  b->launches = launches;
  return to_status(cudaGraphLaunch(exec, s));
}

int yy_batch_last_launch_count(const yy_batch *b) { return b ? b->launches : -1; }

yy_status yy_batch_set_grouping(yy_batch *b, int groups) {
  if (!b || groups < 0 || groups > kBranchesMax) return YY_ERR_INVALID_ARG;
  drop_cache(b);   // later calls record their graphs anew
  b->grouping = groups > 0;
  if (groups > 0) {
    b->n_groups = groups;
    b->tune_groups = 0;
  }
  return YY_OK;
}

int yy_batch_branches(const yy_batch *b) { return b ? b->branches : -1; }

int yy_batch_groups(const yy_batch *b) { return b ? (b->grouping ? b->n_groups : 0) : -1; }

int yy_batch_analysis_splits(const yy_batch *b, int field, yy_precision prec) {
  if (!b || field < 0 || field >= b->n || (int)prec < 0 || (int)prec >= kPrecisions) return -1;
  return b->splits[(size_t)field * kPrecisions + prec];
}

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
