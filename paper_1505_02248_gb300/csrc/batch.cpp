// Batched advance of independent problems under one CUDA graph (lem_batch_*, include/lem.h).
//
// An autotuner captures and times candidate schedules on scratch copies of the states, and
// the fastest one is kept (lem_batch_candidates lists them with their times):
//  * lanes, for several lane counts: every context's own step launches, spread over
//    concurrent lanes (graph branches) by longest-processing-time-first from each problem's
//    measured step time;
//  * fused (all contexts on the same tensor-core split tier), for several window-block
//    widths: one residual launch and one persistent GEMM launch per LEM step for all problems
//    together. Width cap 0 keeps every context's own block of 128 (or 256) windows; a cap c
//    gives each problem the power of two in [16, c] whose blocks load the fewest operand
//    bytes, so small tile grids take narrow MMAs instead of mostly empty blocks.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "lem_internal.h"

struct lem_batch {
  int n = 0, steps = 0, nlanes = 0, device = 0;
  int fused = 0;              // the graph runs the fused schedule
  int fused_cap = 0;          // its window-block width cap
  double lanes_ms = -1.0;     // measured time of one launch of the best candidate of each kind
  double fused_ms = -1.0;     // (-1: none built)
  std::vector<lem_batch_candidate> cands;
  cudaStream_t stream = nullptr;
  std::vector<cudaStream_t> lane_streams;
  std::vector<lem_ctx*> ctxs;
  std::vector<double> est_ms;
  std::vector<int> lane;
  std::vector<std::vector<int>> lane_items;
  lem::SplitBatch* sb = nullptr;  // fused tables the graph reads
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

using lem::fail;

void free_batch(lem_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaStream_t s : b->lane_streams)
    if (s) cudaStreamDestroy(s);
  lem::split_batch_destroy(b->sb);
  delete b;
}

// LEM_OK, or LEM_ECUDA with the call's error as the message.
lem_status cuda_status(cudaError_t e, const char* what) { return e == cudaSuccess ? LEM_OK : lem::cuda_fail(e, what); }

// Capture one launch of a schedule into an executable graph. lanes: each lane's problems in
// sequence on the lane's stream, the lanes in parallel; fused: the multi-problem steps.
lem_status capture(lem_batch* b, double* const* states, lem::SplitBatch* sb, cudaGraph_t* g_out,
                   cudaGraphExec_t* e_out) {
  *g_out = nullptr;
  *e_out = nullptr;
  cudaStream_t cap = nullptr;
  LEM_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  std::vector<cudaEvent_t> ev(b->nlanes + 1, nullptr);
  lem_status st = LEM_OK;
  for (auto& e : ev)
    if (st == LEM_OK) st = cuda_status(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "capture event");
  if (st == LEM_OK) st = cuda_status(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
  if (st == LEM_OK) {
    if (sb) {
      st = lem::split_batch_step(sb, b->steps, cap);
    } else {
      cudaEventRecord(ev[b->nlanes], cap);
      for (int l = 0; l < b->nlanes && st == LEM_OK; ++l) {
        cudaStreamWaitEvent(b->lane_streams[l], ev[b->nlanes], 0);
        for (int i : b->lane_items[l]) {
          lem_ctx* c = b->ctxs[i];
          cudaStream_t keep = c->stream;
          c->stream = b->lane_streams[l];
          st = lem_step(c, states[i], b->steps);
          c->stream = keep;
          if (st != LEM_OK) break;
        }
        cudaEventRecord(ev[l], b->lane_streams[l]);
        cudaStreamWaitEvent(cap, ev[l], 0);
      }
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cap, &g);
    if (st == LEM_OK && e != cudaSuccess) st = lem::cuda_fail(e, "cudaStreamEndCapture");
    if (st == LEM_OK) {
      const cudaError_t e2 = cudaGraphInstantiate(e_out, g, 0);
      if (e2 != cudaSuccess) st = lem::cuda_fail(e2, "cudaGraphInstantiate");
    }
    if (st == LEM_OK) *g_out = g;
    else if (g) cudaGraphDestroy(g);
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  cudaStreamDestroy(cap);
  cudaGetLastError();
  return st;
}

// Lanes for nl lanes: longest problems first, each to the lane with the least work so far.
void assign_lanes(lem_batch* b, int nl) {
  const int n = b->n;
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->est_ms[a] > b->est_ms[c]; });
  std::vector<double> load(nl, 0.0);
  b->nlanes = nl;
  b->lane_items.assign(nl, {});
  b->lane.assign(n, 0);
  for (int i : order) {
    const int l = int(std::min_element(load.begin(), load.end()) - load.begin());
    load[l] += b->est_ms[i];
    b->lane_items[l].push_back(i);
    b->lane[i] = l;
  }
}

// One warm launch, then the best of three timed launches.
lem_status time_graph(cudaGraphExec_t exec, cudaStream_t s, double* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  LEM_CUDA_TRY(cudaEventCreate(&e0));
  LEM_CUDA_TRY(cudaEventCreate(&e1));
  lem_status st = LEM_OK;
  if (cudaGraphLaunch(exec, s) != cudaSuccess) st = lem::cuda_fail(cudaGetLastError(), "timing a batch graph");
  float best = -1.0f;
  for (int r = 0; r < 3 && st == LEM_OK; ++r) {
    if (cudaEventRecord(e0, s) != cudaSuccess || cudaGraphLaunch(exec, s) != cudaSuccess ||
        cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      st = lem::cuda_fail(cudaGetLastError(), "timing a batch graph");
      break;
    }
    float f = 0.0f;
    cudaEventElapsedTime(&f, e0, e1);
    if (best < 0.0f || f < best) best = f;
  }
  *ms = best;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

}  // namespace

extern "C" {

lem_status lem_batch_create(lem_ctx* const* ctxs, double* const* d_states, int n, int steps_per_launch, int lanes,
                            void* cuda_stream, lem_batch** out) {
  if (!out) return fail(LEM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ctxs || !d_states || n <= 0 || steps_per_launch <= 0 || lanes <= 0)
    return fail(LEM_EINVAL, "bad batch arguments");
  const int dev = ctxs[0] ? ctxs[0]->device : -1;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i] || !d_states[i]) return fail(LEM_EINVAL, "NULL context or state");
    if (ctxs[i]->device != dev) return fail(LEM_EINVAL, "contexts on different devices");
    if (ctxs[i]->desc.reaction && ctxs[i]->desc.refresh > 0)
      return fail(LEM_EINVAL, "Jacobian refreshes rebuild propagators and cannot be captured");
    if (ctxs[i]->cplx) return fail(LEM_EINVAL, "batches take real problems (step complex contexts with lem_step)");
    if (ctxs[i]->desc.reaction == 2)
      return fail(LEM_EINVAL, "batches do not take the porous-medium problem (step it with lem_step)");
  }
  lem::DeviceGuard guard(dev);
  lem_batch* b = new lem_batch();
  b->n = n;
  b->steps = steps_per_launch;
  b->device = dev;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->nlanes = std::min(lanes, n);
  b->ctxs.assign(ctxs, ctxs + n);
  lem_status st = LEM_OK;
  // scratch copies of every state: warm-up, per-problem timing and the candidate schedules
  // run on them, so the caller's states are untouched until the first lem_batch_run
  std::vector<double*> tmp(n, nullptr);
  for (int i = 0; i < n && st == LEM_OK; ++i) {
    if (cudaMalloc(&tmp[i], sizeof(double) * ctxs[i]->npts) != cudaSuccess) {
      cudaGetLastError();
      st = fail(LEM_ENOMEM, "batch scratch states");
      break;
    }
    const cudaError_t e = cudaMemcpyAsync(tmp[i], d_states[i], sizeof(double) * ctxs[i]->npts,
                                          cudaMemcpyDeviceToDevice, ctxs[i]->stream);
    if (e != cudaSuccess) st = lem::cuda_fail(e, "batch scratch copy");
  }
  // warm up (builds, lazy buffers, packed propagators) and time each problem
  b->est_ms.assign(n, 0.0);
  if (st == LEM_OK) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int i = 0; i < n && st == LEM_OK; ++i) {
      lem_ctx* c = ctxs[i];
      st = lem_step(c, tmp[i], steps_per_launch);
      if (st == LEM_OK) {
        cudaEventRecord(e0, c->stream);
        st = lem_step(c, tmp[i], steps_per_launch);
        cudaEventRecord(e1, c->stream);
      }
      if (st == LEM_OK && cudaEventSynchronize(e1) == cudaSuccess) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        b->est_ms[i] = ms;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == LEM_OK && cudaDeviceSynchronize() != cudaSuccess) st = lem::cuda_fail(cudaGetLastError(), "warm-up");
  }
  // candidate lane counts (lanes/2, lanes, 2 lanes, within 1..n) and their streams
  std::vector<int> lane_counts;
  for (int nl : {lanes / 2, lanes, 2 * lanes}) {
    nl = std::max(1, std::min(nl, n));
    if (std::find(lane_counts.begin(), lane_counts.end(), nl) == lane_counts.end()) lane_counts.push_back(nl);
  }
  if (st == LEM_OK) {
    b->lane_streams.assign(*std::max_element(lane_counts.begin(), lane_counts.end()), nullptr);
    for (auto& s2 : b->lane_streams) {
      if (st != LEM_OK) break;
      const cudaError_t e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
      if (e != cudaSuccess) st = lem::cuda_fail(e, "lane stream");
    }
  }
  // time every candidate on the scratch states
  for (int nl : lane_counts) {
    if (st != LEM_OK) break;
    assign_lanes(b, nl);
    cudaGraph_t g = nullptr;
    cudaGraphExec_t e = nullptr;
    double ms = -1.0;
    st = capture(b, tmp.data(), nullptr, &g, &e);
    if (st == LEM_OK) st = time_graph(e, b->stream, &ms);
    if (e) cudaGraphExecDestroy(e);
    if (g) cudaGraphDestroy(g);
    if (st == LEM_OK) b->cands.push_back(lem_batch_candidate{0, nl, 0, ms, 0});
  }
  const bool can_fuse = lem::split_batch_eligible(const_cast<lem_ctx* const*>(ctxs), n);
  if (can_fuse) {
    for (int cap : {0, 128, 64, 32}) {
      if (st != LEM_OK) break;
      lem::SplitBatch* sb = nullptr;
      st = lem::split_batch_prepare(const_cast<lem_ctx* const*>(ctxs), tmp.data(), n, cap, &sb);
      cudaGraph_t g = nullptr;
      cudaGraphExec_t e = nullptr;
      double ms = -1.0;
      if (st == LEM_OK) st = capture(b, tmp.data(), sb, &g, &e);
      if (st == LEM_OK) st = time_graph(e, b->stream, &ms);
      if (st == LEM_OK) st = lem::split_batch_check_error(sb);
      if (e) cudaGraphExecDestroy(e);
      if (g) cudaGraphDestroy(g);
      lem::split_batch_destroy(sb);
      if (st == LEM_OK) b->cands.push_back(lem_batch_candidate{1, 0, cap, ms, 0});
    }
  }
  for (double* p : tmp)
    if (p) cudaFree(p);
  // the fastest candidate (LEM_BATCH_SCHEDULE=lanes|fused restricts the choice to one kind,
  // fused:<cap> to one width cap; a fused request on contexts that cannot be fused keeps lanes)
  if (st == LEM_OK) {
    int want = -1, want_cap = -1;
    if (const char* f = std::getenv("LEM_BATCH_SCHEDULE")) {
      if (std::strcmp(f, "lanes") == 0) want = 0;
      if (std::strncmp(f, "fused", 5) == 0 && can_fuse) {
        want = 1;
        if (f[5] == ':') want_cap = std::atoi(f + 6);
      }
    }
    int best = -1;
    for (int k = 0; k < int(b->cands.size()); ++k) {
      const lem_batch_candidate& c = b->cands[k];
      double& kind_best = c.fused ? b->fused_ms : b->lanes_ms;
      if (kind_best < 0.0 || c.ms < kind_best) kind_best = c.ms;
      if (want >= 0 && c.fused != want) continue;
      if (want_cap >= 0 && c.n_cap != want_cap) continue;
      if (best < 0 || c.ms < b->cands[best].ms) best = k;
    }
    if (best < 0) st = fail(LEM_ECUDA, "no batch schedule could be timed");
    if (st == LEM_OK) {
      b->cands[best].chosen = 1;
      const lem_batch_candidate& c = b->cands[best];
      b->fused = c.fused;
      b->fused_cap = c.n_cap;
      if (b->fused) {
        st = lem::split_batch_prepare(const_cast<lem_ctx* const*>(ctxs), const_cast<double* const*>(d_states), n,
                                      c.n_cap, &b->sb);
      } else {
        assign_lanes(b, c.lanes);
      }
      if (st == LEM_OK) st = capture(b, const_cast<double* const*>(d_states), b->sb, &b->graph, &b->exec);
    }
  }
  if (st != LEM_OK) {
    free_batch(b);
    return st;
  }
  *out = b;
  return LEM_OK;
}

lem_status lem_batch_run(lem_batch* b, int launches) {
  if (!b || launches < 0) return fail(LEM_EINVAL, "bad batch run arguments");
  lem::DeviceGuard guard(b->device);
  for (int k = 0; k < launches; ++k) {
    const cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess) return lem::cuda_fail(e, "cudaGraphLaunch");
  }
  return LEM_OK;
}

lem_status lem_batch_sync(lem_batch* b) {
  if (!b) return fail(LEM_EINVAL, "batch is NULL");
  lem::DeviceGuard guard(b->device);
  LEM_CUDA_TRY(cudaStreamSynchronize(b->stream));
  if (b->sb) return lem::split_batch_check_error(b->sb);
  for (lem_ctx* c : b->ctxs) LEM_TRY(lem::split_check_error(c));
  return LEM_OK;
}

lem_status lem_batch_schedule(const lem_batch* b, double* est_ms, int* lane) {
  if (!b) return fail(LEM_EINVAL, "batch is NULL");
  for (int i = 0; i < b->n; ++i) {
    if (est_ms) est_ms[i] = b->est_ms[i];
    if (lane) lane[i] = b->lane[i];
  }
  return LEM_OK;
}

lem_status lem_batch_info(const lem_batch* b, int* fused, double* lanes_ms, double* fused_ms) {
  if (!b) return fail(LEM_EINVAL, "batch is NULL");
  if (fused) *fused = b->fused;
  if (lanes_ms) *lanes_ms = b->lanes_ms;
  if (fused_ms) *fused_ms = b->fused_ms;
  return LEM_OK;
}

lem_status lem_batch_candidates(const lem_batch* b, int max, lem_batch_candidate* out, int* count) {
  if (!b || !count || (max > 0 && !out)) return fail(LEM_EINVAL, "bad batch candidates arguments");
  *count = int(b->cands.size());
  for (int k = 0; k < max && k < int(b->cands.size()); ++k) out[k] = b->cands[k];
  return LEM_OK;
}

lem_status lem_batch_gemm_work(const lem_batch* b, double* algorithmic_flops, double* executed_flops) {
  if (!b || !algorithmic_flops || !executed_flops) return fail(LEM_EINVAL, "NULL argument");
  if (!b->fused) return fail(LEM_EINVAL, "the batch runs the lanes schedule (no fused GEMM)");
  *algorithmic_flops = lem::split_batch_gemm_flops(b->sb, b->ctxs.data());
  *executed_flops = lem::split_batch_executed_flops(b->sb);
  return LEM_OK;
}

lem_status lem_batch_profile(lem_batch* b, int nsteps, double* gemm_ms, double* residual_ms, double* other_ms,
                             double* gemm_flops) {
  if (!b || nsteps <= 0 || !gemm_ms || !residual_ms || !other_ms || !gemm_flops)
    return fail(LEM_EINVAL, "bad batch profile arguments");
  lem::DeviceGuard guard(b->device);
  *gemm_ms = *residual_ms = *other_ms = *gemm_flops = 0.0;
  if (!b->fused) return fail(LEM_EINVAL, "the batch runs the lanes schedule; time its contexts with lem_set_timing");
  std::vector<cudaEvent_t> ev(2 * nsteps + 4, nullptr);
  lem_status st = LEM_OK;
  for (auto& e : ev)
    if (st == LEM_OK) st = cuda_status(cudaEventCreate(&e), "profile event");
  if (st == LEM_OK) st = cuda_status(cudaEventRecord(ev[2 * nsteps + 2], b->stream), "cudaEventRecord");
  if (st == LEM_OK) st = lem::split_batch_step(b->sb, nsteps, b->stream, ev.data());
  if (st == LEM_OK) st = cuda_status(cudaEventRecord(ev[2 * nsteps + 3], b->stream), "cudaEventRecord");
  if (st == LEM_OK) st = cuda_status(cudaEventSynchronize(ev[2 * nsteps + 3]), "cudaEventSynchronize");
  if (st == LEM_OK) {
    float t = 0.0f, total = 0.0f;
    cudaEventElapsedTime(&total, ev[2 * nsteps + 2], ev[2 * nsteps + 3]);
    for (int k = 0; k < nsteps; ++k) {
      cudaEventElapsedTime(&t, ev[1 + 2 * k], ev[2 + 2 * k]);
      *gemm_ms += t;
      cudaEventElapsedTime(&t, k == 0 ? ev[0] : ev[2 * k], ev[1 + 2 * k]);
      *residual_ms += t;
    }
    *other_ms = total - *gemm_ms - *residual_ms;
    *gemm_flops = lem::split_batch_gemm_flops(b->sb, b->ctxs.data()) * nsteps;
    st = lem::split_batch_check_error(b->sb);
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  return st;
}

void lem_batch_destroy(lem_batch* b) {
  if (!b) return;
  lem::DeviceGuard guard(b->device);
  cudaStreamSynchronize(b->stream);
  free_batch(b);
}

}  // extern "C"
