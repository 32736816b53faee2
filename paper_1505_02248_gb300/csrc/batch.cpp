// Batched advance of independent problems under one CUDA graph (lem_batch_*, include/lem.h).
#include <algorithm>
#include <numeric>
#include <vector>

#include "lem_internal.h"

struct lem_batch {
  int n = 0, steps = 0, nlanes = 0, device = 0;
  cudaStream_t stream = nullptr;
  std::vector<cudaStream_t> lane_streams;
  std::vector<double> est_ms;
  std::vector<int> lane;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

void free_batch(lem_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaStream_t s : b->lane_streams) cudaStreamDestroy(s);
  delete b;
}

}  // namespace

extern "C" {

lem_status lem_batch_create(lem_ctx* const* ctxs, double* const* d_states, int n, int steps_per_launch, int lanes,
                            void* cuda_stream, lem_batch** out) {
  if (!out) return lem::fail(LEM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ctxs || !d_states || n <= 0 || steps_per_launch <= 0 || lanes <= 0)
    return lem::fail(LEM_EINVAL, "bad batch arguments");
  const int dev = ctxs[0] ? ctxs[0]->device : -1;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i] || !d_states[i]) return lem::fail(LEM_EINVAL, "NULL context or state");
    if (ctxs[i]->device != dev) return lem::fail(LEM_EINVAL, "contexts on different devices");
    if (ctxs[i]->desc.reaction && ctxs[i]->desc.refresh > 0)
      return lem::fail(LEM_EINVAL, "Jacobian refreshes rebuild propagators and cannot be captured");
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != dev) cudaSetDevice(dev);
  lem_batch* b = new lem_batch();
  b->n = n;
  b->steps = steps_per_launch;
  b->device = dev;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->nlanes = std::min(lanes, n);
  lem_status st = LEM_OK;
  // warm up every context on a copy of its state (builds, lazy buffers, packed propagators)
  // and measure one launch worth of steps
  b->est_ms.assign(n, 0.0);
  {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int i = 0; i < n && st == LEM_OK; ++i) {
      lem_ctx* c = ctxs[i];
      double* tmp = nullptr;
      if (cudaMalloc(&tmp, sizeof(double) * c->npts) != cudaSuccess) { cudaGetLastError(); st = LEM_ENOMEM; break; }
      cudaMemcpyAsync(tmp, d_states[i], sizeof(double) * c->npts, cudaMemcpyDeviceToDevice, c->stream);
      st = lem_step(c, tmp, steps_per_launch);  // first call: builds and allocates
      if (st == LEM_OK) {
        cudaEventRecord(e0, c->stream);
        st = lem_step(c, tmp, steps_per_launch);
        cudaEventRecord(e1, c->stream);
      }
      if (st == LEM_OK && cudaEventSynchronize(e1) == cudaSuccess) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        b->est_ms[i] = ms;
      }
      cudaStreamSynchronize(c->stream);
      cudaFree(tmp);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  if (st != LEM_OK) { free_batch(b); if (prev >= 0) cudaSetDevice(prev); return st; }
  // schedule: longest problems first, each to the lane with the least work so far
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->est_ms[a] > b->est_ms[c]; });
  std::vector<double> load(b->nlanes, 0.0);
  std::vector<std::vector<int>> lane_items(b->nlanes);
  b->lane.assign(n, 0);
  for (int i : order) {
    const int l = int(std::min_element(load.begin(), load.end()) - load.begin());
    load[l] += b->est_ms[i];
    lane_items[l].push_back(i);
    b->lane[i] = l;
  }
  b->lane_streams.resize(b->nlanes, nullptr);
  for (auto& s : b->lane_streams)
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) { cudaGetLastError(); st = LEM_ECUDA; }
  // capture: fork from the batch stream into the lanes, each lane's problems in sequence,
  // join back. Each context is redirected to its lane's stream for the capture.
  cudaStream_t cap = nullptr;
  if (st == LEM_OK && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) st = LEM_ECUDA;
  std::vector<cudaEvent_t> ev(b->nlanes + 1, nullptr);
  for (auto& e : ev)
    if (st == LEM_OK && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) st = LEM_ECUDA;
  if (st == LEM_OK && cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = LEM_ECUDA;
  if (st == LEM_OK) {
    cudaEventRecord(ev[b->nlanes], cap);
    for (int l = 0; l < b->nlanes && st == LEM_OK; ++l) {
      cudaStreamWaitEvent(b->lane_streams[l], ev[b->nlanes], 0);
      for (int i : lane_items[l]) {
        lem_ctx* c = ctxs[i];
        cudaStream_t keep = c->stream;
        c->stream = b->lane_streams[l];
        st = lem_step(c, d_states[i], steps_per_launch);
        c->stream = keep;
        if (st != LEM_OK) break;
      }
      cudaEventRecord(ev[l], b->lane_streams[l]);
      cudaStreamWaitEvent(cap, ev[l], 0);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cap, &g);
    if (st == LEM_OK && e != cudaSuccess) st = lem::cuda_fail(e, "cudaStreamEndCapture");
    b->graph = g;
    if (st == LEM_OK) {
      const cudaError_t e2 = cudaGraphInstantiate(&b->exec, b->graph, 0);
      if (e2 != cudaSuccess) st = lem::cuda_fail(e2, "cudaGraphInstantiate");
    }
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  if (cap) cudaStreamDestroy(cap);
  cudaGetLastError();
  if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  if (st != LEM_OK) { free_batch(b); return st; }
  *out = b;
  return LEM_OK;
}

lem_status lem_batch_run(lem_batch* b, int launches) {
  if (!b || launches < 0) return lem::fail(LEM_EINVAL, "bad batch run arguments");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != b->device) cudaSetDevice(b->device);
  lem_status st = LEM_OK;
  for (int k = 0; k < launches && st == LEM_OK; ++k) {
    const cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess) st = lem::cuda_fail(e, "cudaGraphLaunch");
  }
  if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
  return st;
}

lem_status lem_batch_schedule(const lem_batch* b, double* est_ms, int* lane) {
  if (!b) return lem::fail(LEM_EINVAL, "batch is NULL");
  for (int i = 0; i < b->n; ++i) {
    if (est_ms) est_ms[i] = b->est_ms[i];
    if (lane) lane[i] = b->lane[i];
  }
  return LEM_OK;
}

void lem_batch_destroy(lem_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  free_batch(b);
}

}  // extern "C"
