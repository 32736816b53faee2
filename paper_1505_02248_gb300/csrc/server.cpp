// Serving layer: continuous batching of independent LEM requests on one device
// (lem_server_create / lem_submit / lem_poll / lem_wait / lem_server_get_stats /
// lem_server_destroy, declared in include/lem.h).
//
// One worker thread owns the device work. Each iteration it admits queued requests in
// arrival order while their device memory fits the budget, then gives every admitted
// request that is not waiting on the GPU its next chunk of LEM steps (a lem_step call on the
// stream of the request's context) and checks finished chunks with events. A request whose
// steps are done gets its state copied back and completes. New requests therefore join the
// running set between chunks, and requests on different contexts run on different streams,
// so their kernels overlap on the device.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "lem_internal.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kChunk = 4;                       // LEM steps per scheduling quantum
constexpr size_t kDefaultBudget = size_t(80) << 30;

enum class RS { Queued, Running, CopyBack, Done, Failed };

struct CachedCtx {
  lem_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  int users = 0;
  int64_t bytes = 0;
  uint64_t last_use = 0;
};

struct Request {
  uint64_t id = 0;
  lem_problem_desc desc{};
  std::vector<double> coef[5];
  std::string key;
  double tol = 0.0;
  double* h_state = nullptr;
  int64_t npts = 0;
  int nsteps = 0, remaining = 0, pending = 0;
  RS state = RS::Queued;
  lem_status status = LEM_OK;
  double* d_state = nullptr;
  CachedCtx* cc = nullptr;
  cudaEvent_t ev = nullptr;
  bool in_flight = false;
  bool accounted = false;  // the state's bytes count against the budget
  Clock::time_point t_submit, t_done;
};

uint64_t fnv1a(const void* p, size_t n, uint64_t h = 1469598103934665603ull) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}

// Problem identity for the propagator cache (everything but the state).
std::string make_key(const lem_problem_desc& d, const std::vector<double>* coef) {
  uint64_t h = 1469598103934665603ull;
  h = fnv1a(&d.ndim, sizeof d.ndim, h);
  h = fnv1a(d.n, sizeof d.n, h);
  h = fnv1a(d.bc, sizeof d.bc, h);
  h = fnv1a(&d.coef_stride, sizeof d.coef_stride, h);
  h = fnv1a(&d.reaction, sizeof d.reaction, h);
  h = fnv1a(&d.dt, sizeof d.dt, h);
  h = fnv1a(d.tile, sizeof d.tile, h);
  h = fnv1a(d.overlap, sizeof d.overlap, h);
  h = fnv1a(&d.mode, sizeof d.mode, h);
  h = fnv1a(&d.refresh, sizeof d.refresh, h);
  for (int k = 0; k < 5; ++k)
    if (!coef[k].empty()) h = fnv1a(coef[k].data(), coef[k].size() * sizeof(double), h);
  return std::to_string(h);
}

}  // namespace

struct lem_server {
  int device = 0;
  int64_t budget = 0;
  std::mutex mu;
  std::map<uint64_t, std::shared_ptr<Request>> all;
  std::deque<std::shared_ptr<Request>> queue;
  std::vector<std::shared_ptr<Request>> active;  // worker-owned
  std::map<std::string, std::unique_ptr<CachedCtx>> cache;
  int64_t used = 0;
  uint64_t next_id = 1, tick = 0;
  std::atomic<bool> stop{false};
  std::thread worker;
  // statistics
  int64_t submitted = 0, admitted = 0, completed = 0, failed = 0, dof_steps = 0;
  int64_t ctx_hits = 0, ctx_misses = 0;
  std::vector<double> lat_ms;
  bool any_admitted = false;
  Clock::time_point t_first_admit, t_last_done;
};

namespace {

void finish(lem_server* s, const std::shared_ptr<Request>& r, lem_status st) {
  if (r->ev) { cudaEventDestroy(r->ev); r->ev = nullptr; }
  if (r->d_state) {
    cudaFree(r->d_state);
    r->d_state = nullptr;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (r->accounted) {
    s->used -= int64_t(sizeof(double)) * r->npts;
    r->accounted = false;
  }
  if (r->cc) {
    r->cc->users--;
    r->cc->last_use = ++s->tick;
    r->cc = nullptr;
  }
  r->t_done = Clock::now();
  r->status = st;
  if (st == LEM_OK) {
    r->state = RS::Done;
    s->completed++;
    s->dof_steps += r->npts * r->nsteps;
    s->lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
    s->t_last_done = r->t_done;
  } else {
    r->state = RS::Failed;
    s->failed++;
  }
}

int64_t ctx_bytes_estimate(const lem_problem_desc& d) {
  int64_t nt = 0, nc = 0, nl = 0, ni = 0;
  if (lem_plan_query(&d, &nt, &nc, &nl, &ni, nullptr) != LEM_OK) return -1;
  const int64_t npts = d.ndim == 1 ? d.n[0] : d.n[0] * d.n[1];
  int64_t b = 8 * (nc * ni * nl + 2 * npts + nt * (nl + ni)) + 5 * 8 * (d.coef_stride ? npts : 1);
  if (d.prec == LEM_PREC_SPLIT) b += 4 * 2 * npts + 3 * 2 * (npts + 8 * int64_t(std::sqrt(double(npts))) * 64) +
                                     3 * 2 * ni * nl * 2;
  // transient builder scratch (freed after the build): 19 n_loc^2 doubles per class batch
  const int64_t per = 19 * nl * nl * 8;
  const int64_t batch = std::max<int64_t>(1, std::min<int64_t>(nc, (int64_t(8) << 30) / std::max<int64_t>(per, 1)));
  return b + per * batch;
}

// Admit r if its state (and a new context, when it needs one) fits the budget. Returns
// false if r must keep waiting; fails r (and returns true) when it can never run.
bool try_admit(lem_server* s, const std::shared_ptr<Request>& r) {
  const int64_t sbytes = int64_t(sizeof(double)) * r->npts;
  lem_problem_desc d = r->desc;
  for (int k = 0; k < 5; ++k) d.coef[k] = r->coef[k].empty() ? nullptr : r->coef[k].data();
  const bool want_split = r->tol >= 1e-6;
  CachedCtx* cc = nullptr;
  for (int attempt = want_split ? 0 : 1; attempt < 2 && !cc; ++attempt) {
    d.prec = attempt == 0 ? LEM_PREC_SPLIT : LEM_PREC_FP64;
    const std::string key = r->key + (attempt == 0 ? "/split" : "/fp64");
    {
      std::lock_guard<std::mutex> lk(s->mu);
      auto it = s->cache.find(key);
      if (it != s->cache.end()) {
        if (s->used + sbytes > s->budget) return false;
        cc = it->second.get();
        s->ctx_hits++;
        break;
      }
    }
    const int64_t need = ctx_bytes_estimate(d);
    if (need < 0) {
      finish(s, r, LEM_EINVAL);
      return true;
    }
    if (need + sbytes > s->budget) {  // larger than the whole budget
      if (attempt == 0) continue;
      finish(s, r, LEM_ENOMEM);
      return true;
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      // evict idle contexts, least recently used first, until the new one fits
      while (s->used + need + sbytes > s->budget) {
        auto victim = s->cache.end();
        for (auto it = s->cache.begin(); it != s->cache.end(); ++it)
          if (it->second->users == 0 && (victim == s->cache.end() || it->second->last_use < victim->second->last_use))
            victim = it;
        if (victim == s->cache.end()) break;
        lem_destroy(victim->second->ctx);
        cudaStreamDestroy(victim->second->stream);
        s->used -= victim->second->bytes;
        s->cache.erase(victim);
      }
      if (s->used + need + sbytes > s->budget) return false;  // wait for running requests
    }
    auto c = std::make_unique<CachedCtx>();
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      finish(s, r, LEM_ECUDA);
      return true;
    }
    const lem_status st = lem_create(&d, s->device, c->stream, &c->ctx);
    if (st != LEM_OK) {
      cudaStreamDestroy(c->stream);
      if (st == LEM_EINVAL && attempt == 0) continue;  // not eligible for the split path
      finish(s, r, st);
      return true;
    }
    c->bytes = need;
    std::lock_guard<std::mutex> lk(s->mu);
    s->used += need;
    s->ctx_misses++;
    cc = c.get();
    s->cache[key] = std::move(c);
  }
  if (!cc) {
    finish(s, r, LEM_EINVAL);
    return true;
  }
  if (cudaMalloc(&r->d_state, size_t(sbytes)) != cudaSuccess) {
    cudaGetLastError();
    r->d_state = nullptr;
    finish(s, r, LEM_ENOMEM);
    return true;
  }
  if (cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    finish(s, r, LEM_ECUDA);
    return true;
  }
  cudaMemcpyAsync(r->d_state, r->h_state, size_t(sbytes), cudaMemcpyHostToDevice, cc->stream);
  std::lock_guard<std::mutex> lk(s->mu);
  s->used += sbytes;
  r->accounted = true;
  cc->users++;
  cc->last_use = ++s->tick;
  r->cc = cc;
  r->state = RS::Running;
  r->remaining = r->nsteps;
  s->admitted++;
  if (!s->any_admitted) {
    s->any_admitted = true;
    s->t_first_admit = Clock::now();
  }
  return true;
}

void worker_loop(lem_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    bool progress = false;
    // admission in arrival order
    for (;;) {
      std::shared_ptr<Request> r;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->queue.empty()) break;
        r = s->queue.front();
      }
      if (!try_admit(s, r)) break;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        s->queue.pop_front();
      }
      if (r->state == RS::Running) s->active.push_back(r);
      progress = true;
    }
    // issue and retire chunks
    for (auto& r : s->active) {
      if (r->state != RS::Running && r->state != RS::CopyBack) continue;
      if (!r->in_flight) {
        if (r->state == RS::Running && r->remaining == 0) {
          cudaMemcpyAsync(r->h_state, r->d_state, sizeof(double) * size_t(r->npts), cudaMemcpyDeviceToHost,
                          r->cc->stream);
          r->state = RS::CopyBack;
        } else {
          const int chunk = std::min(r->remaining, kChunk);
          lem_status st = lem_step(r->cc->ctx, r->d_state, chunk);
          if (st != LEM_OK) { finish(s, r, st); progress = true; continue; }
          r->pending = chunk;
        }
        cudaEventRecord(r->ev, r->cc->stream);
        r->in_flight = true;
        progress = true;
        continue;
      }
      const cudaError_t q = cudaEventQuery(r->ev);
      if (q == cudaErrorNotReady) continue;
      r->in_flight = false;
      progress = true;
      if (q != cudaSuccess) { cudaGetLastError(); finish(s, r, LEM_ECUDA); continue; }
      if (r->state == RS::CopyBack) {
        finish(s, r, lem_sync(r->cc->ctx));
      } else {
        r->remaining -= r->pending;
        r->pending = 0;
      }
    }
    s->active.erase(std::remove_if(s->active.begin(), s->active.end(),
                                   [](const std::shared_ptr<Request>& r) {
                                     return r->state == RS::Done || r->state == RS::Failed;
                                   }),
                    s->active.end());
    if (s->stop.load()) {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->active.empty()) {
        for (auto& r : s->queue) { r->state = RS::Failed; r->status = LEM_EBUSY; s->failed++; }
        s->queue.clear();
        break;
      }
    }
    if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

}  // namespace

extern "C" {

lem_status lem_server_create(size_t hbm_budget_bytes, int device, lem_server** out) {
  if (!out) return lem::fail(LEM_EINVAL, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) { cudaGetLastError(); return lem::cuda_fail(e, "cudaGetDeviceCount"); }
  if (device < 0 || device >= ndev) return lem::fail(LEM_EINVAL, "device index out of range");
  lem_server* s = new lem_server();
  s->device = device;
  s->budget = int64_t(hbm_budget_bytes ? hbm_budget_bytes : kDefaultBudget);
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return LEM_OK;
}

lem_status lem_submit(lem_server* s, const lem_problem_desc* desc, double tol, double* h_state, int nsteps,
                      uint64_t* ticket) {
  if (!s || !desc || !h_state || !ticket) return lem::fail(LEM_EINVAL, "NULL argument");
  if (nsteps < 0) return lem::fail(LEM_EINVAL, "nsteps < 0");
  if (!(tol > 0.0)) return lem::fail(LEM_EINVAL, "tol must be > 0");
  LEM_TRY(lem::validate(desc));
  if (s->stop.load()) return lem::fail(LEM_EBUSY, "server is stopping");
  auto r = std::make_shared<Request>();
  r->desc = *desc;
  const int64_t npts = desc->ndim == 1 ? desc->n[0] : desc->n[0] * desc->n[1];
  const int64_t per = desc->coef_stride ? npts : 1;
  const int ncoef = desc->ndim == 1 ? 3 : 5;
  for (int k = 0; k < ncoef; ++k) r->coef[k].assign(desc->coef[k], desc->coef[k] + per);
  for (int k = 0; k < 5; ++k) r->desc.coef[k] = nullptr;
  r->key = make_key(r->desc, r->coef);
  r->tol = tol;
  r->h_state = h_state;
  r->npts = npts;
  r->nsteps = nsteps;
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  r->id = s->next_id++;
  s->all[r->id] = r;
  s->queue.push_back(r);
  s->submitted++;
  *ticket = r->id;
  return LEM_OK;
}

lem_status lem_poll(lem_server* s, uint64_t ticket, int* done) {
  if (!s || !done) return lem::fail(LEM_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return lem::fail(LEM_EINVAL, "unknown ticket");
  const RS st = it->second->state;
  *done = (st == RS::Done || st == RS::Failed) ? 1 : 0;
  if (st == RS::Failed) return lem::fail(it->second->status, "request failed");
  return LEM_OK;
}

lem_status lem_wait(lem_server* s, uint64_t ticket, double timeout_s) {
  const auto t0 = Clock::now();
  for (;;) {
    int done = 0;
    lem_status st = lem_poll(s, ticket, &done);
    if (done || st != LEM_OK) return st;
    if (std::chrono::duration<double>(Clock::now() - t0).count() > timeout_s)
      return lem::fail(LEM_ETIMEOUT, "request not done within the timeout");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

lem_status lem_server_get_stats(lem_server* s, lem_server_stats* o) {
  if (!s || !o) return lem::fail(LEM_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  o->submitted = s->submitted;
  o->admitted = s->admitted;
  o->completed = s->completed;
  o->failed = s->failed;
  o->queued = int64_t(s->queue.size());
  int64_t act = 0;
  for (auto& kv : s->all)
    if (kv.second->state == RS::Running || kv.second->state == RS::CopyBack) ++act;
  o->active = act;
  o->dof_steps = s->dof_steps;
  std::vector<double> l = s->lat_ms;
  std::sort(l.begin(), l.end());
  auto pct = [&](double p) {
    if (l.empty()) return 0.0;
    const size_t i = std::min(l.size() - 1, size_t(std::ceil(p * double(l.size()))) - (p > 0 ? 1 : 0));
    return l[i];
  };
  o->p50_ms = pct(0.50);
  o->p99_ms = pct(0.99);
  o->first_admit_to_last_done_s =
      s->any_admitted && s->completed ? std::chrono::duration<double>(s->t_last_done - s->t_first_admit).count() : 0.0;
  o->device_bytes = s->used;
  o->ctx_hits = s->ctx_hits;
  o->ctx_misses = s->ctx_misses;
  return LEM_OK;
}

void lem_server_destroy(lem_server* s) {
  if (!s) return;
  s->stop.store(true);
  if (s->worker.joinable()) s->worker.join();
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  for (auto& kv : s->cache) {
    lem_destroy(kv.second->ctx);
    cudaStreamDestroy(kv.second->stream);
  }
  s->cache.clear();
  if (prev >= 0) cudaSetDevice(prev);
  delete s;
}

}  // extern "C"
