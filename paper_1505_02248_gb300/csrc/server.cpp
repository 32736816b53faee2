// Serving layer: continuous batching of independent LEM requests on one device
// (lem_server_create / lem_submit / lem_poll / lem_wait / lem_server_get_stats /
// lem_server_destroy, declared in include/lem.h).
//
// One worker thread owns the device work. Each iteration it admits queued requests while
// their device memory fits the budget, then gives every admitted request that is not waiting
// on the GPU its next chunk of LEM steps (on the stream of the request's context) and checks
// finished chunks with events. A request whose steps are done gets its state copied back and
// completes. New requests therefore join the running set between chunks, and requests on
// different contexts run on different streams, so their kernels overlap on the device.
//
// Tiers. Requests with tol >= 1e-6 run on the tensor-core split tier where their problem
// allows it, the others on the FP64 path. The two tiers queue separately, each in arrival
// order: split-tier requests are admitted first; FP64-tier requests only while fewer than
// kMaxFp64Active of them run and the budget keeps a quarter free for the split tier. Streams
// of split-tier contexts have the device's highest priority and FP64-tier ones its lowest,
// and FP64-tier chunks are issued only while the split tier has nothing on the GPU (or one
// every kFp64GapMs), so long FP64 kernels do not hold back the quick tier.
//
// A split-tier request keeps its state in float-float on the device from admission to
// completion, with the residual scale carried from chunk to chunk, so its result is the same
// bit for bit as one lem_step call of all its steps, whatever else runs.
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
constexpr int kMaxFp64Active = 8;               // FP64-tier requests running at once
constexpr double kFp64GapMs = 50.0;             // FP64-tier chunk spacing while the split tier is busy
constexpr double kAdmitMs = 2.0;                // admission work per worker iteration

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
  std::string key;     // problem identity (context cache)
  std::string op_key;  // local operator identity (propagator sharing across mesh sizes)
  double tol = 0.0;
  double* h_state = nullptr;
  int64_t npts = 0;
  int nsteps = 0, remaining = 0, pending = 0;
  RS state = RS::Queued;
  lem_status status = LEM_OK;
  double* d_state = nullptr;
  // split tier: the float-float state (npts + npts floats) and the carried residual scale
  // (one unsigned after them), resident from admission to completion
  float* d_ff = nullptr;
  bool fp64_tier = false;     // tol < 1e-6
  bool counted_fp64 = false;  // counts against kMaxFp64Active
  int64_t acc_bytes = 0;      // bytes counted against the budget while admitted
  // pinned staging copy of the state for the asynchronous transfers: held from admission until
  // the copy in has completed, and again from the copy back until completion, so that the
  // pinned memory in use follows the transfers in flight, not the requests admitted
  double* h_stage = nullptr;
  size_t stage_bytes = 0;
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

// Problem identity for the context cache (everything but the state); with_n = false gives the
// local operator's identity, shared by meshes of every size.
std::string make_key(const lem_problem_desc& d, const std::vector<double>* coef, bool with_n = true) {
  uint64_t h = 1469598103934665603ull;
  h = fnv1a(&d.ndim, sizeof d.ndim, h);
  if (with_n) h = fnv1a(d.n, sizeof d.n, h);
  h = fnv1a(d.bc, sizeof d.bc, h);
  h = fnv1a(&d.coef_stride, sizeof d.coef_stride, h);
  h = fnv1a(&d.reaction, sizeof d.reaction, h);
  h = fnv1a(&d.dt, sizeof d.dt, h);
  h = fnv1a(d.tile, sizeof d.tile, h);
  h = fnv1a(d.overlap, sizeof d.overlap, h);
  h = fnv1a(&d.mode, sizeof d.mode, h);
  h = fnv1a(&d.refresh, sizeof d.refresh, h);
  h = fnv1a(&d.scheme, sizeof d.scheme, h);
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
  std::deque<std::shared_ptr<Request>> queue;    // split tier (tol >= 1e-6)
  std::deque<std::shared_ptr<Request>> queue64;  // FP64 tier
  int fp64_active = 0;                           // worker-owned
  Clock::time_point last_fp64_issue{};           // worker-owned
  std::vector<std::shared_ptr<Request>> active;  // worker-owned
  std::map<std::string, std::unique_ptr<CachedCtx>> cache;
  // pinned host buffers by size class (powers of two), reused across requests: transfers from
  // pageable memory would block the worker until the context's stream drains
  std::map<size_t, std::vector<void*>> stage_pool;
  int64_t stage_bytes_held = 0;
  // a built one-class context per local operator, with an event recorded after its build
  std::map<std::string, std::pair<lem_ctx*, cudaEvent_t>> donors;
  int64_t used = 0;
  uint64_t next_id = 1, tick = 0;
  std::atomic<bool> stop{false};
  std::thread worker;
  // statistics
  int64_t submitted = 0, admitted = 0, completed = 0, failed = 0, dof_steps = 0;
  int64_t ctx_hits = 0, ctx_misses = 0, ctx_adopted = 0;
  double admit_s = 0.0, issue_s = 0.0;  // worker host time in admission and in step launches
  double build_s = 0.0;                  // of admit_s: building donor propagators
  int64_t ctx_built = 0, adopt_failed = 0;
  std::vector<double> lat_ms;
  std::vector<double> lat_tier[2];
  int64_t tier_completed[2] = {0, 0}, tier_dof[2] = {0, 0};
  bool any_admitted = false;
  Clock::time_point t_first_admit, t_last_done;
};

namespace {

constexpr int64_t kStagePoolMax = int64_t(16) << 30;  // pinned bytes kept for reuse

// Host copy between a caller's state and a pinned staging buffer: large states are split over
// several threads (a single core copies about 10 GB/s, and the worker does one copy per
// request in each direction).
void pmemcpy(void* dst, const void* src, size_t bytes) {
  constexpr size_t kPart = size_t(4) << 20;
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t parts = std::min<size_t>(std::min<size_t>(8, hw), (bytes + kPart - 1) / kPart);
  if (parts <= 1) {
    std::memcpy(dst, src, bytes);
    return;
  }
  const size_t chunk = (bytes + parts - 1) / parts;
  std::vector<std::thread> th;
  for (size_t k = 1; k < parts; ++k) {
    const size_t o = k * chunk;
    if (o >= bytes) break;
    th.emplace_back([=] { std::memcpy(static_cast<char*>(dst) + o, static_cast<const char*>(src) + o, std::min(chunk, bytes - o)); });
  }
  std::memcpy(dst, src, std::min(chunk, bytes));
  for (auto& t : th) t.join();
}

void* stage_get(lem_server* s, size_t bytes, size_t* cls) {
  size_t c = 4096;
  while (c < bytes) c <<= 1;
  *cls = c;
  auto& v = s->stage_pool[c];
  if (!v.empty()) {
    void* p = v.back();
    v.pop_back();
    s->stage_bytes_held -= int64_t(c);
    return p;
  }
  void* p = nullptr;
  if (cudaHostAlloc(&p, c, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void stage_put(lem_server* s, void* p, size_t cls) {
  if (!p) return;
  if (s->stage_bytes_held + int64_t(cls) > kStagePoolMax) {
    cudaFreeHost(p);
    return;
  }
  s->stage_pool[cls].push_back(p);
  s->stage_bytes_held += int64_t(cls);
}

void finish(lem_server* s, const std::shared_ptr<Request>& r, lem_status st) {
  if (r->ev) { cudaEventDestroy(r->ev); r->ev = nullptr; }
  if (r->d_state) {
    // stream-ordered: a plain cudaFree would wait for every stream of the device
    cudaFreeAsync(r->d_state, r->cc ? r->cc->stream : nullptr);
    r->d_state = nullptr;
  }
  if (r->d_ff) {
    cudaFreeAsync(r->d_ff, r->cc ? r->cc->stream : nullptr);
    r->d_ff = nullptr;
  }
  if (r->h_stage) {
    if (st == LEM_OK) pmemcpy(r->h_state, r->h_stage, sizeof(double) * size_t(r->npts));
    stage_put(s, r->h_stage, r->stage_bytes);  // worker thread only
    r->h_stage = nullptr;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (r->accounted) {
    s->used -= r->acc_bytes;
    r->accounted = false;
  }
  if (r->counted_fp64) {
    s->fp64_active--;
    r->counted_fp64 = false;
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
    const int tier = r->fp64_tier ? 1 : 0;
    s->lat_tier[tier].push_back(s->lat_ms.back());
    s->tier_completed[tier]++;
    s->tier_dof[tier] += r->npts * r->nsteps;
    s->t_last_done = r->t_done;
  } else {
    r->state = RS::Failed;
    s->failed++;
  }
}

// Device bytes a context keeps (*scratch: the builder's transient workspace, freed after the
// build, which only a context that builds needs on top).
int64_t ctx_bytes_estimate(const lem_problem_desc& d, int64_t* scratch) {
  int64_t nt = 0, nc = 0, nl = 0, ni = 0;
  if (lem_plan_query(&d, &nt, &nc, &nl, &ni, nullptr) != LEM_OK) return -1;
  const int64_t npts = d.ndim == 1 ? d.n[0] : d.n[0] * d.n[1];
  int64_t b = 8 * (nc * ni * nl + 2 * npts + nt * (nl + ni)) + 5 * 8 * (d.coef_stride ? npts : 1);
  if (d.prec == LEM_PREC_SPLIT) b += 4 * 2 * npts + 3 * 2 * (npts + 8 * int64_t(std::sqrt(double(npts))) * 64) +
                                     3 * 2 * ni * nl * 2;
  // transient builder scratch (freed after the build): 19 n_loc^2 doubles per class batch
  const int64_t per = 19 * nl * nl * 8;
  const int64_t batch = std::max<int64_t>(1, std::min<int64_t>(nc, (int64_t(8) << 30) / std::max<int64_t>(per, 1)));
  *scratch = per * batch;
  return b;
}

// Evict idle contexts (no request on them), least recently used first and contexts that lend
// their propagators to later ones last, until `bytes` more fit within `cap` or nothing idle is
// left; `spare` is never evicted. Call with s->mu held.
void make_room(lem_server* s, int64_t bytes, int64_t cap, const CachedCtx* spare) {
  auto is_donor = [&](const lem_ctx* c) {
    for (auto& kv : s->donors)
      if (kv.second.first == c) return true;
    return false;
  };
  while (s->used + bytes > cap) {
    auto victim = s->cache.end();
    bool victim_donor = true;
    for (auto it = s->cache.begin(); it != s->cache.end(); ++it) {
      if (it->second->users != 0 || it->second.get() == spare) continue;
      const bool dn = is_donor(it->second->ctx);
      if (victim == s->cache.end() || (victim_donor && !dn) ||
          (victim_donor == dn && it->second->last_use < victim->second->last_use)) {
        victim = it;
        victim_donor = dn;
      }
    }
    if (victim == s->cache.end()) break;
    for (auto d = s->donors.begin(); d != s->donors.end();) {
      if (d->second.first == victim->second->ctx) {
        cudaEventDestroy(d->second.second);
        d = s->donors.erase(d);
      } else {
        ++d;
      }
    }
    lem_destroy(victim->second->ctx);
    cudaStreamDestroy(victim->second->stream);
    s->used -= victim->second->bytes;
    s->cache.erase(victim);
  }
}

// Admit r if its state (and a new context, when it needs one) fits within `cap` bytes of the
// budget. Returns false if r must keep waiting; fails r (and returns true) when it can never
// run. A split-tier request also holds a float-float copy of its state (8 more bytes a node).
bool try_admit(lem_server* s, const std::shared_ptr<Request>& r, int64_t cap) {
  const bool want_split = r->tol >= 1e-6;
  const int64_t sbytes = int64_t(sizeof(double)) * r->npts * (want_split ? 2 : 1) + (want_split ? 256 : 0);
  {
    // host-side fault injection for tests: LEM_FAULT=admit refuses every admission
    const char* f = std::getenv("LEM_FAULT");
    if (f && std::strcmp(f, "admit") == 0) {
      lem::fail(LEM_ENOMEM, "admission refused (LEM_FAULT=admit)");
      finish(s, r, LEM_ENOMEM);
      return true;
    }
  }
  lem_problem_desc d = r->desc;
  for (int k = 0; k < 5; ++k) d.coef[k] = r->coef[k].empty() ? nullptr : r->coef[k].data();
  CachedCtx* cc = nullptr;
  for (int attempt = want_split ? 0 : 1; attempt < 2 && !cc; ++attempt) {
    d.prec = attempt == 0 ? LEM_PREC_SPLIT : LEM_PREC_FP64;
    const std::string key = r->key + (attempt == 0 ? "/split" : "/fp64");
    {
      std::lock_guard<std::mutex> lk(s->mu);
      auto it = s->cache.find(key);
      if (it != s->cache.end()) {
        make_room(s, sbytes, cap, it->second.get());  // idle contexts make way for this state
        if (s->used + sbytes > cap) return false;
        cc = it->second.get();
        s->ctx_hits++;
        break;
      }
    }
    int64_t scratch = 0;
    const int64_t keep = ctx_bytes_estimate(d, &scratch);
    if (keep < 0) {
      finish(s, r, LEM_EINVAL);
      return true;
    }
    // donors are keyed by the local operator and the kind of products that built them; a
    // tensor-core-built propagator is lent only to split-tier contexts
    const bool tc_build = lem::builder_uses_tc(d.prec);
    const std::string own_key = r->op_key + (tc_build ? "/tc" : "/f64");
    const std::string f64_key = r->op_key + "/f64";
    bool has_donor;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      has_donor = s->donors.count(own_key) > 0 || s->donors.count(f64_key) > 0;
    }
    const int64_t need = keep + (has_donor ? 0 : scratch);  // room needed now
    if (need + sbytes > s->budget) {  // larger than the whole budget
      if (attempt == 0) continue;
      finish(s, r, LEM_ENOMEM);
      return true;
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      make_room(s, need + sbytes, cap, nullptr);
      if (s->used + need + sbytes > cap) return false;  // wait for running requests
    }
    auto c = std::make_unique<CachedCtx>();
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
      cudaGetLastError();
      least = greatest = 0;
    }
    if (cudaStreamCreateWithPriority(&c->stream, cudaStreamNonBlocking, want_split ? greatest : least) != cudaSuccess) {
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
    c->bytes = keep;
    {
      // a context with the same local operator (another mesh size) lends its propagators
      std::pair<lem_ctx*, cudaEvent_t> donor{nullptr, nullptr};
      {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->donors.find(own_key);
        if (it == s->donors.end()) it = s->donors.find(f64_key);
        if (it != s->donors.end()) donor = it->second;
      }
      if (donor.first && lem::adopt_propagators(c->ctx, donor.first, donor.second) == LEM_OK) {
        s->ctx_adopted++;
      } else if (donor.first) {
        s->adopt_failed++;
      } else if (c->ctx->classes.size() == 1) {
        // first context of this local operator: build now and lend the result to later ones
        // (other mesh sizes, the other precision tier)
        const auto tb = Clock::now();
        const lem_status bs = lem_build_propagators(c->ctx, nullptr);
        s->build_s += std::chrono::duration<double>(Clock::now() - tb).count();
        s->ctx_built++;
        cudaEvent_t built = nullptr;
        if (bs == LEM_OK && cudaEventCreateWithFlags(&built, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventRecord(built, c->stream) == cudaSuccess) {
          std::lock_guard<std::mutex> lk(s->mu);
          s->donors.emplace(own_key, std::make_pair(c->ctx, built));
        } else {
          cudaGetLastError();
          if (built) cudaEventDestroy(built);
        }
      }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->used += keep;
    s->ctx_misses++;
    cc = c.get();
    s->cache[key] = std::move(c);
  }
  if (!cc) {
    finish(s, r, LEM_EINVAL);
    return true;
  }
  if (cudaMallocAsync(reinterpret_cast<void**>(&r->d_state), size_t(sbytes), cc->stream) != cudaSuccess) {
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
  r->h_stage = static_cast<double*>(stage_get(s, sizeof(double) * size_t(r->npts), &r->stage_bytes));
  if (!r->h_stage) {
    finish(s, r, LEM_ENOMEM);
    return true;
  }
  const size_t fbytes = sizeof(double) * size_t(r->npts);
  pmemcpy(r->h_stage, r->h_state, fbytes);
  cudaMemcpyAsync(r->d_state, r->h_stage, fbytes, cudaMemcpyHostToDevice, cc->stream);
  if (cc->ctx->apply_path == LEM_APPLY_TC_SPLIT) {
    // resident float-float state + carried scale for the split tier
    if (cudaMallocAsync(reinterpret_cast<void**>(&r->d_ff), fbytes + 256, cc->stream) != cudaSuccess) {
      cudaGetLastError();
      r->d_ff = nullptr;
      finish(s, r, LEM_ENOMEM);
      return true;
    }
    const lem_status cs = lem::split_to_ff(cc->ctx, r->d_state, r->d_ff, r->d_ff + r->npts);
    if (cs != LEM_OK) {
      finish(s, r, cs);
      return true;
    }
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->used += sbytes;
  r->acc_bytes = sbytes;
  r->accounted = true;
  cc->users++;
  cc->last_use = ++s->tick;
  r->cc = cc;
  r->state = RS::Running;
  r->remaining = r->nsteps;
  if (r->fp64_tier) {
    r->counted_fp64 = true;
    s->fp64_active++;
  }
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
    // admission: the split tier first, then the FP64 tier (each in arrival order; FP64-tier
    // requests only while fewer than kMaxFp64Active run, within three quarters of the budget)
    // (at most kAdmitMs of admission work per iteration, so that a burst of arrivals does not
    // keep the worker from issuing the running requests' next steps)
    const auto t_adm = Clock::now();
    for (int tier = 0; tier < 2; ++tier) {
      for (;;) {
        if (tier == 1 && s->fp64_active >= kMaxFp64Active) break;
        if (std::chrono::duration<double, std::milli>(Clock::now() - t_adm).count() > kAdmitMs) break;
        std::shared_ptr<Request> r;
        {
          std::lock_guard<std::mutex> lk(s->mu);
          std::deque<std::shared_ptr<Request>>& q = tier == 0 ? s->queue : s->queue64;
          if (q.empty()) break;
          r = q.front();
        }
        const auto ta = Clock::now();
        const bool admitted = try_admit(s, r, tier == 0 ? s->budget : s->budget - s->budget / 4);
        s->admit_s += std::chrono::duration<double>(Clock::now() - ta).count();
        if (!admitted) break;
        {
          std::lock_guard<std::mutex> lk(s->mu);
          (tier == 0 ? s->queue : s->queue64).pop_front();
        }
        if (r->state == RS::Running) s->active.push_back(r);
        progress = true;
      }
    }
    // issue and retire chunks. FP64-tier steps are issued only while no split-tier request
    // has work on the GPU or waits for admission (a long FP64 kernel holds SMs that the
    // tensor-core kernels need whole), or at most every kFp64GapMs when the split tier never
    // pauses, so that the FP64 tier still advances.
    bool quick_busy = false;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      quick_busy = !s->queue.empty();
    }
    for (auto& r : s->active)
      if (!r->fp64_tier && (r->in_flight || r->state == RS::Running)) quick_busy = true;
    const auto now = Clock::now();
    bool fp64_ok = !quick_busy ||
                   std::chrono::duration<double, std::milli>(now - s->last_fp64_issue).count() >= kFp64GapMs;
    for (auto& r : s->active) {
      if (r->state != RS::Running && r->state != RS::CopyBack) continue;
      if (!r->in_flight) {
        if (r->fp64_tier && r->state == RS::Running && r->remaining > 0) {
          if (!fp64_ok) continue;
          if (quick_busy) fp64_ok = false;  // one FP64 chunk per gap
          s->last_fp64_issue = now;
        }
        if (r->state == RS::Running && r->remaining == 0) {
          if (r->d_ff) {
            const lem_status cs = lem::split_from_ff(r->cc->ctx, r->d_ff, r->d_ff + r->npts, r->d_state);
            if (cs != LEM_OK) { finish(s, r, cs); progress = true; continue; }
          }
          if (!r->h_stage) r->h_stage = static_cast<double*>(stage_get(s, sizeof(double) * size_t(r->npts), &r->stage_bytes));
          if (!r->h_stage) { finish(s, r, LEM_ENOMEM); progress = true; continue; }
          cudaMemcpyAsync(r->h_stage, r->d_state, sizeof(double) * size_t(r->npts), cudaMemcpyDeviceToHost,
                          r->cc->stream);
          r->state = RS::CopyBack;
        } else {
          // FP64-tier requests advance one step per chunk: their steps are long, and shorter
          // chunks interleave better with the split tier
          const int chunk = std::min(r->remaining, r->fp64_tier ? 1 : kChunk);
          const auto ti = Clock::now();
          lem_status st = LEM_OK;
          if (r->d_ff) {  // resident float-float state; the scale carries over from the last chunk
            lem_ctx* c = r->cc->ctx;
            if (!c->built) st = lem_build_propagators(c, nullptr);
            if (st == LEM_OK)
              st = lem::split_run(c, r->d_ff, r->d_ff + r->npts, chunk, reinterpret_cast<unsigned*>(r->d_ff + 2 * r->npts),
                                  r->remaining < r->nsteps);
          } else {
            st = lem_step(r->cc->ctx, r->d_state, chunk);
          }
          s->issue_s += std::chrono::duration<double>(Clock::now() - ti).count();
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
        finish(s, r, lem::split_check_error(r->cc->ctx));  // the event covers this request's work
      } else {
        r->remaining -= r->pending;
        r->pending = 0;
        if (r->h_stage) {  // the copy in ran before this chunk: its staging buffer is free again
          stage_put(s, r->h_stage, r->stage_bytes);
          r->h_stage = nullptr;
        }
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
        for (auto* q : {&s->queue, &s->queue64}) {
          for (auto& r : *q) { r->state = RS::Failed; r->status = LEM_EBUSY; s->failed++; }
          q->clear();
        }
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
  {
    // request states come from the device's stream-ordered pool; keep freed blocks in it
    // (up to the budget) instead of returning them to the CUDA driver at every synchronisation
    lem::DeviceGuard g(device);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
      uint64_t keep = uint64_t(s->budget);
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
  }
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
  if (desc->complex_values) return lem::fail(LEM_EINVAL, "the server takes real problems");
  if (desc->reaction == 2) return lem::fail(LEM_EINVAL, "the server does not take the porous-medium problem");
  if (s->stop.load()) return lem::fail(LEM_EBUSY, "server is stopping");
  auto r = std::make_shared<Request>();
  r->desc = *desc;
  const int64_t npts = desc->ndim == 1 ? desc->n[0] : desc->n[0] * desc->n[1];
  const int64_t per = desc->coef_stride ? npts : 1;
  const int ncoef = desc->ndim == 1 ? 3 : 5;
  for (int k = 0; k < ncoef; ++k) r->coef[k].assign(desc->coef[k], desc->coef[k] + per);
  for (int k = 0; k < 5; ++k) r->desc.coef[k] = nullptr;
  r->key = make_key(r->desc, r->coef);
  r->op_key = make_key(r->desc, r->coef, false);
  r->tol = tol;
  r->fp64_tier = !(tol >= 1e-6);
  r->h_state = h_state;
  r->npts = npts;
  r->nsteps = nsteps;
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  r->id = s->next_id++;
  s->all[r->id] = r;
  (r->fp64_tier ? s->queue64 : s->queue).push_back(r);
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

lem_status lem_server_reset_stats(lem_server* s) {
  if (!s) return lem::fail(LEM_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  s->submitted = s->admitted = s->completed = s->failed = s->dof_steps = 0;
  s->ctx_hits = s->ctx_misses = s->ctx_adopted = s->ctx_built = s->adopt_failed = 0;
  s->admit_s = s->issue_s = s->build_s = 0.0;
  s->lat_ms.clear();
  for (int t = 0; t < 2; ++t) {
    s->lat_tier[t].clear();
    s->tier_completed[t] = s->tier_dof[t] = 0;
  }
  s->any_admitted = false;
  return LEM_OK;
}

lem_status lem_server_get_stats(lem_server* s, lem_server_stats* o) {
  if (!s || !o) return lem::fail(LEM_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  o->submitted = s->submitted;
  o->admitted = s->admitted;
  o->completed = s->completed;
  o->failed = s->failed;
  o->queued = int64_t(s->queue.size() + s->queue64.size());
  int64_t act = 0;
  for (auto& kv : s->all)
    if (kv.second->state == RS::Running || kv.second->state == RS::CopyBack) ++act;
  o->active = act;
  o->dof_steps = s->dof_steps;
  auto pct = [](std::vector<double> l, double p) {
    if (l.empty()) return 0.0;
    std::sort(l.begin(), l.end());
    const size_t i = std::min(l.size() - 1, size_t(std::ceil(p * double(l.size()))) - (p > 0 ? 1 : 0));
    return l[i];
  };
  o->p50_ms = pct(s->lat_ms, 0.50);
  o->p99_ms = pct(s->lat_ms, 0.99);
  for (int t = 0; t < 2; ++t) {
    o->tier_completed[t] = s->tier_completed[t];
    o->tier_dof_steps[t] = s->tier_dof[t];
    o->tier_p50_ms[t] = pct(s->lat_tier[t], 0.50);
    o->tier_p99_ms[t] = pct(s->lat_tier[t], 0.99);
  }
  o->first_admit_to_last_done_s =
      s->any_admitted && s->completed ? std::chrono::duration<double>(s->t_last_done - s->t_first_admit).count() : 0.0;
  o->device_bytes = s->used;
  o->ctx_hits = s->ctx_hits;
  o->ctx_misses = s->ctx_misses;
  o->ctx_adopted = s->ctx_adopted;
  o->worker_admit_s = s->admit_s;
  o->worker_issue_s = s->issue_s;
  o->worker_build_s = s->build_s;
  o->ctx_built = s->ctx_built;
  o->adopt_failed = s->adopt_failed;
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
  for (auto& kv : s->donors) cudaEventDestroy(kv.second.second);
  s->donors.clear();
  for (auto& kv : s->stage_pool)
    for (void* p : kv.second) cudaFreeHost(p);
  s->stage_pool.clear();
  if (prev >= 0) cudaSetDevice(prev);
  delete s;
}

}  // extern "C"
