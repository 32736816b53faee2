// extern "C" entry points of liblem.so (declared in include/lem.h).
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "lem_internal.h"

namespace lem {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

lem_status fail(lem_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

lem_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? LEM_ENOMEM : LEM_ECUDA;
}

// Host-side fault injection for tests: LEM_FAULT=alloc makes every device allocation of
// a context fail with LEM_ENOMEM (no GPU fault is involved).
static bool fault_alloc() {
  const char* f = std::getenv("LEM_FAULT");
  return f && std::strcmp(f, "alloc") == 0;
}

lem_status dev_alloc(lem_ctx* ctx, void** p, size_t bytes) {
  *p = nullptr;
  if (fault_alloc()) return fail(LEM_ENOMEM, "device allocation refused (LEM_FAULT=alloc)");
  if (bytes == 0) bytes = 16;
  // stream-ordered: a context made or freed while other streams run (the server) must not
  // wait for the whole device, as cudaMalloc / cudaFree may
  cudaError_t e = cudaMallocAsync(p, bytes, ctx->stream);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(LEM_ENOMEM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed: " +
                                cudaGetErrorString(e));
  }
  ctx->device_bytes += int64_t(bytes);
  return LEM_OK;
}

}  // namespace lem

lem::Stencil lem_ctx::stencil() const {
  lem::Stencil s{};
  const int64_t step = desc.coef_stride ? npts : 1;
  for (int k = 0; k < 5; ++k) s.c[k] = d_coef + k * step;
  s.stride = desc.coef_stride;
  return s;
}

// Record a start event for one apply-kernel launch; returns its stop event through *stop.
cudaError_t lem_ctx::timing_begin(cudaEvent_t* stop) {
  *stop = nullptr;
  if (!timing) return cudaSuccess;
  if (timing_count++ % timing_period != 0) return cudaSuccess;
  if (ev_used + 2 > ev_pool.size()) {
    for (int i = 0; i < 256; ++i) {
      cudaEvent_t e;
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return r;
      ev_pool.push_back(e);
    }
  }
  cudaEvent_t start = ev_pool[ev_used];
  *stop = ev_pool[ev_used + 1];
  ev_used += 2;
  return cudaEventRecord(start, stream);
}

void lem_ctx::timing_end(cudaEvent_t stop) {
  if (stop) cudaEventRecord(stop, stream);
}

using namespace lem;

namespace {
// NVTX range for profiler timelines (a no-op without a profiler attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

namespace {

void free_ctx(lem_ctx* c) {
  if (!c) return;
  split_destroy(c);
  band_destroy(c);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  cudaFreeAsync(c->d_coef, c->stream);
  cudaFreeAsync(c->d_tiles, c->stream);
  cudaFreeAsync(c->d_class_order, c->stream);
  cudaFreeAsync(c->d_P, c->stream);
  cudaFreeAsync(c->d_P32, c->stream);
  cudaFreeAsync(c->d_P3, c->stream);
  cudaFreeAsync(c->d_P3_32, c->stream);
  cudaFreeAsync(c->d_um, c->stream);
  cudaFreeAsync(c->d_u0, c->stream);
  cudaFreeAsync(c->d_r, c->stream);
  cudaFreeAsync(c->d_U, c->stream);
  cudaFreeAsync(c->d_Y, c->stream);
  cudaFreeAsync(c->d_state_tmp, c->stream);
  cudaFreeAsync(c->d_status, c->stream);
  delete c;
}

lem_status init_plan(lem_ctx* c, const lem_problem_desc* desc) {
  LEM_TRY(validate(desc));
  c->desc = *desc;
  for (int k = 0; k < 5; ++k) c->desc.coef[k] = nullptr;  // host pointers are not kept
  if (desc->ndim == 1) {
    c->ny = 1; c->nx = desc->n[0];
    c->bcy = LEM_BC_DIRICHLET0; c->bcx = desc->bc[0];
  } else {
    c->ny = desc->n[0]; c->nx = desc->n[1];
    c->bcy = desc->bc[0]; c->bcx = desc->bc[1];
  }
  c->npts = c->ny * c->nx;
  LEM_TRY(make_plan(c));
  if (c->tiles.size() > 65535) return fail(LEM_EINVAL, "more than 65535 tiles");
  return LEM_OK;
}

}  // namespace

namespace lem {

// Take the propagators of `src` instead of building them: both contexts have one class whose
// local matrix is the same (same stencil, dt, tile, overlap, mode and window shape; the mesh
// size may differ, which does not change a window that does not wrap onto itself). `built` is
// an event recorded on src's stream after its build: dst's stream waits for it, the host
// does not.
lem_status adopt_propagators(lem_ctx* dst, lem_ctx* src, cudaEvent_t built) {
  if (!dst || !src || !src->built) return fail(LEM_EINVAL, "no built donor");
  if (dst->classes.size() != 1 || src->classes.size() != 1) return fail(LEM_EINVAL, "donor needs one class");
  const ClassDesc &a = dst->classes[0], &b = src->classes[0];
  const lem_problem_desc &da = dst->desc, &db = src->desc;
  bool same = da.ndim == db.ndim && da.mode == db.mode && da.dt == db.dt && da.reaction == 0 && db.reaction == 0 &&
              da.scheme == LEM_SCHEME_EULER && db.scheme == LEM_SCHEME_EULER &&
              da.coef_stride == 0 && db.coef_stride == 0 && dst->n_loc == src->n_loc && dst->n_int == src->n_int;
  for (int k = 0; k < da.ndim && same; ++k)  // per mesh axis (a 1D problem has one)
    same = da.tile[k] == db.tile[k] && da.overlap[k] == db.overlap[k] && da.bc[k] == db.bc[k] &&
           a.wext[k] == b.wext[k] && a.iext[k] == b.iext[k] && a.iofs[k] == b.iofs[k] && !a.whole[k] && !b.whole[k];
  DeviceGuard g(dst->device);
  same = same && dst->h_coef == src->h_coef;  // the dt-scaled constant stencils
  // an FP64-tier context takes only propagators built with FP64 products
  same = same && (dst->build_tc || !src->build_tc);
  if (!same) return fail(LEM_EINVAL, "donor has a different local operator");
  LEM_CUDA_TRY(cudaStreamWaitEvent(dst->stream, built, 0));
  LEM_CUDA_TRY(cudaMemcpyAsync(dst->d_P, src->d_P, sizeof(double) * dst->n_int * dst->n_loc,
                               cudaMemcpyDeviceToDevice, dst->stream));
  dst->squarings = src->squarings;
  dst->built = true;
  dst->build_gen++;
  dst->steps_since_build = 0;
  return LEM_OK;
}

}  // namespace lem

extern "C" {

const char* lem_status_str(lem_status s) {
  switch (s) {
    case LEM_OK: return "LEM_OK";
    case LEM_EINVAL: return "LEM_EINVAL";
    case LEM_ENOMEM: return "LEM_ENOMEM";
    case LEM_ECUDA: return "LEM_ECUDA";
    case LEM_EBUSY: return "LEM_EBUSY";
    case LEM_ENOTREADY: return "LEM_ENOTREADY";
    case LEM_ETIMEOUT: return "LEM_ETIMEOUT";
    case LEM_ENUMERIC: return "LEM_ENUMERIC";
  }
  return "LEM_UNKNOWN";
}

const char* lem_last_error(void) { return lem::g_last_error.c_str(); }

lem_status lem_plan_query(const lem_problem_desc* desc, int64_t* ntiles, int64_t* nclasses,
                          int64_t* n_loc, int64_t* n_int, int32_t* tile_info) {
  lem_ctx tmp;
  LEM_TRY(init_plan(&tmp, desc));
  if (ntiles) *ntiles = int64_t(tmp.tiles.size());
  if (nclasses) *nclasses = int64_t(tmp.classes.size());
  if (n_loc) *n_loc = tmp.n_loc;
  if (n_int) *n_int = tmp.n_int;
  if (tile_info) {
    for (size_t i = 0; i < tmp.tiles.size(); ++i) {
      const TileDesc& t = tmp.tiles[i];
      int32_t* o = tile_info + 11 * i;
      o[0] = t.org[0]; o[1] = t.org[1]; o[2] = t.wext[0]; o[3] = t.wext[1];
      o[4] = t.iofs[0]; o[5] = t.iofs[1]; o[6] = t.iext[0]; o[7] = t.iext[1];
      o[8] = t.t0[0]; o[9] = t.t0[1]; o[10] = t.cls;
    }
  }
  return LEM_OK;
}

lem_status lem_create(const lem_problem_desc* desc, int device, void* cuda_stream, lem_ctx** out) {
  if (!out) return fail(LEM_EINVAL, "out is NULL");
  *out = nullptr;
  lem_ctx* c = new (std::nothrow) lem_ctx();
  if (!c) return fail(LEM_ENOMEM, "host allocation failed");
  lem_status s = init_plan(c, desc);
  if (s != LEM_OK) { delete c; return s; }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || device < 0 || device >= ndev) {
    delete c;
    if (e != cudaSuccess) { cudaGetLastError(); return cuda_fail(e, "cudaGetDeviceCount"); }
    return fail(LEM_EINVAL, "device index out of range");
  }
  c->device = device;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  DeviceGuard g(device);
  // dt-scaled coefficients (complex: the five real parts, then the five imaginary parts)
  const int64_t per = desc->coef_stride ? c->npts : 1;
  c->cplx = desc->complex_values ? 1 : 0;
  std::vector<double> hc((c->cplx ? 10 : 5) * per, 0.0);
  const int ncoef = desc->ndim == 1 ? 3 : 5;
  for (int k = 0; k < ncoef; ++k)
    for (int64_t i = 0; i < per; ++i) {
      hc[k * per + i] = desc->dt * desc->coef[k][i];
      if (c->cplx && desc->coef_im[k]) hc[(5 + k) * per + i] = desc->dt * desc->coef_im[k][i];
    }
  if (c->cplx) {  // propagators of the real embedding: twice the rows and columns
    c->n_loc *= 2;
    c->n_int *= 2;
  }
  const int64_t vals = (c->cplx ? 2 : 1) * c->npts;  // doubles per state
  const size_t nt = c->tiles.size(), nc = c->classes.size();
  s = dev_alloc(c, reinterpret_cast<void**>(&c->d_coef), sizeof(double) * hc.size());
  if (s == LEM_OK) s = dev_alloc(c, reinterpret_cast<void**>(&c->d_tiles), sizeof(TileDesc) * nt);
  if (s == LEM_OK) s = dev_alloc(c, reinterpret_cast<void**>(&c->d_class_order), sizeof(int32_t) * nt);
  if (s == LEM_OK) s = dev_alloc(c, reinterpret_cast<void**>(&c->d_P), sizeof(double) * nc * c->n_int * c->n_loc);
  if (s == LEM_OK) s = dev_alloc(c, reinterpret_cast<void**>(&c->d_r), sizeof(double) * vals);
  if (s == LEM_OK && desc->scheme == LEM_SCHEME_RB3) {
    s = dev_alloc(c, reinterpret_cast<void**>(&c->d_P3), sizeof(double) * nc * c->n_int * c->n_loc);
    if (s == LEM_OK) s = dev_alloc(c, reinterpret_cast<void**>(&c->d_um), sizeof(double) * c->npts);
    if (s == LEM_OK) s = dev_alloc(c, reinterpret_cast<void**>(&c->d_u0), sizeof(double) * c->npts);
  }
  if (s == LEM_OK) s = dev_alloc(c, reinterpret_cast<void**>(&c->d_status), sizeof(int));
  if (s != LEM_OK) { free_ctx(c); return s; }
  if (!desc->coef_stride) c->h_coef = hc;
  e = cudaMemcpyAsync(c->d_coef, hc.data(), sizeof(double) * hc.size(), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_tiles, c->tiles.data(), sizeof(TileDesc) * nt, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_class_order, c->class_order.data(), sizeof(int32_t) * nt, cudaMemcpyHostToDevice,
                        c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
  if (e != cudaSuccess) { free_ctx(c); return cuda_fail(e, "lem_create upload"); }
  // apply path: tensor-core split for a shared propagator, else a batched GEMV when tiles
  // have (mostly) their own propagators or FP32 propagators are asked for, else grouped GEMMs
  const bool many_classes = c->classes.size() * 8 > c->tiles.size();
  c->build_tc = builder_uses_tc(desc->prec);
  const bool split_tier = desc->prec == LEM_PREC_SPLIT || desc->prec == LEM_PREC_SPLIT_FAST;
  if (desc->scheme == LEM_SCHEME_RB3 || c->cplx) {  // two propagator sets / complex: the batched GEMV
    // (FP32 propagators in PHI mode only: in EXP mode they would round the whole state every step)
    c->apply_path = desc->prec == LEM_PREC_SPLIT_FAST && desc->mode == LEM_MODE_PHI ? LEM_APPLY_F32_GEMV
                                                                                   : LEM_APPLY_FP64_GEMV;
  } else if (split_tier && split_eligible(c)) {
    c->apply_path = LEM_APPLY_TC_SPLIT;
    s = split_prepare(c);
    if (s != LEM_OK) { free_ctx(c); return s; }
  } else if (desc->prec == LEM_PREC_SPLIT_FAST && desc->mode == LEM_MODE_PHI) {
    c->apply_path = LEM_APPLY_F32_GEMV;
  } else {
    c->apply_path = many_classes ? LEM_APPLY_FP64_GEMV : LEM_APPLY_FP64_GEMM;
  }
  if (c->apply_path == LEM_APPLY_F32_GEMV || c->apply_path == LEM_APPLY_FP64_GEMV) {
    s = gemv_set_smem(c);
    if (s != LEM_OK) { free_ctx(c); return s; }
  }
  c->apply_path_dense = c->apply_path;
  // the context's memory is ready for use from any stream once its stream has run the
  // allocations, uploads and clears above
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) { free_ctx(c); return cuda_fail(e, "lem_create"); }
  *out = c;
  return LEM_OK;
}

lem_status lem_build_propagators(lem_ctx* ctx, const double* d_state) {
  if (!ctx) return fail(LEM_EINVAL, "ctx is NULL");
  DeviceGuard g(ctx->device);
  LEM_TRY(build_propagators(ctx, d_state));
  return LEM_OK;  // the split path repacks the new propagator lazily (build_gen)
}

// lem_step's work; device_state false: d_state is mapped host memory, which the split path
// reads with a separate streaming conversion rather than in its first stencil pass
static lem_status step_impl(lem_ctx* ctx, double* d_state, int nsteps, bool device_state) {
  if (!ctx) return fail(LEM_EINVAL, "ctx is NULL");
  if (!d_state) return fail(LEM_EINVAL, "state is NULL");
  if (nsteps < 0) return fail(LEM_EINVAL, "nsteps < 0");
  if (nsteps == 0) return LEM_OK;
  DeviceGuard g(ctx->device);
  NvtxRange range("lem_step");
  if (!ctx->built) LEM_TRY(build_propagators(ctx, d_state));
  if (ctx->band_tol >= 0.0) {  // truncated propagators
    for (int k = 0; k < nsteps; ++k) {
      if (ctx->desc.reaction && ctx->desc.refresh > 0 && ctx->steps_since_build >= ctx->desc.refresh)
        LEM_TRY(build_propagators(ctx, d_state));
      LEM_TRY(band_step(ctx, d_state));
      ctx->steps_since_build++;
    }
    return LEM_OK;
  }
  if (ctx->split) return split_step(ctx, d_state, nsteps, device_state);
  if (ctx->apply_path == LEM_APPLY_FP64_GEMV || ctx->apply_path == LEM_APPLY_F32_GEMV) {
    bool done = false;  // small linear problems: every step in one persistent launch
    LEM_TRY(step_gemv_multi(ctx, d_state, nsteps, ctx->apply_path == LEM_APPLY_F32_GEMV, &done));
    if (done) {
      ctx->steps_since_build += nsteps;
      return LEM_OK;
    }
  }
  for (int k = 0; k < nsteps; ++k) {
    if (ctx->desc.reaction && ctx->desc.refresh > 0 && ctx->steps_since_build >= ctx->desc.refresh)
      LEM_TRY(build_propagators(ctx, d_state));
    if (ctx->apply_path == LEM_APPLY_FP64_GEMM) LEM_TRY(step_fp64(ctx, d_state));
    else LEM_TRY(step_gemv(ctx, d_state, ctx->apply_path == LEM_APPLY_F32_GEMV));
    ctx->steps_since_build++;
  }
  return LEM_OK;
}

lem_status lem_step(lem_ctx* ctx, double* d_state, int nsteps) { return step_impl(ctx, d_state, nsteps, true); }

lem_status lem_step_host(lem_ctx* ctx, double* h_state, int nsteps) {
  if (!ctx) return fail(LEM_EINVAL, "ctx is NULL");
  if (!h_state) return fail(LEM_EINVAL, "state is NULL");
  DeviceGuard g(ctx->device);
  // The tensor-core split path reads the FP64 state once (into its float-float state) and
  // writes it once at the end. When the host buffer is pinned memory mapped into the device's
  // address space, those two kernels use it in place: one pass over the host link each way
  // and no separate copies.
  if (ctx->split && ctx->built && ctx->band_tol < 0.0 && nsteps > 0) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, h_state) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer) {
      LEM_TRY(step_impl(ctx, static_cast<double*>(at.devicePointer), nsteps, false));
      LEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
      return split_check_error(ctx);
    }
    cudaGetLastError();  // (pageable memory: the query's error, if any, is not the caller's)
  }
  const size_t bytes = sizeof(double) * ctx->npts * (ctx->cplx ? 2 : 1);
  if (!ctx->d_state_tmp) LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->d_state_tmp), bytes));
  LEM_CUDA_TRY(cudaMemcpyAsync(ctx->d_state_tmp, h_state, bytes, cudaMemcpyHostToDevice, ctx->stream));
  LEM_TRY(lem_step(ctx, ctx->d_state_tmp, nsteps));
  LEM_CUDA_TRY(cudaMemcpyAsync(h_state, ctx->d_state_tmp, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  LEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return split_check_error(ctx);
}

lem_status lem_get_propagator(lem_ctx* ctx, int64_t cls, double* h_out) {
  if (!ctx || !h_out) return fail(LEM_EINVAL, "NULL argument");
  if (cls < 0 || cls >= int64_t(ctx->classes.size())) return fail(LEM_EINVAL, "class out of range");
  if (!ctx->built) return fail(LEM_ENOTREADY, "propagators not built");
  DeviceGuard g(ctx->device);
  LEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  LEM_CUDA_TRY(cudaMemcpy(h_out, ctx->d_P + cls * ctx->n_int * ctx->n_loc,
                          sizeof(double) * ctx->n_int * ctx->n_loc, cudaMemcpyDeviceToHost));
  return LEM_OK;
}

lem_status lem_get_propagator_phi3(lem_ctx* ctx, int64_t cls, double* h_out) {
  if (!ctx || !h_out) return fail(LEM_EINVAL, "NULL argument");
  if (!ctx->d_P3) return fail(LEM_EINVAL, "no phi_3 propagators (scheme is not LEM_SCHEME_RB3)");
  if (cls < 0 || cls >= int64_t(ctx->classes.size())) return fail(LEM_EINVAL, "class out of range");
  if (!ctx->built) return fail(LEM_ENOTREADY, "propagators not built");
  DeviceGuard g(ctx->device);
  LEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  LEM_CUDA_TRY(cudaMemcpy(h_out, ctx->d_P3 + cls * ctx->n_int * ctx->n_loc,
                          sizeof(double) * ctx->n_int * ctx->n_loc, cudaMemcpyDeviceToHost));
  return LEM_OK;
}

lem_status lem_set_propagators(lem_ctx* ctx, const double* h_P, const int* h_squarings) {
  if (!ctx || !h_P) return fail(LEM_EINVAL, "NULL argument");
  if (ctx->d_P3) return fail(LEM_EINVAL, "a third-order Rosenbrock context builds both propagator sets itself");
  DeviceGuard g(ctx->device);
  const size_t n = size_t(ctx->classes.size()) * size_t(ctx->n_int) * size_t(ctx->n_loc);
  LEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  LEM_CUDA_TRY(cudaMemcpy(ctx->d_P, h_P, sizeof(double) * n, cudaMemcpyHostToDevice));
  for (size_t c = 0; c < ctx->classes.size(); ++c) ctx->squarings[c] = h_squarings ? h_squarings[c] : -1;
  ctx->built = true;
  ctx->build_gen++;
  ctx->steps_since_build = 0;
  return LEM_OK;
}

int64_t lem_tile_class(const lem_ctx* ctx, int64_t tile) {
  if (!ctx || tile < 0 || tile >= int64_t(ctx->tiles.size())) return -1;
  return ctx->tiles[tile].cls;
}

int lem_class_squarings(const lem_ctx* ctx, int64_t cls) {
  if (!ctx || cls < 0 || cls >= int64_t(ctx->classes.size())) return -1;
  return ctx->squarings[cls];
}

lem_status lem_get_info(const lem_ctx* ctx, lem_info* out) {
  if (!ctx || !out) return fail(LEM_EINVAL, "NULL argument");
  out->ntiles = int64_t(ctx->tiles.size());
  out->nclasses = int64_t(ctx->classes.size());
  out->n_loc = ctx->n_loc;
  out->n_int = ctx->n_int;
  int smax = -1;
  for (int s : ctx->squarings) smax = s > smax ? s : smax;
  out->squarings_max = smax;
  out->built = ctx->built ? 1 : 0;
  out->split_path = ctx->split ? 1 : 0;
  out->device_bytes = ctx->device_bytes;
  out->apply_path = ctx->apply_path;
  return LEM_OK;
}

lem_status lem_set_truncation(lem_ctx* ctx, double tol) {
  if (!ctx) return fail(LEM_EINVAL, "ctx is NULL");
  if (tol != tol) return fail(LEM_EINVAL, "tol is NaN");
  if (tol < 0.0) {
    ctx->band_tol = -1.0;
    ctx->apply_path = ctx->apply_path_dense;
    return LEM_OK;
  }
  if (ctx->cplx) return fail(LEM_EINVAL, "truncated propagators take real problems only");
  if (ctx->desc.scheme != LEM_SCHEME_EULER)
    return fail(LEM_EINVAL, "truncated propagators take the exponential Euler scheme only");
  ctx->band_tol = tol;
  ctx->band_gen = -1;  // extents follow the new tolerance at the next step
  const bool f32 = ctx->desc.prec == LEM_PREC_SPLIT_FAST && ctx->desc.mode == LEM_MODE_PHI;
  ctx->apply_path = f32 ? LEM_APPLY_F32_BAND : LEM_APPLY_FP64_BAND;
  return LEM_OK;
}

lem_status lem_get_band(lem_ctx* ctx, int64_t cls, int32_t* ext, int64_t* row_values) {
  if (!ctx || !ext) return fail(LEM_EINVAL, "NULL argument");
  if (ctx->band_tol < 0.0) return fail(LEM_EINVAL, "no truncation set (lem_set_truncation)");
  if (cls < -1 || cls >= int64_t(ctx->classes.size())) return fail(LEM_EINVAL, "class out of range");
  if (!ctx->built) return fail(LEM_ENOTREADY, "propagators not built");
  DeviceGuard g(ctx->device);
  return band_get(ctx, cls, ext, row_values);
}

lem_status lem_set_timing(lem_ctx* ctx, int enable) {
  if (!ctx) return fail(LEM_EINVAL, "ctx is NULL");
  if (enable < 0) return fail(LEM_EINVAL, "enable < 0");
  ctx->timing = enable != 0;
  ctx->timing_period = enable > 1 ? enable : 1;
  ctx->timing_count = 0;
  return LEM_OK;
}

lem_status lem_get_timing(lem_ctx* ctx, double* total_ms, int64_t* launches) {
  if (!ctx || !total_ms || !launches) return fail(LEM_EINVAL, "NULL argument");
  DeviceGuard g(ctx->device);
  LEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  double tot = 0.0;
  for (size_t i = 0; i + 1 < ctx->ev_used; i += 2) {
    float ms = 0.0f;
    LEM_CUDA_TRY(cudaEventElapsedTime(&ms, ctx->ev_pool[i], ctx->ev_pool[i + 1]));
    tot += ms;
  }
  *total_ms = tot;
  *launches = int64_t(ctx->ev_used / 2);
  ctx->ev_used = 0;
  return LEM_OK;
}

lem_status lem_sync(lem_ctx* ctx) {
  if (!ctx) return fail(LEM_EINVAL, "ctx is NULL");
  DeviceGuard g(ctx->device);
  LEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return split_check_error(ctx);
}

void lem_destroy(lem_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  free_ctx(ctx);
}

}  // extern "C"
