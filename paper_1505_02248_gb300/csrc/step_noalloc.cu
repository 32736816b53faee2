// Allocation-free FP64 LEM step (lem_step_fp64_noalloc).
//
// Some callers cannot call cudaMalloc while they advance a state: runtimes that hand all
// device memory to their own pool at start-up and forbid later driver allocations, and
// latency-critical loops that cannot afford cudaMalloc's implicit device synchronisation.
// For them this entry point takes its per-step scratch (the residual, and on the GEMM path
// the gathered windows and local results) from a fixed array in the library's static device
// memory instead of allocating it. The array exists on every GPU that loads the library,
// until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "lem_internal.h"

namespace lem {
lem_status step_fp64_scratch(lem_ctx* ctx, double* d_u, double* r, double* U, double* Y);
lem_status step_gemv_scratch(lem_ctx* ctx, double* d_u, double* r);
}

namespace {

// 8 MiB of FP64 scratch, shared by every call of lem_step_fp64_noalloc on a device.
constexpr size_t kScratchDoubles = size_t(1) << 20;
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once per device).
// In host code g_noalloc_scratch names a host-side shadow, not device memory, so the
// kernels get the address that cudaGetSymbolAddress returns for the current device. The
// address is kept for the life of the process: a device reset (cudaDeviceReset) unloads the
// module and makes it stale, so this entry point must not be used after one.
lem_status scratch_address(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return lem::fail(LEM_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return lem::cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_scratch_ptr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[device];
  return LEM_OK;
}

inline int64_t round_up(int64_t n, int64_t m) { return (n + m - 1) / m * m; }

}  // namespace

extern "C" lem_status lem_step_fp64_noalloc(lem_ctx* ctx, double* d_state, int nsteps) {
  if (!ctx) return lem::fail(LEM_EINVAL, "ctx is NULL");
  if (!d_state) return lem::fail(LEM_EINVAL, "state is NULL");
  if (nsteps < 0) return lem::fail(LEM_EINVAL, "nsteps < 0");
  if (ctx->desc.prec != LEM_PREC_FP64) return lem::fail(LEM_EINVAL, "lem_step_fp64_noalloc needs an LEM_PREC_FP64 context");
  if (ctx->cplx || ctx->desc.scheme != LEM_SCHEME_EULER)
    return lem::fail(LEM_EINVAL, "lem_step_fp64_noalloc covers real problems with the exponential Euler scheme");
  if (!ctx->built) return lem::fail(LEM_ENOTREADY, "build the propagators (lem_build_propagators) before the allocation-free step");
  if (ctx->desc.reaction && ctx->desc.refresh > 0)
    return lem::fail(LEM_EINVAL, "Jacobian refreshes rebuild propagators, which allocates; use refresh = 0");
  if (ctx->desc.reaction == 2)
    return lem::fail(LEM_EINVAL, "lem_step_fp64_noalloc does not take the porous-medium problem");
  if (ctx->band_tol >= 0.0)
    return lem::fail(LEM_EINVAL, "lem_step_fp64_noalloc does not take truncated propagators (use lem_step)");
  // scratch layout: r | U | Y, each start 256-byte aligned. The batched GEMV (contexts with
  // many propagator classes) reads the windows straight from r and needs r alone.
  const bool gemv = ctx->apply_path == LEM_APPLY_FP64_GEMV;
  const int64_t nt = int64_t(ctx->tiles.size());
  const int64_t n_r = round_up(ctx->npts, 32);
  const int64_t n_U = gemv ? 0 : round_up(nt * ctx->n_loc, 32);
  const int64_t n_Y = gemv ? 0 : round_up(nt * ctx->n_int, 32);
  const int64_t need = n_r + n_U + n_Y;
  if (need > int64_t(kScratchDoubles))
    return lem::fail(LEM_EINVAL, "problem needs " + std::to_string(need * 8) + " bytes of step scratch; " +
                                     "lem_step_fp64_noalloc is limited to " + std::to_string(kScratchDoubles * 8) +
                                     " bytes (use lem_step)");
  if (nsteps == 0) return LEM_OK;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (prev != ctx->device) {
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return lem::cuda_fail(e, "cudaSetDevice");
  }
  double* base = nullptr;
  lem_status s = scratch_address(ctx->device, &base);
  for (int k = 0; s == LEM_OK && k < nsteps; ++k)
    s = gemv ? lem::step_gemv_scratch(ctx, d_state, base)
             : lem::step_fp64_scratch(ctx, d_state, base, base + n_r, base + n_r + n_U);
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  return s;
}
