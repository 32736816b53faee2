// Per-tile propagator application (Sec. 3 steps 1-3, Eq. lem) as one batched GEMV launch:
// one CTA per owner tile gathers the tile's window of the residual (or of the state in EXP
// mode) into shared memory, its warps stream the rows of the tile's propagator, and every
// row's result is written straight into its owner node (u_D += y, or u_D = y in EXP mode).
// The launch is bound by the propagator bytes in HBM (n_int x n_loc per tile), so the
// reduced-precision variant stores propagators in FP32 (half the bytes) and accumulates the
// products in float-float; the FP64 variant is the plain reference arithmetic.
//
// Jacobi update: all tiles must read u^n, so in EXP mode the source is a copy of u^n and in
// PHI mode the residual array (computed from u^n before this launch).
#include "lem_internal.h"

namespace lem {

namespace {

__device__ __forceinline__ void two_sum_d(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

template <typename PT>
__global__ void __launch_bounds__(256) gemv_tiles_kernel(const PT* __restrict__ P, int64_t n_int, int64_t n_loc,
                                                         const TileDesc* __restrict__ tiles,
                                                         const double* __restrict__ src, double* __restrict__ u,
                                                         int64_t ny, int64_t nx, int accumulate) {
  extern __shared__ double w[];  // n_loc window values
  const int t = blockIdx.x;
  const TileDesc td = tiles[t];
  const int wl = td.wext[0] * td.wext[1];
  for (int k = threadIdx.x; k < wl; k += blockDim.x) {
    const int a = k / td.wext[1], b = k % td.wext[1];
    int64_t gy = int64_t(td.org[0]) + a, gx = int64_t(td.org[1]) + b;
    gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
    gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
    w[k] = src[gy * nx + gx];
  }
  __syncthreads();
  const PT* Pt = P + int64_t(td.cls) * n_int * n_loc;
  const int ie = td.iext[0] * td.iext[1];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  for (int i = warp; i < ie; i += nw) {
    const PT* row = Pt + int64_t(i) * n_loc;
    double y;
    if constexpr (sizeof(PT) == 8) {
      double acc = 0.0;
      for (int k = lane; k < wl; k += 32) acc = fma(row[k], w[k], acc);
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      y = acc;
    } else {
      // float-float accumulation of float products: each product is split exactly (FMA)
      float hi = 0.0f, lo = 0.0f;
      for (int k = lane; k < wl; k += 32) {
        const float a = row[k];
        const float b = float(w[k]);
        const float p = __fmul_rn(a, b);
        const float pe = fmaf(a, b, -p);
        float s, e;
        two_sum_d(hi, p, s, e);
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(e, pe));
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
        const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
        float s, e;
        two_sum_d(hi, oh, s, e);
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(ol, e));
      }
      y = double(hi) + double(lo);
    }
    if (lane == 0) {
      const int64_t p = int64_t(td.t0[0] + i / td.iext[1]) * nx + td.t0[1] + i % td.iext[1];
      u[p] = accumulate ? u[p] + y : y;
    }
  }
}

__global__ void f64_to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    b[i] = __double2float_rn(a[i]);
}

}  // namespace

cudaError_t launch_residual_fp64(const lem_ctx* ctx, double* r, const double* u);

// FP32 copy of the propagators for the reduced-precision GEMV (refreshed after each build).
lem_status gemv_prepare_f32(lem_ctx* ctx) {
  const int64_t n = int64_t(ctx->classes.size()) * ctx->n_int * ctx->n_loc;
  if (!ctx->d_P32) LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->d_P32), sizeof(float) * n));
  f64_to_f32_kernel<<<1024, 256, 0, ctx->stream>>>(ctx->d_P, ctx->d_P32, n);
  LEM_CUDA_TRY(cudaGetLastError());
  ctx->p32_gen = ctx->build_gen;
  return LEM_OK;
}

// One LEM step by the batched GEMV: PHI reads the residual, EXP a copy of u^n.
lem_status step_gemv(lem_ctx* ctx, double* d_u, bool f32) {
  cudaStream_t st = ctx->stream;
  const bool phi = ctx->desc.mode == LEM_MODE_PHI;
  const double* src;
  if (phi) {
    LEM_CUDA_TRY(launch_residual_fp64(ctx, ctx->d_r, d_u));
    src = ctx->d_r;
  } else {
    LEM_CUDA_TRY(cudaMemcpyAsync(ctx->d_r, d_u, sizeof(double) * ctx->npts, cudaMemcpyDeviceToDevice, st));
    src = ctx->d_r;
  }
  if (f32 && ctx->p32_gen != ctx->build_gen) LEM_TRY(gemv_prepare_f32(ctx));
  const size_t smem = sizeof(double) * size_t(ctx->n_loc);
  const unsigned nt = unsigned(ctx->tiles.size());
  cudaEvent_t stop;
  LEM_CUDA_TRY(ctx->timing_begin(&stop));
  if (f32)
    gemv_tiles_kernel<float><<<nt, 256, smem, st>>>(ctx->d_P32, ctx->n_int, ctx->n_loc, ctx->d_tiles, src, d_u,
                                                    ctx->ny, ctx->nx, phi ? 1 : 0);
  else
    gemv_tiles_kernel<double><<<nt, 256, smem, st>>>(ctx->d_P, ctx->n_int, ctx->n_loc, ctx->d_tiles, src, d_u,
                                                     ctx->ny, ctx->nx, phi ? 1 : 0);
  ctx->timing_end(stop);
  LEM_CUDA_TRY(cudaGetLastError());
  return LEM_OK;
}

lem_status gemv_set_smem(lem_ctx* ctx) {
  const int bytes = int(sizeof(double) * ctx->n_loc);
  if (bytes > 48 * 1024) {
    LEM_CUDA_TRY(cudaFuncSetAttribute(gemv_tiles_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    LEM_CUDA_TRY(cudaFuncSetAttribute(gemv_tiles_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  }
  return LEM_OK;
}

}  // namespace lem
