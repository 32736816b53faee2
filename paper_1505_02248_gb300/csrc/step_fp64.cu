// Plain FP64 LEM step (Sec. 3 steps 1-3, Eq. lem): the reference GPU path.
//   PHI:  r = dt F(u^n) (stencil residual, Eq. spacedisc with g = 0, plus dt(u - u^3), or the
//         stencil applied to |u|^(m-1) u for the porous-medium equation);
//         U_i = r|_{M_i} (halo gather); Y_i = P_{c(i)} U_i; u_D += Y_i (owner scatter).
//   EXP:  U_i = u^n|_{M_i}; Y_i = P_{c(i)} U_i; u_D = Y_i.
// All windows read u^n: the gather completes before any owner node is written, and
// every node has exactly one owner, so the update is in place.
#include "dgemm.cuh"
#include "lem_internal.h"

namespace lem {

namespace {

// r[p] = sum of the dt-scaled stencil around p (+ dt (u - u^3)); walls drop neighbours.
// NL (the reaction kind) 2, porous medium (Eq. porous): the stencil acts on
// phi(u) = |u|^(m-1) u.
template <int NL>
__global__ void residual_fp64_kernel(double* __restrict__ r, const double* __restrict__ u,
                                     const double* __restrict__ coef, int64_t cstride,
                                     int64_t ny, int64_t nx, int ndim, int pery, int perx,
                                     double dt, double pm) {
  const int64_t npts = ny * nx;
  for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < npts;
       p += int64_t(gridDim.x) * blockDim.x) {
    const int64_t y = p / nx, x = p % nx;
    // coefficient `w` (0..4 = C, W, E, S, N) at node p
    auto cf = [&](int w) { return cstride ? coef[int64_t(w) * npts + p] : coef[w]; };
    auto val = [&](int64_t q) {
      const double v = u[q];
      if constexpr (NL == 2) return pow(fabs(v), pm - 1.0) * v;
      return v;
    };
    const double uc = u[p];
    double acc = cf(0) * val(p);
    if (x > 0) acc = fma(cf(1), val(p - 1), acc);
    else if (perx) acc = fma(cf(1), val(p + nx - 1), acc);
    if (x + 1 < nx) acc = fma(cf(2), val(p + 1), acc);
    else if (perx) acc = fma(cf(2), val(p + 1 - nx), acc);
    if (ndim == 2) {
      if (y > 0) acc = fma(cf(3), val(p - nx), acc);
      else if (pery) acc = fma(cf(3), val(p + (ny - 1) * nx), acc);
      if (y + 1 < ny) acc = fma(cf(4), val(p + nx), acc);
      else if (pery) acc = fma(cf(4), val(p - (ny - 1) * nx), acc);
    }
    if constexpr (NL == 1) acc = fma(dt, uc - uc * uc * uc, acc);
    r[p] = acc;
  }
}

// Complex problems: r = X u with interleaved (re, im) states; coefficient w's real part at
// coef[w], its imaginary part at coef[5 + w] (per node when cstride).
__global__ void residual_complex_kernel(double* __restrict__ r, const double* __restrict__ u,
                                        const double* __restrict__ coef, int64_t cstride, int64_t ny, int64_t nx,
                                        int ndim, int pery, int perx) {
  const int64_t npts = ny * nx;
  for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < npts;
       p += int64_t(gridDim.x) * blockDim.x) {
    const int64_t y = p / nx, x = p % nx;
    double ar = 0.0, ai = 0.0;
    auto mac = [&](int w, int64_t q) {
      const double a = cstride ? coef[int64_t(w) * npts + p] : coef[w];
      const double b = cstride ? coef[int64_t(5 + w) * npts + p] : coef[5 + w];
      const double xr = u[2 * q], xi = u[2 * q + 1];
      ar = fma(a, xr, fma(-b, xi, ar));
      ai = fma(a, xi, fma(b, xr, ai));
    };
    mac(0, p);
    if (x > 0) mac(1, p - 1);
    else if (perx) mac(1, p + nx - 1);
    if (x + 1 < nx) mac(2, p + 1);
    else if (perx) mac(2, p + 1 - nx);
    if (ndim == 2) {
      if (y > 0) mac(3, p - nx);
      else if (pery) mac(3, p + (ny - 1) * nx);
      if (y + 1 < ny) mac(4, p + nx);
      else if (pery) mac(4, p - (ny - 1) * nx);
    }
    r[2 * p] = ar;
    r[2 * p + 1] = ai;
  }
}

// U[t][k] = src(window node k of tile t), zero beyond the window (padding)
__global__ void gather_fp64_kernel(double* __restrict__ U, const double* __restrict__ src,
                                   const TileDesc* __restrict__ tiles, int64_t n_loc, int64_t ny,
                                   int64_t nx) {
  const int t = blockIdx.y;
  const TileDesc td = tiles[t];
  const int wl = td.wext[0] * td.wext[1];
  for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n_loc;
       k += int64_t(gridDim.x) * blockDim.x) {
    double v = 0.0;
    if (k < wl) {
      const int a = int(k / td.wext[1]), b = int(k % td.wext[1]);
      int64_t gy = (int64_t(td.org[0]) + a) % ny;
      if (gy < 0) gy += ny;
      int64_t gx = (int64_t(td.org[1]) + b) % nx;
      if (gx < 0) gx += nx;
      v = src[gy * nx + gx];
    }
    U[int64_t(t) * n_loc + k] = v;
  }
}

// owner scatter: u[node(i)] = (accumulate ? u : 0) + Y[t][i]
__global__ void scatter_fp64_kernel(double* __restrict__ u, const double* __restrict__ Y,
                                    const TileDesc* __restrict__ tiles, int64_t n_int, int64_t nx,
                                    int accumulate) {
  const int t = blockIdx.y;
  const TileDesc td = tiles[t];
  const int ie = td.iext[0] * td.iext[1];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ie; i += gridDim.x * blockDim.x) {
    const int64_t p = int64_t(td.t0[0] + i / td.iext[1]) * nx + td.t0[1] + i % td.iext[1];
    const double y = Y[int64_t(t) * n_int + i];
    u[p] = accumulate ? u[p] + y : y;
  }
}

}  // namespace

cudaError_t launch_residual_fp64(const lem_ctx* ctx, double* r, const double* u) {
  const lem_problem_desc& d = ctx->desc;
  int blocks = int(std::min<int64_t>((ctx->npts + 255) / 256, 152 * 16));
  if (ctx->cplx) {
    residual_complex_kernel<<<blocks, 256, 0, ctx->stream>>>(r, u, ctx->d_coef, d.coef_stride, ctx->ny, ctx->nx,
                                                             d.ndim, ctx->bcy == LEM_BC_PERIODIC,
                                                             ctx->bcx == LEM_BC_PERIODIC);
    return cudaGetLastError();
  }
  const int py = ctx->bcy == LEM_BC_PERIODIC, px = ctx->bcx == LEM_BC_PERIODIC;
  if (d.reaction == 2)
    residual_fp64_kernel<2><<<blocks, 256, 0, ctx->stream>>>(r, u, ctx->d_coef, d.coef_stride, ctx->ny, ctx->nx,
                                                             d.ndim, py, px, d.dt, d.porous_m);
  else if (d.reaction == 1)
    residual_fp64_kernel<1><<<blocks, 256, 0, ctx->stream>>>(r, u, ctx->d_coef, d.coef_stride, ctx->ny, ctx->nx,
                                                             d.ndim, py, px, d.dt, d.porous_m);
  else
    residual_fp64_kernel<0><<<blocks, 256, 0, ctx->stream>>>(r, u, ctx->d_coef, d.coef_stride, ctx->ny, ctx->nx,
                                                             d.ndim, py, px, d.dt, d.porous_m);
  return cudaGetLastError();
}

lem_status step_fp64(lem_ctx* ctx, double* d_u) {
  cudaStream_t st = ctx->stream;
  const int64_t nt = int64_t(ctx->tiles.size());
  if (!ctx->d_U) {
    LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->d_U), sizeof(double) * nt * ctx->n_loc));
    LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->d_Y), sizeof(double) * nt * ctx->n_int));
  }
  const bool phi = ctx->desc.mode == LEM_MODE_PHI;
  const double* src = d_u;
  if (phi) {
    LEM_CUDA_TRY(launch_residual_fp64(ctx, ctx->d_r, d_u));
    src = ctx->d_r;
  }
  {
    int bx = int(std::min<int64_t>((ctx->n_loc + 255) / 256, 64));
    gather_fp64_kernel<<<dim3(bx, unsigned(nt)), 256, 0, st>>>(ctx->d_U, src, ctx->d_tiles,
                                                               ctx->n_loc, ctx->ny, ctx->nx);
    LEM_CUDA_TRY(cudaGetLastError());
  }
  // Y[tiles of class c] = U[tiles of class c] * P_c^T   (one gathered GEMM per class)
  cudaEvent_t stop;
  LEM_CUDA_TRY(ctx->timing_begin(&stop));
  const int64_t nc = int64_t(ctx->classes.size());
  for (int64_t c = 0; c < nc; ++c) {
    const int off = ctx->class_offset[c], cnt = ctx->class_offset[c + 1] - off;
    if (cnt == 0) continue;
    DgemmArgs g{};
    g.M = cnt; g.N = int(ctx->n_int); g.K = int(ctx->n_loc);
    g.A = ctx->d_U; g.lda = ctx->n_loc; g.sA = 0;
    g.B = ctx->d_P + c * ctx->n_int * ctx->n_loc; g.ldb = ctx->n_loc; g.sB = 0; g.transB = 1;
    g.C = ctx->d_Y; g.ldc = ctx->n_int; g.sC = 0;
    g.alpha = 1.0; g.beta = 0.0;
    g.rowidx = ctx->d_class_order + off;
    LEM_CUDA_TRY(dgemm(g, 1, st));
  }
  ctx->timing_end(stop);
  {
    int bx = int(std::min<int64_t>((ctx->n_int + 255) / 256, 64));
    scatter_fp64_kernel<<<dim3(bx, unsigned(nt)), 256, 0, st>>>(d_u, ctx->d_Y, ctx->d_tiles,
                                                                ctx->n_int, ctx->nx, phi ? 1 : 0);
    LEM_CUDA_TRY(cudaGetLastError());
  }
  return LEM_OK;
}

}  // namespace lem

namespace lem {

// One FP64 LEM step with caller-provided scratch: r (npts), U (ntiles x n_loc) and
// Y (ntiles x n_int). Used by the allocation-free entry point; it launches the same
// kernels as step_fp64 and writes every scratch element it later reads.
lem_status step_fp64_scratch(lem_ctx* ctx, double* d_u, double* r, double* U, double* Y) {
  cudaStream_t st = ctx->stream;
  const int64_t nt = int64_t(ctx->tiles.size());
  const bool phi = ctx->desc.mode == LEM_MODE_PHI;
  const double* src = d_u;
  if (phi) {
    LEM_CUDA_TRY(launch_residual_fp64(ctx, r, d_u));
    src = r;
  }
  int bx = int(std::min<int64_t>((ctx->n_loc + 255) / 256, 64));
  gather_fp64_kernel<<<dim3(bx, unsigned(nt)), 256, 0, st>>>(U, src, ctx->d_tiles, ctx->n_loc, ctx->ny, ctx->nx);
  LEM_CUDA_TRY(cudaGetLastError());
  const int64_t nc = int64_t(ctx->classes.size());
  for (int64_t c = 0; c < nc; ++c) {
    const int off = ctx->class_offset[c], cnt = ctx->class_offset[c + 1] - off;
    if (cnt == 0) continue;
    DgemmArgs g{};
    g.M = cnt; g.N = int(ctx->n_int); g.K = int(ctx->n_loc);
    g.A = U; g.lda = ctx->n_loc; g.sA = 0;
    g.B = ctx->d_P + c * ctx->n_int * ctx->n_loc; g.ldb = ctx->n_loc; g.sB = 0; g.transB = 1;
    g.C = Y; g.ldc = ctx->n_int; g.sC = 0;
    g.alpha = 1.0; g.beta = 0.0;
    g.rowidx = ctx->d_class_order + off;
    LEM_CUDA_TRY(dgemm(g, 1, st));
  }
  bx = int(std::min<int64_t>((ctx->n_int + 255) / 256, 64));
  scatter_fp64_kernel<<<dim3(bx, unsigned(nt)), 256, 0, st>>>(d_u, Y, ctx->d_tiles, ctx->n_int, ctx->nx, phi ? 1 : 0);
  LEM_CUDA_TRY(cudaGetLastError());
  return LEM_OK;
}

}  // namespace lem
