// Per-tile propagator application (Sec. 3 steps 1-3, Eq. lem) as one batched GEMV launch:
// one CTA per owner tile gathers the tile's window of the residual (or of the state in EXP
// mode) into shared memory, its warps stream the rows of the tile's propagator, and every
// row's result is written straight into its owner node (u_D += y, or u_D = y in EXP mode).
// The launch is bound by the propagator bytes in HBM (n_int x n_loc per tile), so the
// reduced-precision variant stores propagators in FP32 (half the bytes) and accumulates the
// products in float-float (complex rows: per-chunk FMA sums); the FP64 variant is the plain
// reference arithmetic.
//
// Jacobi update: all tiles must read u^n, so in EXP mode the source is a copy of u^n and in
// PHI mode the residual array (computed from u^n before this launch).
#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include <cooperative_groups.h>

#include "lem_internal.h"

namespace lem {

namespace {

__device__ __forceinline__ void two_sum_d(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Per-lane accumulators. FP64 rows: fused multiply-add. FP32 rows: each product split exactly
// (FMA) and accumulated in float-float.
struct AccD {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
};
struct AccF {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = fmaf(a, b, -p);
    float s, e;
    two_sum_d(hi, p, s, e);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, pe));
  }
  // adds a partial sum already rounded to FP32
  __device__ __forceinline__ void add1(float x) {
    float s, e;
    two_sum_d(hi, x, s, e);
    hi = s;
    lo = __fadd_rn(lo, e);
  }
};

// Reduction over the 8 lanes of a row group (lanes 8g .. 8g + 7).
__device__ __forceinline__ double group_reduce(AccD& a) {
  for (int o = 4; o > 0; o >>= 1) a.s += __shfl_xor_sync(0xffffffffu, a.s, o);
  return a.s;
}
__device__ __forceinline__ double group_reduce(AccF& a) {
  for (int o = 4; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, a.hi, o);
    const float ol = __shfl_xor_sync(0xffffffffu, a.lo, o);
    float s, e;
    two_sum_d(a.hi, oh, s, e);
    a.hi = s;
    a.lo = __fadd_rn(a.lo, __fadd_rn(ol, e));
  }
  return double(a.hi) + double(a.lo);
}

// Four propagator rows per warp, 8 lanes per row: y_i = sum_k P[i, k] w[k]. With vec (row
// length a multiple of the vector width, rows 16-byte aligned) each lane streams its row in
// 16-byte loads, four in flight; else scalar loads. Several rows in flight per warp keep the
// load pipe busy through each row's reduction and owner update.
// CPLX: complex states (interleaved re, im) with real-embedded propagators
// [[Re P, -Im P], [Im P, Re P]]: the window is staged as [re parts | im parts] (n_loc / 2 nodes
// each, zero padded); each owner's Re and Im rows are read once, left halves only.
template <typename PT, bool CPLX>
__global__ void __launch_bounds__(256) gemv_tiles_kernel(const PT* __restrict__ P, int64_t n_int, int64_t n_loc,
                                                         const TileDesc* __restrict__ tiles,
                                                         const double* __restrict__ src, double* __restrict__ u,
                                                         int64_t ny, int64_t nx, int accumulate, int rsplit) {
  // the tile's window values, converted once to the propagator's precision
  extern __shared__ __align__(16) unsigned char wraw[];
  PT* w = reinterpret_cast<PT*>(wraw);
  // rsplit blocks share a tile, each taking a contiguous share of its owner rows: several
  // waves of short blocks instead of one wave of long ones (a shorter tail)
  const int t = blockIdx.x / rsplit, part = blockIdx.x % rsplit;
  const TileDesc td = tiles[t];
  const int wn = td.wext[0] * td.wext[1];  // window nodes
  const int hn = int(n_loc / 2);            // CPLX: padded window nodes
  const int wl = CPLX ? int(n_loc) : wn;    // staged window values
  for (int k = threadIdx.x; k < wl; k += blockDim.x) {
    const int node = CPLX ? k % hn : k, comp = CPLX ? k / hn : 0;
    if (node >= wn) {
      w[k] = PT(0);
      continue;
    }
    const int a = node / td.wext[1], b = node % td.wext[1];
    int64_t gy = int64_t(td.org[0]) + a, gx = int64_t(td.org[1]) + b;
    gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
    gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
    w[k] = PT(CPLX ? src[2 * (gy * nx + gx) + comp] : src[gy * nx + gx]);
  }
  __syncthreads();
  const PT* Pt = P + int64_t(td.cls) * n_int * n_loc;
  const int ien = td.iext[0] * td.iext[1];  // owner nodes
  const int ie_all = ien;                   // owner nodes of this tile (CPLX: one group does both parts)
  const int rows_per = (ie_all + rsplit - 1) / rsplit;
  const int ib = part * rows_per, ie = min(ie_all, ib + rows_per);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  const int grp = lane / 8, gl = lane % 8;
  constexpr int V = 16 / sizeof(PT);
  constexpr int U = 4;  // 16-byte loads in flight per lane
  const bool vec = (n_loc % V) == 0 && (wl % V) == 0;
  using Acc = typename std::conditional<sizeof(PT) == 8, AccD, AccF>::type;
  if constexpr (CPLX) {
    // complex: a row group per owner node o, reading its Re row (row o) and Im row (row
    // n_int / 2 + o) of the stored embedding, left halves only (the right halves repeat them):
    //   y_re = Re w_re - Im w_im,   y_im = Im w_re + Re w_im
    const int hl = hn;  // window columns per part
    const bool cvec = (n_loc % V) == 0 && (hl % V) == 0;
    for (int o0 = ib + warp * 4; o0 < ie; o0 += nw * 4) {
      const int o = o0 + grp;
      const bool live = o < ie;
      const PT* rre = Pt + int64_t(live ? o : 0) * n_loc;
      const PT* rim = Pt + int64_t(live ? int(n_int / 2) + o : 0) * n_loc;
      Acc are, aim;
      if (cvec) {
        // FP32 rows: four 16-byte loads per lane and row in flight, so a window of up to 128
        // nodes takes one round trip per row pair; FP64 rows are bound by the FP64 pipe.
        constexpr int CU = sizeof(PT) == 4 ? 4 : 2;
        const int nv = hl / V;
        const int4* a4 = reinterpret_cast<const int4*>(rre);
        const int4* b4 = reinterpret_cast<const int4*>(rim);
        for (int j = gl; j < nv; j += 8 * CU) {
          int4 qa[CU], qb[CU];
#pragma unroll
          for (int k = 0; k < CU; ++k) {
            const bool ok = live && j + 8 * k < nv;
            qa[k] = ok ? __ldcs(a4 + j + 8 * k) : make_int4(0, 0, 0, 0);
            qb[k] = ok ? __ldcs(b4 + j + 8 * k) : make_int4(0, 0, 0, 0);
          }
#pragma unroll
          for (int k = 0; k < CU; ++k) {
            if (j + 8 * k >= nv) break;
            const PT* pa = reinterpret_cast<const PT*>(&qa[k]);
            const PT* pb = reinterpret_cast<const PT*>(&qb[k]);
            const int4 wr4 = *reinterpret_cast<const int4*>(w + (j + 8 * k) * V);
            const int4 wi4 = *reinterpret_cast<const int4*>(w + hl + (j + 8 * k) * V);
            const PT* wr = reinterpret_cast<const PT*>(&wr4);
            const PT* wi = reinterpret_cast<const PT*>(&wi4);
            if constexpr (sizeof(PT) == 4) {
              // FP32 rows: a chunk's eight products per part are summed by FMA in FP32 and the
              // chunk sum enters the float-float accumulator (an exact product split for each of
              // the four products an element takes part in would make the launch ALU-bound)
              float sr = 0.0f, si = 0.0f;
#pragma unroll
              for (int h = 0; h < V; ++h) {
                sr = fmaf(pa[h], wr[h], sr);
                sr = fmaf(-pb[h], wi[h], sr);
                si = fmaf(pb[h], wr[h], si);
                si = fmaf(pa[h], wi[h], si);
              }
              are.add1(sr);
              aim.add1(si);
            } else {
#pragma unroll
              for (int h = 0; h < V; ++h) {
                are.add(pa[h], wr[h]);
                are.add(-pb[h], wi[h]);
                aim.add(pb[h], wr[h]);
                aim.add(pa[h], wi[h]);
              }
            }
          }
        }
      } else if (live) {
        for (int k = gl; k < hl; k += 8) {
          are.add(rre[k], w[k]);
          are.add(-rim[k], w[hl + k]);
          aim.add(rim[k], w[k]);
          aim.add(rre[k], w[hl + k]);
        }
      }
      const double yr = group_reduce(are), yi = group_reduce(aim);
      if (live && gl == 0) {
        const int64_t p = int64_t(td.t0[0] + o / td.iext[1]) * nx + td.t0[1] + o % td.iext[1];
        u[2 * p] = accumulate ? u[2 * p] + yr : yr;
        u[2 * p + 1] = accumulate ? u[2 * p + 1] + yi : yi;
      }
    }
  } else {
    // every lane runs the same number of row iterations (the shuffles need the whole warp)
    for (int i0 = ib + warp * 4; i0 < ie; i0 += nw * 4) {
      const int i = i0 + grp;
      const bool live = i < ie;
      const PT* row = Pt + int64_t(live ? i : 0) * n_loc;
      Acc acc;
      if (vec) {
        const int nv = wl / V;
        const int4* r4 = reinterpret_cast<const int4*>(row);
        for (int j = gl; j < nv; j += 8 * U) {
          int4 q[U];
  #pragma unroll
          for (int k = 0; k < U; ++k) q[k] = (live && j + 8 * k < nv) ? __ldcs(r4 + j + 8 * k) : make_int4(0, 0, 0, 0);
  #pragma unroll
          for (int k = 0; k < U; ++k) {
            if (j + 8 * k >= nv) break;
            const PT* pq = reinterpret_cast<const PT*>(&q[k]);
            const int4 wq = *reinterpret_cast<const int4*>(w + (j + 8 * k) * V);  // same 16 bytes of w
            const PT* pw = reinterpret_cast<const PT*>(&wq);
  #pragma unroll
            for (int h = 0; h < V; ++h) acc.add(pq[h], pw[h]);
          }
        }
      } else if (live) {
        for (int k = gl; k < wl; k += 8) acc.add(row[k], w[k]);
      }
      const double y = group_reduce(acc);
      if (live && gl == 0) {
        const int64_t p = int64_t(td.t0[0] + i / td.iext[1]) * nx + td.t0[1] + i % td.iext[1];
        u[p] = accumulate ? u[p] + y : y;
      }
    }
  }
}


// The defect of the third-order Rosenbrock step, times two: 2 dt (G(U) - G(u)) with
// G(v) = F(v) - J(u_m) v. The linear parts cancel, so it is pointwise:
// 2 dt [(U - U^3) - (u - u^3) - (1 - 3 u_m^2)(U - u)].
__global__ void rb3_defect_kernel(const double* __restrict__ U, const double* __restrict__ u,
                                  const double* __restrict__ um, double dt, double* __restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double Ui = U[i], ui = u[i], mi = um[i];
    d[i] = 2.0 * dt * ((Ui - Ui * Ui * Ui) - (ui - ui * ui * ui) - (1.0 - 3.0 * mi * mi) * (Ui - ui));
  }
}

__global__ void f64_to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    b[i] = __double2float_rn(a[i]);
}

}  // namespace


// FP32 copy of the propagators for the reduced-precision GEMV (refreshed after each build).
lem_status gemv_prepare_f32(lem_ctx* ctx) {
  const int64_t n = int64_t(ctx->classes.size()) * ctx->n_int * ctx->n_loc;
  if (!ctx->d_P32) LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->d_P32), sizeof(float) * n));
  f64_to_f32_kernel<<<1024, 256, 0, ctx->stream>>>(ctx->d_P, ctx->d_P32, n);
  if (ctx->d_P3) {
    if (!ctx->d_P3_32) LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->d_P3_32), sizeof(float) * n));
    f64_to_f32_kernel<<<1024, 256, 0, ctx->stream>>>(ctx->d_P3, ctx->d_P3_32, n);
  }
  LEM_CUDA_TRY(cudaGetLastError());
  ctx->p32_gen = ctx->build_gen;
  return LEM_OK;
}

// ---------------------------------------------------------------- persistent multi-step
// Small problems (config 1: 16 tiles of a 1024-node mesh) are bound by launch latency, two
// launches per step. This cooperative kernel runs all nsteps in one launch. Per step every
// block takes its tiles: it forms the window's source straight from u^n (the residual dt A u^n
// at each window node in PHI mode, u^n in EXP mode) in shared memory, applies the tile's
// propagator (four rows per warp) and writes the owner values of u^{n+1} into the other state
// buffer; one grid barrier ends the step. Linear real problems on the GEMV path only (no
// Jacobian refresh, one scheme stage).
// SMEMP: one tile per block, its propagator kept in shared memory for all steps.
template <typename PT, bool SMEMP>
__global__ void __launch_bounds__(256) gemv_persistent_kernel(const PT* __restrict__ P, int64_t n_int, int64_t n_loc,
                                                              const TileDesc* __restrict__ tiles, int ntiles,
                                                              const double* __restrict__ coef, int64_t cstride,
                                                              int64_t ny, int64_t nx, int ndim, int pery, int perx,
                                                              int phi, double* __restrict__ src,
                                                              double* __restrict__ u, int nsteps) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char wraw[];
  PT* w = reinterpret_cast<PT*>(wraw);
  const int64_t npts = ny * nx;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  const int grp = lane / 8, gl = lane % 8;
  using Acc = typename std::conditional<sizeof(PT) == 8, AccD, AccF>::type;
  // SMEMP: the block's tile propagator (n_int x n_loc) after the window buffer
  PT* Ps = reinterpret_cast<PT*>(wraw + ((sizeof(double) * size_t(n_loc) + 15) & ~size_t(15)));
  if (SMEMP) {
    const PT* src_p = P + int64_t(tiles[blockIdx.x].cls) * n_int * n_loc;
    for (int64_t e = threadIdx.x; e < n_int * n_loc; e += blockDim.x) Ps[e] = src_p[e];
    __syncthreads();
  }
  // u^n and u^{n+1} alternate between u and src (every node has exactly one owner tile, so
  // each step writes the whole of the other buffer); one grid barrier per step
  double* cur = u;
  double* nxt = src;
  for (int step = 0; step < nsteps; ++step) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const TileDesc td = tiles[t];
      const int wl = td.wext[0] * td.wext[1];
      // the window's source from u^n: the residual dt A u^n at each window node (PHI), or u^n
      for (int k = threadIdx.x; k < wl; k += blockDim.x) {
        const int a = k / td.wext[1], b = k % td.wext[1];
        int64_t gy = int64_t(td.org[0]) + a, gx = int64_t(td.org[1]) + b;
        gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
        gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
        const int64_t p = gy * nx + gx;
        double v = cur[p];
        if (phi) {
          auto cf = [&](int c) { return cstride ? coef[int64_t(c) * npts + p] : coef[c]; };
          double acc = cf(0) * v;
          if (gx > 0) acc = fma(cf(1), cur[p - 1], acc);
          else if (perx) acc = fma(cf(1), cur[p + nx - 1], acc);
          if (gx + 1 < nx) acc = fma(cf(2), cur[p + 1], acc);
          else if (perx) acc = fma(cf(2), cur[p + 1 - nx], acc);
          if (ndim == 2) {
            if (gy > 0) acc = fma(cf(3), cur[p - nx], acc);
            else if (pery) acc = fma(cf(3), cur[p + (ny - 1) * nx], acc);
            if (gy + 1 < ny) acc = fma(cf(4), cur[p + nx], acc);
            else if (pery) acc = fma(cf(4), cur[p - (ny - 1) * nx], acc);
          }
          v = acc;
        }
        w[k] = PT(v);
      }
      __syncthreads();
      const PT* Pt = SMEMP ? Ps : P + int64_t(td.cls) * n_int * n_loc;
      const int ie = td.iext[0] * td.iext[1];
      constexpr int V = 16 / sizeof(PT);
      const bool vec = (n_loc % V) == 0 && (wl % V) == 0;
      for (int i0 = warp * 4; i0 < ie; i0 += nw * 4) {
        const int i = i0 + grp;
        const bool live = i < ie;
        const PT* row = Pt + int64_t(live ? i : 0) * n_loc;
        // the same partition of a row over the 8 lanes, and the same order, as gemv_tiles_kernel
        // (16-byte chunks j = lane, lane + 8, ... when rows allow them): bit-identical results
        Acc acc;
        if (live) {
          if (vec) {
            const int4* r4 = reinterpret_cast<const int4*>(row);
            for (int j = gl; j < wl / V; j += 8) {
              const int4 q = SMEMP ? r4[j] : __ldcs(r4 + j);
              const PT* pq = reinterpret_cast<const PT*>(&q);
#pragma unroll
              for (int h = 0; h < V; ++h) acc.add(pq[h], w[j * V + h]);
            }
          } else {
            for (int k = gl; k < wl; k += 8) acc.add(row[k], w[k]);
          }
        }
        const double y = group_reduce(acc);
        if (live && gl == 0) {
          const int64_t p = int64_t(td.t0[0] + i / td.iext[1]) * nx + td.t0[1] + i % td.iext[1];
          nxt[p] = phi ? cur[p] + y : y;
        }
      }
      __syncthreads();  // the window buffer is reused by the block's next tile
    }
    grid.sync();  // u^{n+1} complete before any block reads it
    double* tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  if (cur != u)  // an odd number of steps ended in the scratch buffer
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < npts; p += int64_t(gridDim.x) * blockDim.x)
      u[p] = cur[p];
}

// Whether lem_step may run its steps in one persistent launch, and with how many blocks.
static int persistent_blocks(lem_ctx* ctx, bool f32, int nsteps) {
  const lem_problem_desc& d = ctx->desc;
  if (nsteps < 2 || d.reaction || d.scheme != LEM_SCHEME_EULER || ctx->cplx) return 0;
  if (ctx->npts > (int64_t(1) << 20) || ctx->tiles.size() > 4096) return 0;
  if (std::getenv("LEM_NO_PERSISTENT")) return 0;  // switch for comparisons
  int dev_coop = 0, nsm = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&dev_coop, cudaDevAttrCooperativeLaunch, ctx->device) != cudaSuccess || !dev_coop ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const size_t smem = sizeof(double) * size_t(ctx->n_loc);
  cudaError_t e = f32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gemv_persistent_kernel<float, false>, 256, smem)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gemv_persistent_kernel<double, false>, 256, smem);
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  // one block per tile, within what the device holds at once
  return int(std::min<int64_t>(int64_t(per_sm) * nsm, int64_t(ctx->tiles.size())));
}

lem_status step_gemv_multi(lem_ctx* ctx, double* d_u, int nsteps, bool f32, bool* done) {
  *done = false;
  const int blocks = persistent_blocks(ctx, f32, nsteps);
  if (blocks < 1) return LEM_OK;
  if (f32 && ctx->p32_gen != ctx->build_gen) LEM_TRY(gemv_prepare_f32(ctx));
  const lem_problem_desc& d = ctx->desc;
  // one tile per block with a propagator small enough for shared memory: keep it there
  const size_t wbytes = (sizeof(double) * size_t(ctx->n_loc) + 15) & ~size_t(15);
  const size_t pbytes = (f32 ? sizeof(float) : sizeof(double)) * size_t(ctx->n_int) * size_t(ctx->n_loc);
  bool smemp = blocks == int(ctx->tiles.size()) && wbytes + pbytes <= 200 * 1024 &&
               std::getenv("LEM_NO_SMEM_P") == nullptr;
  const void* fn_s = f32 ? reinterpret_cast<const void*>(gemv_persistent_kernel<float, true>)
                         : reinterpret_cast<const void*>(gemv_persistent_kernel<double, true>);
  if (smemp) {  // every block must still be co-resident with the larger footprint
    int per_sm = 0, nsm = 0;
    if (cudaFuncSetAttribute(fn_s, cudaFuncAttributeMaxDynamicSharedMemorySize, int(wbytes + pbytes)) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn_s, 256, wbytes + pbytes) != cudaSuccess ||
        int64_t(per_sm) * nsm < blocks) {
      cudaGetLastError();
      smemp = false;
    }
  }
  const size_t smem = smemp ? wbytes + pbytes : sizeof(double) * size_t(ctx->n_loc);
  const void* fn = smemp ? fn_s
                         : (f32 ? reinterpret_cast<const void*>(gemv_persistent_kernel<float, false>)
                                : reinterpret_cast<const void*>(gemv_persistent_kernel<double, false>));
  int ntiles = int(ctx->tiles.size()), ndim = d.ndim, pery = ctx->bcy == LEM_BC_PERIODIC,
      perx = ctx->bcx == LEM_BC_PERIODIC, phi = d.mode == LEM_MODE_PHI;
  int64_t n_int = ctx->n_int, n_loc = ctx->n_loc, cstride = d.coef_stride, ny = ctx->ny, nx = ctx->nx;
  const void* P = f32 ? static_cast<const void*>(ctx->d_P32) : static_cast<const void*>(ctx->d_P);
  void* args[] = {&P, &n_int, &n_loc, &ctx->d_tiles, &ntiles, &ctx->d_coef, &cstride, &ny, &nx,
                  &ndim, &pery, &perx, &phi, &ctx->d_r, &d_u, &nsteps};
  cudaEvent_t stop;
  LEM_CUDA_TRY(ctx->timing_begin(&stop));
  LEM_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(256), args, smem, ctx->stream));
  ctx->timing_end(stop);
  *done = true;
  return LEM_OK;
}

// Threads per GEMV block: 128 for the complex FP32 kernel (short rows, little work per block,
// more blocks resident per SM), 256 otherwise.
static int gemv_threads(const lem_ctx* ctx, bool f32) { return (ctx->cplx && f32) ? 128 : 256; }

// Blocks per tile: about four waves of blocks (6 to 8 resident per SM), at least 32 owner rows
// per block, each block's share a whole number of passes (a pass: 4 rows per warp), so that no
// pass runs part empty (512^2 variable diffusion: 4 blocks of 64 rows per tile, not 5 of 52).
int gemv_row_split(const lem_ctx* ctx, int threads) {
  const int64_t nt = int64_t(ctx->tiles.size());
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || nsm < 1) nsm = 152;
  const int rmax = std::max<int>(1, int(ctx->n_int / 32));
  int rsplit = std::max(1, std::min<int>(rmax, int((4LL * 8 * nsm + nt - 1) / nt)));
  const int owners = int(ctx->cplx ? ctx->n_int / 2 : ctx->n_int), pass = threads / 8;
  const int rows = ((owners + rsplit - 1) / rsplit + pass - 1) / pass * pass;
  return std::max(1, (owners + rows - 1) / rows);
}

// One LEM step by the batched GEMV: PHI reads the residual, EXP a copy of u^n.
lem_status step_gemv(lem_ctx* ctx, double* d_u, bool f32) {
  cudaStream_t st = ctx->stream;
  const bool phi = ctx->desc.mode == LEM_MODE_PHI;
  const bool rb3 = ctx->desc.scheme == LEM_SCHEME_RB3 && ctx->desc.reaction;  // (linear: the defect is 0)
  if (rb3)
    LEM_CUDA_TRY(cudaMemcpyAsync(ctx->d_u0, d_u, sizeof(double) * ctx->npts, cudaMemcpyDeviceToDevice, st));
  const double* src;
  if (phi) {
    LEM_CUDA_TRY(launch_residual_fp64(ctx, ctx->d_r, d_u));
    src = ctx->d_r;
  } else {
    LEM_CUDA_TRY(cudaMemcpyAsync(ctx->d_r, d_u, sizeof(double) * ctx->npts * (ctx->cplx ? 2 : 1),
                                 cudaMemcpyDeviceToDevice, st));
    src = ctx->d_r;
  }
  if (f32 && ctx->p32_gen != ctx->build_gen) LEM_TRY(gemv_prepare_f32(ctx));
  const size_t smem = sizeof(double) * size_t(ctx->n_loc);
  const unsigned nt = unsigned(ctx->tiles.size());
  const int threads = gemv_threads(ctx, f32);
  const int rsplit = gemv_row_split(ctx, threads);
  cudaEvent_t stop;
  LEM_CUDA_TRY(ctx->timing_begin(&stop));
  auto gemv = [&](const double* P64, const float* P32, const double* x) {
    const int acc = phi ? 1 : 0;
    if (ctx->cplx) {
      if (f32)  // short rows, little work per block: 128 threads, more blocks resident per SM
        gemv_tiles_kernel<float, true><<<nt * rsplit, threads, smem, st>>>(P32, ctx->n_int, ctx->n_loc, ctx->d_tiles, x,
                                                                       d_u, ctx->ny, ctx->nx, acc, rsplit);
      else
        gemv_tiles_kernel<double, true><<<nt * rsplit, 256, smem, st>>>(P64, ctx->n_int, ctx->n_loc, ctx->d_tiles, x,
                                                                        d_u, ctx->ny, ctx->nx, acc, rsplit);
    } else if (f32) {
      gemv_tiles_kernel<float, false><<<nt * rsplit, 256, smem, st>>>(P32, ctx->n_int, ctx->n_loc, ctx->d_tiles, x,
                                                                      d_u, ctx->ny, ctx->nx, acc, rsplit);
    } else {
      gemv_tiles_kernel<double, false><<<nt * rsplit, 256, smem, st>>>(P64, ctx->n_int, ctx->n_loc, ctx->d_tiles, x,
                                                                       d_u, ctx->ny, ctx->nx, acc, rsplit);
    }
  };
  gemv(ctx->d_P, ctx->d_P32, src);
  if (rb3) {  // second stage: u^{n+1} = U + 2 phi_3(dt J_m) dt (G(U) - G(u^n)), window by window
    rb3_defect_kernel<<<1024, 256, 0, st>>>(d_u, ctx->d_u0, ctx->d_um, ctx->desc.dt, ctx->d_r, ctx->npts);
    gemv(ctx->d_P3, ctx->d_P3_32, ctx->d_r);
  }
  ctx->timing_end(stop);
  LEM_CUDA_TRY(cudaGetLastError());
  return LEM_OK;
}

// One FP64 GEMV step of a real exponential-Euler problem with caller-provided scratch r (npts
// doubles): the kernels and launch shape of step_gemv, so the result is the same bit for bit.
// Used by the allocation-free entry point.
lem_status step_gemv_scratch(lem_ctx* ctx, double* d_u, double* r) {
  cudaStream_t st = ctx->stream;
  if (ctx->desc.mode == LEM_MODE_PHI) {
    LEM_CUDA_TRY(launch_residual_fp64(ctx, r, d_u));
  } else {
    LEM_CUDA_TRY(cudaMemcpyAsync(r, d_u, sizeof(double) * ctx->npts, cudaMemcpyDeviceToDevice, st));
  }
  const size_t smem = sizeof(double) * size_t(ctx->n_loc);
  const unsigned nt = unsigned(ctx->tiles.size());
  const int threads = gemv_threads(ctx, false);
  const int rsplit = gemv_row_split(ctx, threads);
  const int acc = ctx->desc.mode == LEM_MODE_PHI ? 1 : 0;
  gemv_tiles_kernel<double, false><<<nt * rsplit, threads, smem, st>>>(ctx->d_P, ctx->n_int, ctx->n_loc, ctx->d_tiles,
                                                                       r, d_u, ctx->ny, ctx->nx, acc, rsplit);
  LEM_CUDA_TRY(cudaGetLastError());
  return LEM_OK;
}

lem_status gemv_set_smem(lem_ctx* ctx) {
  const int bytes = int(sizeof(double) * ctx->n_loc);
  if (bytes > 48 * 1024) {
    LEM_CUDA_TRY(cudaFuncSetAttribute(gemv_tiles_kernel<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      bytes));
    LEM_CUDA_TRY(cudaFuncSetAttribute(gemv_tiles_kernel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      bytes));
    LEM_CUDA_TRY(cudaFuncSetAttribute(gemv_tiles_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      bytes));
    LEM_CUDA_TRY(cudaFuncSetAttribute(gemv_tiles_kernel<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      bytes));
  }
  return LEM_OK;
}

}  // namespace lem
