// Truncated propagators (Sec. 2, Theorem 1: the entries of the exponential of a banded matrix
// decay faster than exponentially away from the band). Each owner row of a class's propagator
// keeps only the window nodes inside a box around its owner node, offsets -ly..hy along y and
// -lx..hx along x; every other entry is dropped. The apply then streams and multiplies box
// entries only, so the bytes and the multiply-adds per dof-step fall with the box.
//
// Three kernels:
//  1. band_extents_kernel: per class, each side's extent from a tolerance. For the side "x
//     below the owner" the dropped mass of extent e is T(e) = max_d sum_{m : ox_dm < -e} |P_dm|;
//     the extent is the smallest e with T(e) <= (tol / 4) max_d sum_m |P_dm|, so the four sides
//     together drop at most tol of the largest row mass. T comes from per-row marginals of |P|
//     over window columns (rows) and their prefix sums.
//  2. band_pack_kernel: the kept entries of each row as a dense box of BYc x BXp values
//     (BYc = min(ly + hy + 1, wy) rows, BXc = min(lx + hx + 1, wx) columns padded to a
//     multiple of 4), the box shifted inside the window where it would overhang an edge
//     (entries outside the owner's own box stay zero). A row never holds more values than
//     the window (rounded up to 4).
//  3. gemv_band_row_kernel (short rows: one thread per owner row) or gemv_band_kernel (long
//     rows: 4 or 8 lanes per row): one CTA per tile (or part of its owner rows) stages the
//     window in shared memory, the box rows stream in 16-byte loads, and each row's result
//     goes straight to its owner node.
#include <algorithm>
#include <string>
#include <type_traits>
#include <vector>

#include "lem_internal.h"

namespace lem {

namespace {

// Geometry of one class (host-uploaded) and its packed box.
struct BandClass {
  int wy, wx;        // window extents
  int iy, ix;        // owner-tile extents
  int oy, ox;        // owner-tile offset inside the window
  int ly, hy, lx, hx;  // box extents (filled in by the extents kernel on the host copy)
  int byc, bxc, bxp;   // stored box rows, used columns, padded columns
  int L;               // values per stored row: byc * bxp
  int64_t off;         // first value of the class's rows in the packed array
};

constexpr int EXT_THREADS = 256;
constexpr int EXT_WARPS = EXT_THREADS / 32;

// One block per class. Dynamic shared memory: per warp the column and row marginals of one
// row (wxm + wym doubles), their prefix sums pre[k] = sum_{j < k} and suffix sums
// suf[k] = sum_{j >= k} (each wxm + 1 or wym + 1; tails are sums, never differences, so a
// small tail keeps its relative accuracy), then the block's running maxima of the four side
// tails (2 wym + 2 wxm, as the bit patterns of non-negative doubles, which order like unsigned
// integers) and of the row mass.
__global__ void __launch_bounds__(EXT_THREADS) band_extents_kernel(const double* __restrict__ P, int64_t n_int,
                                                                  int64_t n_loc, const BandClass* __restrict__ cls,
                                                                  int wym, int wxm, double tol, int* __restrict__ ext) {
  extern __shared__ __align__(16) unsigned char sraw[];
  const BandClass c = cls[blockIdx.x];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int per_warp = 3 * (wxm + wym) + 4;
  double* mx = reinterpret_cast<double*>(sraw) + warp * per_warp;  // column marginals
  double* my = mx + wxm;                                              // row marginals
  double* px_pre = my + wym;                                          // wxm + 1 prefix sums
  double* px_suf = px_pre + wxm + 1;                                  // wxm + 1 suffix sums
  double* py_pre = px_suf + wxm + 1;                                  // wym + 1 prefix sums
  double* py_suf = py_pre + wym + 1;                                  // wym + 1 suffix sums
  unsigned long long* tmax = reinterpret_cast<unsigned long long*>(reinterpret_cast<double*>(sraw) +
                                                                   EXT_WARPS * per_warp);
  unsigned long long* tS = tmax;            // [wym] y below the owner
  unsigned long long* tN = tS + wym;        // [wym] y above
  unsigned long long* tW = tN + wym;        // [wxm] x below
  unsigned long long* tE = tW + wxm;        // [wxm] x above
  unsigned long long* smass = tE + wxm;     // [1] largest row mass
  __shared__ int cnt[4];
  for (int k = threadIdx.x; k < 2 * (wym + wxm) + 1; k += blockDim.x) tmax[k] = 0ull;
  if (threadIdx.x < 4) cnt[threadIdx.x] = 0;
  __syncthreads();
  const double* Pc = P + int64_t(blockIdx.x) * n_int * n_loc;
  const int nrows = c.iy * c.ix;
  for (int d = warp; d < nrows; d += EXT_WARPS) {
    const double* row = Pc + int64_t(d) * n_loc;
    for (int x = lane; x < c.wx; x += 32) {
      double s = 0.0;
      for (int y = 0; y < c.wy; ++y) s += fabs(row[y * c.wx + x]);
      mx[x] = s;
    }
    for (int y = lane; y < c.wy; y += 32) {
      double s = 0.0;
      for (int x = 0; x < c.wx; ++x) s += fabs(row[y * c.wx + x]);
      my[y] = s;
    }
    __syncwarp();
    if (lane == 0) {
      double a = 0.0;
      for (int x = 0; x < c.wx; ++x) {
        px_pre[x] = a;
        a += mx[x];
      }
      px_pre[c.wx] = a;
      double z = 0.0;
      px_suf[c.wx] = 0.0;
      for (int x = c.wx - 1; x >= 0; --x) {
        z += mx[x];
        px_suf[x] = z;
      }
      double b = 0.0;
      for (int y = 0; y < c.wy; ++y) {
        py_pre[y] = b;
        b += my[y];
      }
      py_pre[c.wy] = b;
      z = 0.0;
      py_suf[c.wy] = 0.0;
      for (int y = c.wy - 1; y >= 0; --y) {
        z += my[y];
        py_suf[y] = z;
      }
      atomicMax(smass, static_cast<unsigned long long>(__double_as_longlong(a)));
    }
    __syncwarp();
    const int py = c.oy + d / c.ix, pxo = c.ox + d % c.ix;
    for (int e = lane; e < c.wx; e += 32) {
      const double w = px_pre[max(0, pxo - e)];            // columns x < px - e
      const double east = px_suf[min(c.wx, pxo + e + 1)];  // columns x > px + e
      atomicMax(tW + e, static_cast<unsigned long long>(__double_as_longlong(w)));
      atomicMax(tE + e, static_cast<unsigned long long>(__double_as_longlong(east)));
    }
    for (int e = lane; e < c.wy; e += 32) {
      const double s = py_pre[max(0, py - e)];
      const double n = py_suf[min(c.wy, py + e + 1)];
      atomicMax(tS + e, static_cast<unsigned long long>(__double_as_longlong(s)));
      atomicMax(tN + e, static_cast<unsigned long long>(__double_as_longlong(n)));
    }
    __syncwarp();
  }
  __syncthreads();
  // extent = the number of e >= 0 whose tail exceeds the bar (the tails do not increase with e)
  const double bar = 0.25 * tol * __longlong_as_double(static_cast<long long>(*smass));
  for (int e = threadIdx.x; e < c.wy; e += blockDim.x) {
    if (__longlong_as_double(static_cast<long long>(tS[e])) > bar) atomicAdd(&cnt[0], 1);
    if (__longlong_as_double(static_cast<long long>(tN[e])) > bar) atomicAdd(&cnt[1], 1);
  }
  for (int e = threadIdx.x; e < c.wx; e += blockDim.x) {
    if (__longlong_as_double(static_cast<long long>(tW[e])) > bar) atomicAdd(&cnt[2], 1);
    if (__longlong_as_double(static_cast<long long>(tE[e])) > bar) atomicAdd(&cnt[3], 1);
  }
  __syncthreads();
  if (threadIdx.x < 4) ext[4 * blockIdx.x + threadIdx.x] = cnt[threadIdx.x];
}

__device__ __forceinline__ void box_origin(const BandClass& c, int d, int& py, int& px, int& y0, int& x0) {
  py = c.oy + d / c.ix;
  px = c.ox + d % c.ix;
  y0 = min(max(py - c.ly, 0), c.wy - c.byc);
  x0 = min(max(px - c.lx, 0), c.wx - c.bxc);
}

// grid (owner rows, classes): row d of class c as its stored box (FP64, and FP32 if Pb32)
__global__ void band_pack_kernel(const double* __restrict__ P, int64_t n_int, int64_t n_loc,
                                 const BandClass* __restrict__ cls, double* __restrict__ Pb,
                                 float* __restrict__ Pb32) {
  const BandClass c = cls[blockIdx.y];
  const int d = blockIdx.x;
  if (d >= c.iy * c.ix) return;
  int py, px, y0, x0;
  box_origin(c, d, py, px, y0, x0);
  const double* row = P + (int64_t(blockIdx.y) * n_int + d) * n_loc;
  const int64_t o = c.off + int64_t(d) * c.L;
  for (int k = threadIdx.x; k < c.L; k += blockDim.x) {
    const int a = k / c.bxp, j = k % c.bxp;
    const int y = y0 + a, x = x0 + j;
    const bool keep = j < c.bxc && y - py >= -c.ly && y - py <= c.hy && x - px >= -c.lx && x - px <= c.hx;
    const double v = keep ? row[y * c.wx + x] : 0.0;
    Pb[o + k] = v;
    if (Pb32) Pb32[o + k] = float(v);
  }
}

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// FP64 rows: fused multiply-add. FP32 rows: each product split exactly (FMA) and accumulated
// in float-float, as the dense FP32 GEMV does. reduce<LPR>: sum over the LPR lanes of a row.
struct BAccD {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  template <int LPR>
  __device__ __forceinline__ double reduce() {
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
  }
};
struct BAccF {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = fmaf(a, b, -p);
    float s, e;
    two_sum_f(hi, p, s, e);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, pe));
  }
  template <int LPR>
  __device__ __forceinline__ double reduce() {
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
      const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
      float s, e;
      two_sum_f(hi, oh, s, e);
      hi = s;
      lo = __fadd_rn(lo, __fadd_rn(ol, e));
    }
    return double(hi) + double(lo);
  }
};

constexpr int BU = 4;  // 16-byte chunks per lane loaded ahead

// One CTA per (tile, part of its owner rows). LPR lanes per box row (2, 4 or 8, chosen from
// the box length so that short rows do not leave lanes idle), 32 / LPR rows per warp, each
// lane streaming 16-byte chunks (2 FP64 or 4 FP32 values). The first BU chunks of a lane's
// next row are loaded before the current row is reduced, and those of its first row before
// the window is staged, so the box loads overlap the staging and the reductions.
template <typename PT, int LPR>
__global__ void __launch_bounds__(256) gemv_band_kernel(const PT* __restrict__ Pb, const BandClass* __restrict__ cls,
                                                        const TileDesc* __restrict__ tiles,
                                                        const double* __restrict__ src, double* __restrict__ u,
                                                        int64_t ny, int64_t nx, int accumulate, int rsplit) {
  extern __shared__ __align__(16) unsigned char wraw[];
  PT* w = reinterpret_cast<PT*>(wraw);
  const int t = blockIdx.x / rsplit, part = blockIdx.x % rsplit;
  const TileDesc td = tiles[t];
  const BandClass c = cls[td.cls];
  const int ien = td.iext[0] * td.iext[1];
  const int rows_per = (ien + rsplit - 1) / rsplit;
  const int ib = part * rows_per, ie = min(ien, ib + rows_per);
  constexpr int RPW = 32 / LPR;
  constexpr int V = 16 / sizeof(PT);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  const int grp = lane / LPR, gl = lane % LPR;
  const int cpr = c.bxp / V;      // chunks per box row
  const int nch = c.byc * cpr;    // chunks per stored row
  auto row_ptr = [&](int i) { return reinterpret_cast<const int4*>(Pb + c.off + int64_t(i) * c.L); };
  auto load_head = [&](int i, int4 (&v)[BU]) {
    const bool live = i < ie;
    const int4* r4 = row_ptr(live ? i : ib);
#pragma unroll
    for (int k = 0; k < BU; ++k) {
      const int q = gl + LPR * k;
      v[k] = (live && q < nch) ? __ldcs(r4 + q) : make_int4(0, 0, 0, 0);
    }
  };
  int i = ib + warp * RPW + grp;
  int4 head[BU];
  load_head(i, head);
  const int wn = td.wext[0] * td.wext[1];
  for (int k = threadIdx.x; k < wn + 4; k += blockDim.x) {
    if (k >= wn) {  // padding read by the last chunk of a box row (its P values are zero)
      w[k] = PT(0);
      continue;
    }
    const int a = k / td.wext[1], b = k % td.wext[1];
    int64_t gy = int64_t(td.org[0]) + a, gx = int64_t(td.org[1]) + b;
    gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
    gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
    w[k] = PT(src[gy * nx + gx]);
  }
  __syncthreads();
  using Acc = typename std::conditional<sizeof(PT) == 8, BAccD, BAccF>::type;
  // every lane runs the same number of row iterations (the shuffles need the whole warp)
  for (int i0 = ib + warp * RPW; i0 < ie; i0 += nw * RPW, i += nw * RPW) {
    const bool live = i < ie;
    int py, px, y0, x0;
    box_origin(c, live ? i : ib, py, px, y0, x0);
    Acc acc;
    auto consume = [&](const int4& v, int q) {
      const int a = q / cpr, j0 = (q - a * cpr) * V;
      const PT* pv = reinterpret_cast<const PT*>(&v);
      const PT* wv = w + (y0 + a) * c.wx + x0 + j0;
#pragma unroll
      for (int h = 0; h < V; ++h) acc.add(pv[h], wv[h]);
    };
#pragma unroll
    for (int k = 0; k < BU; ++k) {
      const int q = gl + LPR * k;
      if (q < nch) consume(head[k], q);
    }
    // the rest of a long row, BU chunks per lane in flight
    const int4* r4 = row_ptr(live ? i : ib);
    for (int q0 = gl + LPR * BU; q0 < nch; q0 += LPR * BU) {
      int4 v[BU];
#pragma unroll
      for (int k = 0; k < BU; ++k) {
        const int q = q0 + LPR * k;
        v[k] = (live && q < nch) ? __ldcs(r4 + q) : make_int4(0, 0, 0, 0);
      }
#pragma unroll
      for (int k = 0; k < BU; ++k) {
        const int q = q0 + LPR * k;
        if (q < nch) consume(v[k], q);
      }
    }
    load_head(i + nw * RPW, head);  // the next row's first chunks, in flight during the reduce
    const double y = acc.template reduce<LPR>();
    if (live && gl == 0) {
      const int64_t p = int64_t(td.t0[0] + i / td.iext[1]) * nx + td.t0[1] + i % td.iext[1];
      u[p] = accumulate ? u[p] + y : y;
    }
  }
}

// Short box rows (1D windows, small 2D boxes): one thread per owner row, no reduction. Each
// thread walks its row's chunks in order with BU 16-byte loads ahead (read-only path, so the
// other half of each 32-byte sector a warp touches is still in L1 when the next chunk needs
// it), box coordinates (a, j) advanced incrementally. FP32 rows sum a chunk's products by FMA
// and add the chunk sum into a float-float accumulator; FP64 rows use FMAs throughout.
template <typename PT>
__global__ void __launch_bounds__(256) gemv_band_row_kernel(const PT* __restrict__ Pb,
                                                            const BandClass* __restrict__ cls,
                                                            const TileDesc* __restrict__ tiles,
                                                            const double* __restrict__ src, double* __restrict__ u,
                                                            int64_t ny, int64_t nx, int accumulate, int rsplit) {
  extern __shared__ __align__(16) unsigned char wraw[];
  PT* w = reinterpret_cast<PT*>(wraw);
  const int t = blockIdx.x / rsplit, part = blockIdx.x % rsplit;
  const TileDesc td = tiles[t];
  const BandClass c = cls[td.cls];
  const int ien = td.iext[0] * td.iext[1];
  const int rows_per = (ien + rsplit - 1) / rsplit;
  const int ib = part * rows_per, ie = min(ien, ib + rows_per);
  constexpr int V = 16 / sizeof(PT);
  const int cpr = c.bxp / V;
  const int nch = c.byc * cpr;
  int i = ib + int(threadIdx.x);
  int4 v[BU];
  auto load = [&](int row, int q0, int4 (&dst)[BU]) {
    const bool live = row < ie;
    const int4* r4 = reinterpret_cast<const int4*>(Pb + c.off + int64_t(live ? row : ib) * c.L);
#pragma unroll
    for (int k = 0; k < BU; ++k) dst[k] = (live && q0 + k < nch) ? __ldg(r4 + q0 + k) : make_int4(0, 0, 0, 0);
  };
  load(i, 0, v);  // in flight while the window is staged
  const int wn = td.wext[0] * td.wext[1];
  for (int k = threadIdx.x; k < wn + 4; k += blockDim.x) {
    if (k >= wn) {  // padding read by the last chunk of a box row (its P values are zero)
      w[k] = PT(0);
      continue;
    }
    const int a = k / td.wext[1], b = k % td.wext[1];
    int64_t gy = int64_t(td.org[0]) + a, gx = int64_t(td.org[1]) + b;
    gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
    gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
    w[k] = PT(src[gy * nx + gx]);
  }
  __syncthreads();
  for (; i < ie; i += blockDim.x) {
    int py, px, y0, x0;
    box_origin(c, i, py, px, y0, x0);
    double acc = 0.0;
    float hi = 0.0f, lo = 0.0f;
    int a = 0, j = 0;  // box row and chunk of chunk q
    for (int q0 = 0; q0 < nch; q0 += BU) {
      int4 nv[BU];
      load(i, q0 + BU, nv);
#pragma unroll
      for (int k = 0; k < BU; ++k) {
        if (q0 + k < nch) {
          const PT* pv = reinterpret_cast<const PT*>(&v[k]);
          const PT* wv = w + (y0 + a) * c.wx + x0 + j * V;
          if constexpr (sizeof(PT) == 8) {
#pragma unroll
            for (int h = 0; h < V; ++h) acc = fma(double(pv[h]), double(wv[h]), acc);
          } else {
            float sc = 0.0f;
#pragma unroll
            for (int h = 0; h < V; ++h) sc = fmaf(float(pv[h]), float(wv[h]), sc);
            float s, e;
            two_sum_f(hi, sc, s, e);
            hi = s;
            lo = __fadd_rn(lo, e);
          }
          if (++j == cpr) {
            j = 0;
            ++a;
          }
        }
      }
#pragma unroll
      for (int k = 0; k < BU; ++k) v[k] = nv[k];
    }
    const double y = sizeof(PT) == 8 ? acc : double(hi) + double(lo);
    const int64_t p = int64_t(td.t0[0] + i / td.iext[1]) * nx + td.t0[1] + i % td.iext[1];
    u[p] = accumulate ? u[p] + y : y;
    load(i + int(blockDim.x), 0, v);
  }
}

template <typename PT>
using BandKernel = void (*)(const PT*, const BandClass*, const TileDesc*, const double*, double*, int64_t, int64_t, int,
                            int);

template <typename PT>
BandKernel<PT> band_kernel_for(int lpr) {
  if (lpr == 1) return gemv_band_row_kernel<PT>;
  if (lpr == 2) return gemv_band_kernel<PT, 2>;
  if (lpr == 4) return gemv_band_kernel<PT, 4>;
  return gemv_band_kernel<PT, 8>;
}

// Launch shape of the band GEMV for one value size: lanes per row from the longest stored
// row (in 16-byte chunks: at most about BU chunks per lane), threads per block to cover a
// tile's owner rows in one pass where they fit in 256 threads, and blocks per tile so that
// the launch has about four waves of blocks.
struct BandLaunch {
  int lpr = 8, threads = 256, rsplit = 1;
};

BandLaunch band_launch(const lem_ctx* ctx, const std::vector<BandClass>& cls, int value_bytes) {
  BandLaunch L;
  int nch = 1, rows = 1;
  for (const BandClass& c : cls) {
    nch = std::max(nch, c.byc * c.bxp * value_bytes / 16);
    rows = std::max(rows, c.iy * c.ix);
  }
  // one thread per row up to 8 BU chunks per row (FP32: 128 values, FP64: 64), else
  // lanes per row so that each lane takes about BU chunks
  L.lpr = nch <= 8 * BU ? 1 : (nch <= 2 * BU * 8 ? 4 : 8);
  const int rpw = 32 / L.lpr;
  L.threads = std::min(256, std::max(32, (rows + rpw - 1) / rpw * 32));
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || nsm < 1) nsm = 152;
  const int64_t nt = int64_t(ctx->tiles.size());
  const int per_sm = std::max(1, 2048 / L.threads);
  const int rows_per_pass = (L.threads / 32) * rpw;
  const int max_split = std::max(1, rows / rows_per_pass);
  L.rsplit = int(std::max<int64_t>(1, std::min<int64_t>(max_split, (4LL * per_sm * nsm + nt - 1) / nt)));
  return L;
}

}  // namespace

// Host side of the truncated apply, kept with the context.
struct BandPlan {
  std::vector<BandClass> cls;
  BandClass* d_cls = nullptr;
  int* d_ext = nullptr;
  double* d_Pb = nullptr;
  float* d_Pb32 = nullptr;
  int64_t cap = 0;  // values the packed arrays hold
  int64_t used = 0;
  int wmax = 0;     // largest window (nodes) of any class, for the staged window
  BandLaunch l64, l32;  // launch shapes for FP64 and FP32 boxes
};

void band_destroy(lem_ctx* ctx) {
  BandPlan* b = ctx->band;
  if (!b) return;
  for (void* p : {static_cast<void*>(b->d_cls), static_cast<void*>(b->d_ext), static_cast<void*>(b->d_Pb),
                  static_cast<void*>(b->d_Pb32)})
    if (p) cudaFreeAsync(p, ctx->stream);
  delete b;
  ctx->band = nullptr;
}

// Extents from the tolerance and the packed boxes for the current propagators (synchronises
// the context stream once, to read the extents back).
lem_status band_prepare(lem_ctx* ctx) {
  if (!ctx->built) return fail(LEM_ENOTREADY, "propagators not built");
  if (!ctx->band) ctx->band = new BandPlan();
  BandPlan* b = ctx->band;
  const int nc = int(ctx->classes.size());
  cudaStream_t st = ctx->stream;
  int wym = 1, wxm = 1;
  for (const ClassDesc& cd : ctx->classes) {
    wym = std::max(wym, int(cd.wext[0]));
    wxm = std::max(wxm, int(cd.wext[1]));
  }
  if (wym > 1024 || wxm > 1024) return fail(LEM_EINVAL, "truncation supports windows of at most 1024 nodes per axis");
  const size_t smem = sizeof(double) * (size_t(EXT_WARPS) * (3 * (wxm + wym) + 4) + 2 * (wym + wxm) + 1);
  if (b->cls.empty()) {
    LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&b->d_cls), sizeof(BandClass) * nc));
    LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&b->d_ext), sizeof(int) * 4 * nc));
    LEM_CUDA_TRY(cudaFuncSetAttribute(band_extents_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    b->cls.resize(nc);
    for (int k = 0; k < nc; ++k) {
      const ClassDesc& cd = ctx->classes[k];
      BandClass& c = b->cls[k];
      c = BandClass{};
      c.wy = cd.wext[0]; c.wx = cd.wext[1]; c.iy = cd.iext[0]; c.ix = cd.iext[1];
      c.oy = cd.iofs[0]; c.ox = cd.iofs[1];
      b->wmax = std::max(b->wmax, c.wy * c.wx);
    }
  }
  LEM_CUDA_TRY(cudaMemcpyAsync(b->d_cls, b->cls.data(), sizeof(BandClass) * nc, cudaMemcpyHostToDevice, st));
  band_extents_kernel<<<nc, EXT_THREADS, smem, st>>>(ctx->d_P, ctx->n_int, ctx->n_loc, b->d_cls, wym, wxm,
                                                      ctx->band_tol, b->d_ext);
  LEM_CUDA_TRY(cudaGetLastError());
  std::vector<int> ext(4 * size_t(nc));
  LEM_CUDA_TRY(cudaMemcpyAsync(ext.data(), b->d_ext, sizeof(int) * ext.size(), cudaMemcpyDeviceToHost, st));
  LEM_CUDA_TRY(cudaStreamSynchronize(st));
  int64_t total = 0;
  for (int k = 0; k < nc; ++k) {
    BandClass& c = b->cls[k];
    c.ly = ext[4 * k]; c.hy = ext[4 * k + 1]; c.lx = ext[4 * k + 2]; c.hx = ext[4 * k + 3];
    c.byc = std::min(c.ly + c.hy + 1, c.wy);
    c.bxc = std::min(c.lx + c.hx + 1, c.wx);
    c.bxp = (c.bxc + 3) / 4 * 4;
    c.L = c.byc * c.bxp;
    c.off = total;
    total += int64_t(c.iy) * c.ix * c.L;
  }
  const bool f32 = ctx->apply_path == LEM_APPLY_F32_BAND;
  if (total > b->cap) {
    if (b->d_Pb) cudaFreeAsync(b->d_Pb, st);
    if (b->d_Pb32) cudaFreeAsync(b->d_Pb32, st);
    b->d_Pb = nullptr;
    b->d_Pb32 = nullptr;
    b->cap = 0;
    LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&b->d_Pb), sizeof(double) * size_t(total)));
    if (f32) LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&b->d_Pb32), sizeof(float) * size_t(total)));
    b->cap = total;
  } else if (f32 && !b->d_Pb32) {
    LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&b->d_Pb32), sizeof(float) * size_t(b->cap)));
  }
  b->used = total;
  LEM_CUDA_TRY(cudaMemcpyAsync(b->d_cls, b->cls.data(), sizeof(BandClass) * nc, cudaMemcpyHostToDevice, st));
  band_pack_kernel<<<dim3(unsigned(ctx->n_int), unsigned(nc)), 128, 0, st>>>(ctx->d_P, ctx->n_int, ctx->n_loc, b->d_cls,
                                                                           b->d_Pb, f32 ? b->d_Pb32 : nullptr);
  LEM_CUDA_TRY(cudaGetLastError());
  b->l64 = band_launch(ctx, b->cls, 8);
  b->l32 = band_launch(ctx, b->cls, 4);
  const int bytes = int(sizeof(double) * size_t(b->wmax + 4));
  if (bytes > 48 * 1024) {
    for (int lpr : {1, 2, 4, 8}) {
      LEM_CUDA_TRY(cudaFuncSetAttribute(band_kernel_for<double>(lpr), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
      LEM_CUDA_TRY(cudaFuncSetAttribute(band_kernel_for<float>(lpr), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    }
  }
  ctx->band_gen = ctx->build_gen;
  return LEM_OK;
}

lem_status band_get(lem_ctx* ctx, int64_t cls, int32_t* ext, int64_t* row_values) {
  if (ctx->band_gen != ctx->build_gen) LEM_TRY(band_prepare(ctx));
  if (cls < 0) {
    ext[0] = ext[1] = ext[2] = ext[3] = 0;
    if (row_values) *row_values = ctx->band->used;
    return LEM_OK;
  }
  const BandClass& c = ctx->band->cls[cls];
  ext[0] = c.ly; ext[1] = c.hy; ext[2] = c.lx; ext[3] = c.hx;
  if (row_values) *row_values = c.L;
  return LEM_OK;
}

int64_t band_values(const lem_ctx* ctx) { return ctx->band ? ctx->band->used : 0; }

// One LEM step with the truncated propagators: PHI reads the residual, EXP a copy of u^n.
lem_status band_step(lem_ctx* ctx, double* d_u) {
  if (ctx->band_gen != ctx->build_gen) LEM_TRY(band_prepare(ctx));
  BandPlan* b = ctx->band;
  cudaStream_t st = ctx->stream;
  const bool phi = ctx->desc.mode == LEM_MODE_PHI;
  if (phi) {
    LEM_CUDA_TRY(launch_residual_fp64(ctx, ctx->d_r, d_u));
  } else {
    LEM_CUDA_TRY(cudaMemcpyAsync(ctx->d_r, d_u, sizeof(double) * ctx->npts, cudaMemcpyDeviceToDevice, st));
  }
  const bool f32 = ctx->apply_path == LEM_APPLY_F32_BAND;
  const unsigned nt = unsigned(ctx->tiles.size());
  const BandLaunch& L = f32 ? b->l32 : b->l64;
  cudaEvent_t stop;
  LEM_CUDA_TRY(ctx->timing_begin(&stop));
  if (f32) {
    const size_t smem = sizeof(float) * size_t(b->wmax + 4);
    band_kernel_for<float>(L.lpr)<<<nt * L.rsplit, L.threads, smem, st>>>(b->d_Pb32, b->d_cls, ctx->d_tiles, ctx->d_r,
                                                                         d_u, ctx->ny, ctx->nx, phi ? 1 : 0, L.rsplit);
  } else {
    const size_t smem = sizeof(double) * size_t(b->wmax + 4);
    band_kernel_for<double>(L.lpr)<<<nt * L.rsplit, L.threads, smem, st>>>(b->d_Pb, b->d_cls, ctx->d_tiles, ctx->d_r,
                                                                          d_u, ctx->ny, ctx->nx, phi ? 1 : 0, L.rsplit);
  }
  ctx->timing_end(stop);
  LEM_CUDA_TRY(cudaGetLastError());
  return LEM_OK;
}

}  // namespace lem
