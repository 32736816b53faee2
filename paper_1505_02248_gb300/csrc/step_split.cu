// Split-precision LEM step on the tcgen05 tensor cores (Sec. 3 steps 1-3, Eq. lem) for
// problems whose windows all share one local operator (constant coefficients, periodic 2D
// mesh, tiles dividing the mesh). One step is two kernels:
//
//  1. residual_split_kernel: r = dt A u^n from the float-float state (float-float
//     arithmetic: the stencil differences of a smooth field cancel), scaled by one global
//     power of two 2^er and written as two FP16 slices r*2^er = r_int + r2 into a
//     ghost-padded [ny + 2Hy][pitch] array (the periodic halo is materialised here, so
//     every window is a plain rectangle of it). r_int is an integer (|r_int| <= 2^rb),
//     r2 the FP16-rounded remainder (with three pieces, r3 the FP16-rounded remainder of
//     that). er comes from the previous step's max|r|.
//  2. split_gemm_kernel: Y = P R (M = Ty*Tx owner rows, N = tiles, K = window nodes).
//     P is stored per row i as P*2^eP_i = P_int + P2 with |P_int| <= 2^9 an integer.
//     Each K block is one window row (Wx = 16, 32, 48 or 64 nodes: ceil(Wx / 16) * 16 columns
//     loaded into 128-byte swizzled rows): TMA loads P_int/P2 and the 128 windows' rows of
//     r_int/r2 straight from the padded residual
//     through a 4D tensor map (the halo gather happens inside TMA). One thread issues
//     tcgen05.mma: P_int r_int into the main TMEM accumulator and P_int r2, P2 r_int and
//     P2 r2 into a correction accumulator. Because sum_k |P_int| |r_int| < 2^24
//     (checked when P is packed), every partial sum of the main product is an integer that
//     FP32 holds exactly, whatever rounding the tensor pipe's accumulator applies; only the
//     small correction products see that rounding. The epilogue forms
//     y = (main + corr) 2^-(eP_i + er) and adds it into the owner nodes of the float-float
//     state (the scatter).
//
// The float-float state (u_hi + u_lo, about 48 bits) is converted from/to the caller's
// FP64 buffer once per lem_step call.
#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ff_convert.h"
#include "lem_internal.h"
#include "tc_ptx.cuh"

namespace lem {

namespace {

constexpr int BM = 128;            // owner rows per CTA tile (TMEM lanes)
constexpr int KB = 64;             // fp16 elements per 128-byte K row (window rows padded to it)
constexpr int A_BYTES = BM * KB * 2;  // one P slice of a stage: 128 rows x 128 B = 16 KB
constexpr int RING_BYTES = 192 * 1024;
constexpr int SMEM_BYTES = RING_BYTES + 1024 + 256;
constexpr uint32_t TMEM_COLS = 512;   // main + correction accumulators: 2 sets for BN = 128, 1 for 256

// Tile shape: BN windows per CTA tile (TMEM columns per accumulator), NP pieces of each
// operand (2: P_int + P2 and r_int + r2, four products; 3: a third FP16 piece of each, six
// products). BN = 256 halves the shared-memory operand traffic per MMA (an N = 128 MMA reads
// its 8 KB of operands at the full 128 B/clk shared-memory rate); it leaves room for one
// accumulator set and two stages of two pieces.
template <int BN, int NP>
struct Shape {
  static constexpr int B_BYTES = BN * KB * 2;                      // one residual slice of a stage
  static constexpr int STAGE_BYTES = NP * (A_BYTES + B_BYTES);      // P pieces, then r pieces
  static constexpr int STAGES = RING_BYTES / STAGE_BYTES;           // 3 (BN 128, NP 2) or 2
  static constexpr int NBUF = BN == 256 ? 1 : 2;                    // TMEM accumulator sets
  static_assert(STAGES >= 2, "at least two stages");
};
// Thread roles: warp 0 TMA producer, warp 1 MMA issuer, warps 2-9 the epilogue, two per TMEM
// lane quarter (warp % 4), the one of warps 2-5 taking the even 32-column blocks of the
// accumulators and the one of warps 6-9 the odd ones. With two pieces the epilogue reads the
// accumulators once per tile. With three pieces (DRAIN) it also drains the correction
// accumulator into registers after every window row: the tensor pipe's FP32 accumulation of
// the correction then spans only 5 * ceil(Wx/16) MMAs, and the sum over window rows is a
// correctly rounded FP32 add. Two warps per quarter halve each drain and each scatter.
constexpr int EPI_WARPS = 8;
constexpr int GEMM_THREADS = 64 + 32 * EPI_WARPS;
constexpr int P_INT_BITS = 9;            // |P_int| <= 2^9
constexpr uint64_t WAIT_NS = 2000000000ull;  // 2 s bound on every mbarrier wait

enum : int { ERR_TIMEOUT_PRODUCER = 1, ERR_TIMEOUT_MMA = 2, ERR_TIMEOUT_EPI = 3, ERR_NUMERIC = 4 };

// Geometry of one problem's GEMM (all counts in tiles unless stated).
struct GemmGeom {
  int Wy, Wx, Ty, Tx, nx, BNx, BNy, ntx, nty;
  int M;                // owner rows (Ty * Tx); M blocks past it are masked
  int nbx;              // window blocks per row of the tile grid
  int bnp;              // windows per block (BNx * BNy <= BN, a multiple of 16): the MMA's N
  int lbx;              // log2 BNx (BNx is a power of two)
  int balance;          // one problem: spread the last, partial wave's window rows over every CTA
  float* part;          // balance: per CTA, the folded sums of a tile part it leaves to another CTA
  unsigned* flags;      // balance: per CTA and epilogue warp, the launch epoch of its stored part
  int nMB, nNB;         // M blocks of 128 owner rows, window blocks of BN windows
  int drain_rows;       // three pieces: window rows per correction drain
  int kx;               // K columns loaded per window row: Wx rounded up to 16 (the MMA's K steps)
  int unit0;            // multi-problem launch: this problem's first unit
  int fault;            // test hook (LEM_FAULT=timeout): CTA 0 arms its first stage but loads
                        // nothing, so the MMA issuer's bounded wait expires
  const __half* Pt;     // P pieces as shared-memory images [M blocks][Wy][NP][BM x kx]
  const int* eP;        // per owner row: P scale exponent
  const int* escale;    // [2] residual scale exponent of each step parity
  unsigned* rmax;       // [2] max|r| accumulators (the GEMM clears the current one)
  float* uh;            // float-float state
  float* ul;
};

// Everything one problem's GEMM reads: its six tensor maps (P_int, P2, P3, r_int, r2, r3;
// the third pieces unused with two) and its geometry. Passed by value (__grid_constant__)
// for a single problem, or as a device array for a multi-problem launch.
struct SplitProblem {
  CUtensorMap tm[6];
  GemmGeom g;
};

struct ResParams {
  int ny, nx, Hy, Hx, pitch, prow;
  float c_hi[5], c_lo[5];   // dt-scaled C, W, E, S, N as float pairs
  float csum_hi, csum_lo;   // sum of all five
  const int* rb;            // device: |r_int| target 2^(rb-1) (2x headroom below 2^rb), set at packing
  int has_lo;               // some coefficient (or their sum) is not exact in float
};

__device__ __forceinline__ float pow2f(int e) {  // exact 2^e for -126 <= e <= 127
  return __int_as_float((127 + e) << 23);
}

// Float-float helpers. The _rn intrinsics keep the compiler from contracting the
// error-free transformations into FMAs (which would break TwoSum's exactness).
struct ffv {
  float h, l;
};

__device__ __forceinline__ ffv two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// (ah + al) - (bh + bl) as an unnormalised pair
__device__ __forceinline__ ffv ff_sub(float ah, float al, float bh, float bl) {
  ffv t = two_sum(ah, -bh);
  t.l = __fadd_rn(t.l, __fsub_rn(al, bl));
  return t;
}

// acc += (ch + cl) * d, keeping the product's rounding error (exact through the FMA);
// HAS_LO = false when the coefficient is exact in float (cl == 0)
template <bool HAS_LO>
__device__ __forceinline__ void ff_mac(ffv& acc, float ch, float cl, ffv d) {
  const float p = __fmul_rn(ch, d.h);
  float pe = fmaf(ch, d.h, -p);
  if (HAS_LO) pe = fmaf(cl, d.h, pe);
  pe = fmaf(ch, d.l, pe);
  const ffv s = two_sum(acc.h, p);
  acc.h = s.h;
  acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, pe));
}

// exponent e with |x| < 2^e (x > 0)
__device__ __forceinline__ int exponent_above(float x) {
  int e;
  frexpf(x, &e);
  return e;
}

constexpr int RTX = 64, RTY = 32;  // residual output tile (padded coordinates) per block

// One RTX x RTY tile of the padded residual per 256-thread block: the (RTY+2) x (RTX+2)
// float-float patch of u around it (mesh coordinates wrapped, any number of times for small
// meshes) is staged in shared memory row by row, so each node is read from global memory once
// per block. Each thread then forms the outputs of columns tx and tx + 32 in four rows, so a
// warp's shared-memory reads and its FP16 stores are consecutive (no bank conflicts).
// measure != 0: only accumulate max|r| into rmax[parity ^ 1].
// FROM64: the patch comes from the FP64 state u64 instead, converted to float-float as it is
// staged, and the padded interior's nodes (each mesh node once over the grid) also write that
// float-float state to (oh, ol).
template <bool FROM64 = false>
__device__ __forceinline__ void residual_tile(const float* __restrict__ uh, const float* __restrict__ ul,
                                              __half* __restrict__ Rint, __half* __restrict__ R2,
                                              __half* __restrict__ R3, const ResParams& p, unsigned* rmax,
                                              int* escale, int parity, int measure, int bx, int by,
                                              const double* __restrict__ u64 = nullptr, float* __restrict__ oh = nullptr,
                                              float* __restrict__ ol = nullptr) {
  constexpr int SW = RTX + 3;  // staged row stride (odd: conflict-free column reads)
  __shared__ float sh[RTY + 2][SW], sl[RTY + 2][SW];
  __shared__ float red[8];
  const float rm = __uint_as_float(rmax[parity]);
  const int er = rm > 0.0f ? (*p.rb - 1) - exponent_above(rm) : 0;
  const float scale = pow2f(er);
  if (!measure && bx == 0 && by == 0 && threadIdx.x == 0) escale[parity] = er;
  const int x0 = bx * RTX, y0 = by * RTY;  // padded tile origin
  const int wpad = p.nx + 2 * p.Hx;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 32 x 8
  // stage u over padded rows y0-1 .. y0+RTY and columns x0-1 .. x0+RTX: the three wrapped
  // mesh columns of this thread first, then row by row
  auto wrap = [](int v, int n) {  // v mod n in [0, n); one add or subtract in the usual case
    if (v >= 0 && v < n) return v;
    if (v < 0 && v >= -n) return v + n;
    if (v >= n && v < 2 * n) return v - n;
    v %= n;  // meshes smaller than the halo
    return v < 0 ? v + n : v;
  };
  int gx[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) gx[j] = wrap(x0 + tx + 32 * j - 1 - p.Hx, p.nx);
  for (int ly = ty; ly < RTY + 2; ly += 8) {
    const int y = wrap(y0 + ly - 1 - p.Hy, p.ny);
    if constexpr (FROM64) {
      const double* rv = u64 + int64_t(y) * p.nx;
      // padded row yp = y0 + ly - 1 inside [Hy, Hy + ny) is mesh row y = yp - Hy
      const int yp = y0 + ly - 1;
      const bool row_own = ly >= 1 && ly <= RTY && yp >= p.Hy && yp < p.Hy + p.ny;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int lx = tx + 32 * j;
        if (lx < RTX + 2) {
          float h, l;
          f64_to_pair(rv[gx[j]], h, l);
          sh[ly][lx] = h;
          sl[ly][lx] = l;
          const int xp = x0 + lx - 1;  // inside [Hx, Hx + nx): mesh column gx[j] = xp - Hx
          if (row_own && lx >= 1 && lx <= RTX && xp >= p.Hx && xp < p.Hx + p.nx) {
            oh[int64_t(y) * p.nx + gx[j]] = h;
            ol[int64_t(y) * p.nx + gx[j]] = l;
          }
        }
      }
    } else {
      const float* rh = uh + int64_t(y) * p.nx;
      const float* rl = ul + int64_t(y) * p.nx;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int lx = tx + 32 * j;
        if (lx < RTX + 2) {
          sh[ly][lx] = rh[gx[j]];
          sl[ly][lx] = rl[gx[j]];
        }
      }
    }
  }
  __syncthreads();
  float rabs = 0.0f;
  // r = sum_nbr c_j (u_j - u_C) + (sum_all c) u_C, every term and the sum in float-float:
  // the W/E (S/N) differences of a smooth field nearly cancel, so a float sum would lose
  // about log2(|c d| / |r|) bits of r. The first product starts the sum as 0 + p, 0 + pe
  // (what adding it to a zero pair gives).
  auto first = [&](float ch, float cl, ffv d) -> ffv {
    const float q = __fmul_rn(ch, d.h);
    float pe = fmaf(ch, d.h, -q);
    if (p.has_lo) pe = fmaf(cl, d.h, pe);
    pe = fmaf(ch, d.l, pe);
    return {__fadd_rn(0.0f, q), __fadd_rn(0.0f, __fadd_rn(0.0f, pe))};
  };
  auto rest = [&](ffv& acc, float ch, float cl, ffv d) {
    if (p.has_lo) ff_mac<true>(acc, ch, cl, d);
    else ff_mac<false>(acc, ch, 0.0f, d);
  };
  // r 2^er = r_int + r2 (+ r3), split from the float-float value: r_int an integer, the
  // remainder t + l (t exact in float) rounded to FP16 twice. Three pieces carry about rb + 22
  // bits, more than one float holds, so the low word takes part.
  auto pieces = [&](ffv r, __half& hi, __half& h2, __half& h3) {
    const float rh = __fmul_rn(r.h, scale), rl = __fmul_rn(r.l, scale);  // exact (powers of two)
    hi = __float2half_rn(rintf(rh));
    const float t = __fsub_rn(rh, __half2float(hi));  // exact (r_int may round in FP16 past 2048)
    h2 = __float2half_rn(__fadd_rn(t, rl));
    h3 = __float2half_rn(__fadd_rn(__fsub_rn(t, __half2float(h2)), rl));  // t - r2 exact
  };
  // Each thread forms columns tx and tx + 32 of four consecutive rows 4 ty .. 4 ty + 3, so the
  // difference to the row above, u_N - u_C, is the next row's u_S - u_C negated (exactly: the
  // float-float difference is antisymmetric under round-to-nearest).
  const bool csum = p.has_lo || p.csum_hi != 0.0f;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int lx = tx + 32 * j;
    const int xp = x0 + lx;
    if (xp >= wpad) continue;
    const int cx = lx + 1;
    const int cy0 = 4 * ty + 1;
    // u_{row0} - u_{row0 - 1}: the first row's u_S - u_C, negated
    ffv below = ff_sub(sh[cy0][cx], sl[cy0][cx], sh[cy0 - 1][cx], sl[cy0 - 1][cx]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int cy = cy0 + k;
      const int yp = y0 + cy - 1;
      if (yp >= p.prow) break;
      const float ch = sh[cy][cx], cl = sl[cy][cx];
      const ffv dW = ff_sub(sh[cy][cx - 1], sl[cy][cx - 1], ch, cl);
      const ffv dE = ff_sub(sh[cy][cx + 1], sl[cy][cx + 1], ch, cl);
      const ffv dS{-below.h, -below.l};
      const ffv dN = ff_sub(sh[cy + 1][cx], sl[cy + 1][cx], ch, cl);
      below = dN;
      ffv acc = first(p.c_hi[1], p.c_lo[1], dW);
      rest(acc, p.c_hi[2], p.c_lo[2], dE);
      rest(acc, p.c_hi[3], p.c_lo[3], dS);
      rest(acc, p.c_hi[4], p.c_lo[4], dN);
      if (csum) rest(acc, p.csum_hi, p.csum_lo, ffv{ch, cl});
      const ffv r = two_sum(acc.h, acc.l);  // normalised: |r.l| <= ulp(r.h) / 2
      rabs = fmaxf(rabs, fabsf(r.h));
      if (measure) continue;
      __half h1, h2, h3;
      pieces(r, h1, h2, h3);
      const int64_t o = int64_t(yp) * p.pitch + xp;
      Rint[o] = h1;
      R2[o] = h2;
      if (R3) R3[o] = h3;
    }
  }
  for (int o = 16; o > 0; o >>= 1) rabs = fmaxf(rabs, __shfl_xor_sync(0xffffffffu, rabs, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = rabs;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = red[0];
    for (int w = 1; w < 8; ++w) m = fmaxf(m, red[w]);
    atomicMax(rmax + (parity ^ 1), __float_as_uint(m));
  }
}

// Programmatic dependent launch: a kernel launched with programmatic stream serialization may
// start while the previous kernel of the stream finishes; it waits for that kernel's results
// here (a no-op for an ordinary launch) and lets the next kernel start its own set-up.
__device__ __forceinline__ void pdl_wait_and_release() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__global__ void __launch_bounds__(256) residual_split_kernel(const float* __restrict__ uh,
                                                             const float* __restrict__ ul,
                                                             __half* __restrict__ Rint,
                                                             __half* __restrict__ R2,
                                                             __half* __restrict__ R3, ResParams p,
                                                             unsigned* rmax, int* escale, int parity,
                                                             int measure) {
  pdl_wait_and_release();
  residual_tile(uh, ul, Rint, R2, R3, p, rmax, escale, parity, measure, int(blockIdx.x), int(blockIdx.y));
}

// The measuring pass (max|r| of the first step into rmax[0]) on the FP64 state u64, which it
// also converts to the float-float state (uh, ul) the steps run on.
__global__ void __launch_bounds__(256) residual_measure_f64_kernel(const double* __restrict__ u64,
                                                                   float* __restrict__ uh, float* __restrict__ ul,
                                                                   ResParams p, unsigned* rmax, int* escale) {
  pdl_wait_and_release();
  residual_tile<true>(nullptr, nullptr, nullptr, nullptr, nullptr, p, rmax, escale, 1, 1, int(blockIdx.x),
                      int(blockIdx.y), u64, uh, ul);
}

// One problem of a multi-problem step: its residual arrays, parameters and block range.
struct ResProblem {
  ResParams p;
  const float* uh;
  const float* ul;
  __half* Rint;
  __half* R2;
  __half* R3;
  unsigned* rmax;
  int* escale;
  int gx;      // residual tiles along x
  int block0;  // first block of this problem
};

__device__ __forceinline__ int find_block(const int* __restrict__ first, int n, int b) {
  int lo = 0, hi = n - 1;  // last problem whose first block is <= b
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// The residual of every problem of a batch in one launch (one RTX x RTY tile per block).
__global__ void __launch_bounds__(256) residual_multi_kernel(const ResProblem* __restrict__ rps,
                                                             const int* __restrict__ first, int nprob, int parity,
                                                             int measure) {
  const int i = find_block(first, nprob, int(blockIdx.x));
  const ResProblem& q = rps[i];
  const int lb = int(blockIdx.x) - q.block0;
  residual_tile(q.uh, q.ul, q.Rint, q.R2, q.R3, q.p, q.rmax, q.escale, parity, measure, lb % q.gx, lb / q.gx);
}

// FP64 <-> float-float for every problem of a batch; to_ff also clears each max|r| pair.
struct ConvProblem {
  double* u;
  float* uh;
  float* ul;
  unsigned* rmax;
  int64_t n;
  int block0;
};
constexpr int CONV_CHUNK = 4096;

__global__ void __launch_bounds__(256) convert_multi_kernel(const ConvProblem* __restrict__ cps,
                                                            const int* __restrict__ first, int nprob, int to_ff) {
  const int i = find_block(first, nprob, int(blockIdx.x));
  const ConvProblem& q = cps[i];
  const int64_t b0 = int64_t(int(blockIdx.x) - q.block0) * CONV_CHUNK;
  const int64_t b1 = b0 + CONV_CHUNK < q.n ? b0 + CONV_CHUNK : q.n;
  if (to_ff) {
    if (b0 == 0 && threadIdx.x < 2) q.rmax[threadIdx.x] = 0u;
    for (int64_t k = b0 + threadIdx.x; k < b1; k += blockDim.x) {
      float h, l;
      f64_to_pair(q.u[k], h, l);
      q.uh[k] = h;
      q.ul[k] = l;
    }
  } else {
    for (int64_t k = b0 + threadIdx.x; k < b1; k += blockDim.x) q.u[k] = pair_to_f64(q.uh[k], q.ul[k]);
  }
}

// FP64 <-> float-float over n values, two per thread and iteration when the arrays allow it
// (the FP64 one 16-byte aligned, the float ones 8-byte aligned): a warp then reads and writes
// whole contiguous runs (256 bytes of each float array, 512 of the FP64 one), which also keeps
// writes over the host link to a mapped host state in whole lines. An odd last value, or
// unaligned arrays, go one by one.
__device__ __forceinline__ bool pairs_aligned(const void* u64, const void* a, const void* b) {
  return (reinterpret_cast<uintptr_t>(u64) & 15u) == 0 &&
         ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 7u) == 0;
}

__global__ void __launch_bounds__(256) f64_to_ff_kernel(const double* __restrict__ u, float* __restrict__ uh,
                                                        float* __restrict__ ul, int64_t n) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x, stride = int64_t(gridDim.x) * blockDim.x;
  int64_t done = 0;
  if (pairs_aligned(u, uh, ul)) {
    const int64_t n2 = n >> 1;
    for (int64_t k = t; k < n2; k += stride) {
      const double2 v = reinterpret_cast<const double2*>(u)[k];
      float2 h, l;
      f64_to_pair(v.x, h.x, l.x);
      f64_to_pair(v.y, h.y, l.y);
      reinterpret_cast<float2*>(uh)[k] = h;
      reinterpret_cast<float2*>(ul)[k] = l;
    }
    done = n2 << 1;
  }
  for (int64_t i = done + t; i < n; i += stride) {
    float h, l;
    f64_to_pair(u[i], h, l);
    uh[i] = h;
    ul[i] = l;
  }
}

__global__ void __launch_bounds__(256) ff_to_f64_kernel(const float* __restrict__ uh, const float* __restrict__ ul,
                                                        double* __restrict__ u, int64_t n) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x, stride = int64_t(gridDim.x) * blockDim.x;
  int64_t done = 0;
  if (pairs_aligned(u, uh, ul)) {
    const int64_t n2 = n >> 1;
    for (int64_t k = t; k < n2; k += stride) {
      const float2 h = reinterpret_cast<const float2*>(uh)[k];
      const float2 l = reinterpret_cast<const float2*>(ul)[k];
      reinterpret_cast<double2*>(u)[k] = make_double2(pair_to_f64(h.x, l.x), pair_to_f64(h.y, l.y));
    }
    done = n2 << 1;
  }
  for (int64_t i = done + t; i < n; i += stride) u[i] = pair_to_f64(uh[i], ul[i]);
}

// Per owner row i of P (FP64, n_int x n_loc, window row-major): eP_i with
// max_k |P[i,k]| 2^eP_i < 2^P_INT_BITS, then P 2^eP_i = P_int + P2 (+ P3), and S_i =
// sum_k |P_int[i,k]| (the exactness bound of the main product). The pieces are stored as the
// shared-memory images the MMA reads: one tile per (M block, window row, piece) of BM rows x
// kx columns (kx = Wx rounded up to 16, the MMA's K steps), in the unswizzled K-major layout
// of 8-row x 16-byte core matrices (128 contiguous bytes each; K-adjacent ones 128 B apart,
// row-adjacent ones kx * 16 B apart), so that one bulk copy of BM * kx * 2 bytes with no
// padding loads a tile (Pt: [M blocks][Wy][np][BM x kx]).
__device__ __forceinline__ int64_t ptile_index(int i, int wy, int q, int k, int Wy, int np, int kx) {
  const int mb = i / BM, r = i % BM;
  return ((int64_t(mb) * Wy + wy) * np + q) * (BM * kx) + ((r >> 3) * (kx >> 3) + (k >> 3)) * 64 + (r & 7) * 8 +
         (k & 7);
}

__global__ void pack_p_kernel(const double* __restrict__ P, int64_t n_loc, int M, int Wy, int Wx, int kpad, int np,
                              int kx, __half* __restrict__ Pt, int* __restrict__ eP, double* __restrict__ S) {
  const int i = blockIdx.x;
  if (i >= M) return;
  __shared__ double red[256];
  double m = 0.0;
  for (int k = threadIdx.x; k < Wy * Wx; k += blockDim.x) m = fmax(m, fabs(P[int64_t(i) * n_loc + k]));
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  int e = 0;
  if (red[0] > 0.0) frexp(red[0], &e);
  const int ei = red[0] > 0.0 ? P_INT_BITS - e : 0;
  __syncthreads();
  double sum = 0.0;
  for (int col = threadIdx.x; col < Wy * kpad; col += blockDim.x) {
    const int wy = col / kpad, wx = col % kpad;
    const double v = wx < Wx ? P[int64_t(i) * n_loc + int64_t(wy) * Wx + wx] : 0.0;
    const double x = ldexp(v, ei);
    const double xi = rint(x);
    const __half hi = __double2half(xi);  // exact: |xi| <= 2^9
    const __half h2 = __double2half(x - xi);
    if (wx < kx) {  // (columns past kx are zero and never read)
      Pt[ptile_index(i, wy, 0, wx, Wy, np, kx)] = hi;
      Pt[ptile_index(i, wy, 1, wx, Wy, np, kx)] = h2;
      if (np == 3) Pt[ptile_index(i, wy, 2, wx, Wy, np, kx)] = __double2half(x - xi - double(__half2float(h2)));
    }
    sum += fabs(xi);
  }
  red[threadIdx.x] = sum;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    eP[i] = ei;
    S[i] = red[0];
  }
}

// rb from the packed rows' exactness sums S_i: the largest rb <= 12 with
// max_i S_i 2^(rb+1) < 2^24 (rb <= 12: the target |r_int| <= 2^11 is an integer FP16 holds
// exactly). Rows too heavy for rb >= 4 set the numeric error flag.
__global__ void choose_rb_kernel(const double* __restrict__ S, int M, int* rb, int* err) {
  __shared__ double red[256];
  double m = 1.0;
  for (int i = threadIdx.x; i < M; i += blockDim.x) m = fmax(m, S[i]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + k]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int r = 0;
    while (ldexp(red[0], r + 1) < 16777216.0 && r < 12) ++r;
    if (r < 4) {
      atomicExch(err, ERR_NUMERIC);
      r = 4;
    }
    *rb = r;
  }
}

// Shared-memory descriptors of one stage's operand pieces at K step 0.
struct StageDesc {
  uint64_t P[3], R[3];
};
// K step kk of 16: P (unswizzled core matrices) advances 256 B, the residual (128-byte
// swizzled rows) 32 B; in 16-byte units of the descriptor's address field.
constexpr uint64_t ADV_P = 256 >> 4, ADV_R = 32 >> 4;

// Main product P_int r_int over KS K steps (exact: integer partial sums).
template <int KS>
__device__ __forceinline__ void issue_main(uint32_t main, const StageDesc& d, uint32_t idesc, uint32_t acc0) {
#pragma unroll
  for (int kk = 0; kk < KS; ++kk)
    ptx::mma_f16(main, d.P[0] + kk * ADV_P, d.R[0] + kk * ADV_R, idesc, kk == 0 ? acc0 : 1u);
}
// Two-piece corrections P_int r2 + P2 r_int + P2 r2.
template <int KS>
__device__ __forceinline__ void issue_corr2(uint32_t corr, const StageDesc& d, uint32_t idesc, uint32_t acc0) {
#pragma unroll
  for (int kk = 0; kk < KS; ++kk) {
    const uint64_t a = kk * ADV_P, r = kk * ADV_R;
    ptx::mma_f16(corr, d.P[0] + a, d.R[1] + r, idesc, kk == 0 ? acc0 : 1u);
    ptx::mma_f16(corr, d.P[1] + a, d.R[0] + r, idesc, 1u);
    ptx::mma_f16(corr, d.P[1] + a, d.R[1] + r, idesc, 1u);
  }
}
// Three pieces: per K step the main product and the five corrections P_int r2, P2 r_int,
// P2 r2, P_int r3, P3 r_int.
template <int KS>
__device__ __forceinline__ void issue_six(uint32_t main, uint32_t corr, const StageDesc& d, uint32_t idesc,
                                          uint32_t acc0, uint32_t cacc0) {
#pragma unroll
  for (int kk = 0; kk < KS; ++kk) {
    const uint64_t a = kk * ADV_P, r = kk * ADV_R;
    ptx::mma_f16(main, d.P[0] + a, d.R[0] + r, idesc, kk == 0 ? acc0 : 1u);
    ptx::mma_f16(corr, d.P[0] + a, d.R[1] + r, idesc, kk == 0 ? cacc0 : 1u);
    ptx::mma_f16(corr, d.P[1] + a, d.R[0] + r, idesc, 1u);
    ptx::mma_f16(corr, d.P[1] + a, d.R[1] + r, idesc, 1u);
    ptx::mma_f16(corr, d.P[0] + a, d.R[2] + r, idesc, 1u);
    ptx::mma_f16(corr, d.P[2] + a, d.R[0] + r, idesc, 1u);
  }
}

// Persistent GEMM: each CTA walks output units u = blockIdx.x, + gridDim.x, ...
// A unit is one (M block, window block) tile of one problem: of the single problem `one`
// (M block u % nMB, window block u / nMB), or, when `many` is given, of the problem whose
// unit range holds u (a multi-problem launch: every problem of a batch advances by one step
// in one launch). Two TMEM accumulator sets alternate between tiles, so the epilogue of one
// tile overlaps the MMAs of the next.
template <int BN, int NP, bool MULTI>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    split_gemm_kernel(const __grid_constant__ SplitProblem one, const SplitProblem* __restrict__ many, int nprob,
                      int nunits_many, int parity, int* err, unsigned epoch) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int STAGES = Shape<BN, NP>::STAGES, STAGE_BYTES = Shape<BN, NP>::STAGE_BYTES;
  constexpr int B_BYTES = Shape<BN, NP>::B_BYTES, NBUF = Shape<BN, NP>::NBUF;
  constexpr int R_OFF = NP * A_BYTES;  // r pieces follow the P pieces in a stage
  // [stage][P_int, P2, (P3) (A_BYTES each), r_int, r2, (r3) (B_BYTES each)]
  uint8_t* tiles = smem;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + RING_BYTES);
  // NG load barriers per stage: two pieces complete separately (the main product starts on the
  // first); three pieces complete together
  constexpr int NG = NP == 2 ? 2 : 1;
  uint64_t* full = bars;                 // [STAGES][NG] stage loaded (NG = 2: piece q loaded)
  uint64_t* empty = bars + STAGES * NG;  // [STAGES] stage released by the MMA issuer
  constexpr bool DRAIN = NP == 3;
  static_assert(!DRAIN || BN == 128, "drained correction: main[2] + corr[2] of 128 columns fill TMEM");
  uint64_t* accf = empty + STAGES;       // [2] accumulator set (main) ready (DRAIN: [0] only)
  uint64_t* acce = accf + 2;             // [2] accumulator set (main) drained (DRAIN: [0] only)
  uint64_t* cf = acce + 2;               // DRAIN: [3] correction buffer ready
  uint64_t* ce = cf + 3;                 // DRAIN: [3] correction buffer free again
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ce + 3);
  __shared__ volatile int s_abort;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int unit0 = int(blockIdx.x);
  const int nunit_step = int(gridDim.x);
  const int nunits = MULTI ? nunits_many : one.g.nMB * one.g.nNB;
  // unit -> problem and its tile (one problem: the by-value parameter, addressed statically)
  auto locate = [&](int u, int& lu) -> const SplitProblem* {
    if constexpr (!MULTI) {
      lu = u;
      return &one;
    }
    int lo = 0, hi = nprob - 1;  // last problem with unit0 <= u
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (many[mid].g.unit0 <= u) lo = mid;
      else hi = mid - 1;
    }
    lu = u - many[lo].g.unit0;
    return many + lo;
  };
  auto tile_of = [&](const GemmGeom& g, int lu, int& m0, int& tx0, int& ty0) {
    const int mb = lu % g.nMB;
    const int nb = lu / g.nMB;
    m0 = mb * BM;
    tx0 = (nb % g.nbx) * g.BNx;
    ty0 = (nb / g.nbx) * g.BNy;
  };
  // Work items (segments: unit u, window rows kb0 .. kb1 - 1; kb1 = -1: all rows of the unit).
  // Without balance: whole units u = unit0, + step, ... With balance (one problem whose unit
  // count is not a multiple of the grid): the full waves' units as before, then the window rows
  // of the remaining units, laid end to end, in equal consecutive ranges, one per CTA; a unit
  // whose rows fall to several CTAs is finished by the CTA holding its first rows (which it
  // reaches last), after the others have stored the folded sums of their rows.
  const bool balanced = !MULTI && one.g.balance;
  const int waves = nunits / nunit_step;
  const int tail0 = waves * nunit_step;  // first unit of the partial wave
  const int64_t tail_rows = int64_t(nunits - tail0) * one.g.Wy;
  auto range_start = [&](int c) { return int64_t(c) * tail_rows / nunit_step; };
  struct Cur {
    int w;      // whole units taken
    int64_t q;  // next tail row (balance) or next unit (no balance)
  };
  auto next_seg = [&](Cur& cur, int& u, int& kb0, int& kb1) -> bool {
    if (!balanced) {
      if (cur.q >= nunits) return false;
      u = int(cur.q);
      kb0 = 0;
      kb1 = -1;
      cur.q += nunit_step;
      return true;
    }
    if (cur.w < waves) {
      u = unit0 + cur.w * nunit_step;
      kb0 = 0;
      kb1 = -1;
      ++cur.w;
      return true;
    }
    const int64_t q1 = range_start(unit0 + 1);
    if (cur.q >= q1) return false;
    const int Wy = one.g.Wy;
    u = tail0 + int(cur.q / Wy);
    kb0 = int(cur.q % Wy);
    kb1 = int(kb0 + q1 - cur.q < Wy ? kb0 + q1 - cur.q : Wy);
    cur.q += kb1 - kb0;
    return true;
  };
  const Cur cur0{0, balanced ? range_start(unit0) : int64_t(unit0)};

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < STAGES; ++s) {
      for (int q = 0; q < NG; ++q) ptx::mbar_init(&full[s * NG + q], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(&accf[b], 1);
      ptx::mbar_init(&acce[b], EPI_WARPS);
    }
    for (int b = 0; b < 3; ++b) {
      ptx::mbar_init(&cf[b], 1);
      ptx::mbar_init(&ce[b], EPI_WARPS);
    }
    ptx::fence_barrier_init();
    if (!MULTI) {
      for (int q = 0; q < NP; ++q) ptx::tma_prefetch_desc(&one.tm[3 + q]);
    }
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, TMEM_COLS);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // the set-up above may overlap the residual kernel's tail; everything below reads its output
  pdl_wait_and_release();
  if (threadIdx.x == 0) {
    // max|r| of this step's parity has been consumed by the residual kernel; clear it for
    // the next-but-one step (no other kernel touches it while this one runs)
    if (!MULTI) {
      if (blockIdx.x == 0) one.g.rmax[parity] = 0u;
    } else {
      for (int i = int(blockIdx.x); i < nprob; i += int(gridDim.x)) many[i].g.rmax[parity] = 0u;
    }
  }

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int it = 0, issued = 0;
      Cur cur = cur0;
      int u, kb0, kb1;
      while (!s_abort && next_seg(cur, u, kb0, kb1)) {
        int lu;
        const SplitProblem* pr = locate(u, lu);
        const GemmGeom& g = pr->g;
        if (kb1 < 0) kb1 = g.Wy;
        int m0, tx0, ty0;
        tile_of(g, lu, m0, tx0, ty0);
        for (int kb = kb0; kb < kb1; ++kb, ++it) {
          const int s = it % STAGES;
          const uint32_t use = it / STAGES;
          if (it >= STAGES && !ptx::mbar_wait(&empty[s], (use & 1) ^ 1, WAIT_NS)) {
            atomicExch(err, ERR_TIMEOUT_PRODUCER);
            s_abort = 1;
            break;
          }
          if (s_abort) break;
          uint8_t* st = tiles + s * STAGE_BYTES;
          // piece q of the stage (its P tile and its residual tile, bnp window rows) completes on
          // its own barrier, so the MMAs on the first pieces start while the later ones stream.
          // (TMA lands each row's kx columns at their places in the 128-byte swizzled row; the
          // rest of the row is never read: the MMAs take ceil(Wx / 16) K steps of 16)
          // a piece: its P tile (one bulk copy of BM * kx * 2 bytes, the unswizzled image) and
          // its window tile (bnp TMA rows of kx columns)
          const uint32_t piece_bytes = uint32_t((BM + g.bnp) * g.kx * 2);
          const __half* ptile = g.Pt + (int64_t(m0 / BM) * g.Wy + kb) * NP * (BM * g.kx);
          const bool fault = g.fault && blockIdx.x == 0 && it == 0;  // test hook: bytes never arrive
          for (int q = 0; q < NG; ++q) ptx::mbar_arrive_expect_tx(&full[s * NG + q], piece_bytes * (NP / NG));
#pragma unroll
          for (int q = 0; q < NP; ++q) {
            if (fault) continue;
            uint64_t* bar = &full[s * NG + (NG == 1 ? 0 : q)];
            ptx::bulk_load(st + q * A_BYTES, ptile + q * (BM * g.kx), uint32_t(BM * g.kx * 2), bar);
            ptx::tma_load_4d(st + R_OFF + q * B_BYTES, &pr->tm[3 + q], bar, 0, tx0, kb, ty0);
          }
          issued = it + 1;
        }
      }
      // every copy this thread issued into this CTA has landed before the CTA may exit
      for (int k = (issued > STAGES ? issued - STAGES : 0); k < issued; ++k)
        for (int q = 0; q < NG; ++q) ptx::mbar_wait(&full[(k % STAGES) * NG + q], (k / STAGES) & 1, WAIT_NS);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    // TMEM columns: without DRAIN, set b = [main | corr] at b * 2BN (two sets alternate between
    // tiles); with DRAIN, main at 0 and three correction buffers at BN, 2BN, 3BN used in turn,
    // each collecting drain_rows window rows before the epilogue takes it. The epilogue folds a
    // tile's main sum into its last correction buffer and frees main at once.
    if (lane == 0) {
      // The issue loop is kept short: a tcgen05.mma costs this thread tens of cycles to issue,
      // about as long as an N = 128 product takes on the tensor pipe, so descriptors are set
      // up once per tile and only advanced per stage and K step.
      bool ok = true;
      int lt = 0, kc = 0;
      int s = 0;         // ring slot of the next stage
      uint32_t ph = 0;   // its fill phase
      int cj = 0;        // DRAIN: correction buffer of the current row group (kc % 3)
      Cur cur = cur0;
      int u, kb0, kb1;
      const uint32_t tiles_addr = ptx::smem_u32(tiles);
      for (; ok && next_seg(cur, u, kb0, kb1); ++lt) {
        int lu;
        const GemmGeom& g = locate(u, lu)->g;
        if (kb1 < 0) kb1 = g.Wy;
        const int ksteps = (g.Wx + 15) / 16, dr = DRAIN ? g.drain_rows : 1;
        const uint32_t idesc = ptx::idesc_f16_f32(BM, g.bnp);  // N = this problem's window block
        const int nbuf = DRAIN ? 1 : NBUF;
        const int b = lt % nbuf;
        if (lt >= nbuf) {
          if (!ptx::mbar_wait(&acce[b], ((lt / nbuf) - 1) & 1, WAIT_NS)) { ok = false; break; }
          ptx::tc_fence_after();
        }
        const uint32_t main = DRAIN ? tmem : tmem + b * 2 * BN;
        uint32_t corr = main + BN;
        // stage-0 descriptors of the pieces. P tiles: unswizzled core matrices (K-adjacent
        // 128 B apart, row groups kx * 16 B apart); residual tiles: 128-byte swizzled rows.
        // Stage s adds s * STAGE_BYTES to the (16-byte unit) address field.
        const uint32_t sbo = uint32_t(g.kx) * 16u;
        StageDesc d0;
        d0.P[0] = ptx::plain_kmajor_desc(tiles_addr, 128, sbo);
        d0.P[1] = d0.P[0] + uint64_t(A_BYTES >> 4);
        d0.P[2] = d0.P[0] + uint64_t(2 * A_BYTES >> 4);  // NP == 3 only
        d0.R[0] = ptx::sw128_kmajor_desc(tiles_addr + R_OFF);
        d0.R[1] = d0.R[0] + uint64_t(B_BYTES >> 4);
        d0.R[2] = d0.R[0] + uint64_t(2 * B_BYTES >> 4);  // NP == 3 only
        int gpos = 0;  // DRAIN: window row within its row group
        for (int kb = kb0; kb < kb1; ++kb) {
          if (!ptx::mbar_wait(&full[s * NG], ph, WAIT_NS)) { ok = false; break; }
          const bool group_first = DRAIN && gpos == 0;
          const bool group_last = DRAIN && (gpos == dr - 1 || kb == kb1 - 1);
          if (group_first) {
            if (kc >= 3 && !ptx::mbar_wait(&ce[cj], ((kc / 3) - 1) & 1, WAIT_NS)) { ok = false; break; }
            corr = tmem + (1 + cj) * BN;
          }
          ptx::tc_fence_after();
          const uint64_t sd = uint64_t(s) * uint64_t(STAGE_BYTES >> 4);
          StageDesc d;
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            d.P[q] = d0.P[q] + sd;
            d.R[q] = d0.R[q] + sd;
          }
          const uint32_t acc0 = kb > kb0 ? 1u : 0u;  // the tile's first product starts the sum
          // ceil(Wx / 16) K steps: P is zero beyond Wx in each padded window row.
          if constexpr (NP == 2) {
            // two pieces: the main product on piece 0 while piece 1 still streams, then the
            // three corrections (GB300, 2048^2: 65.8 us per launch against 70.7 us waiting for
            // the whole stage)
            switch (ksteps) {
              case 1: issue_main<1>(main, d, idesc, acc0); break;
              case 2: issue_main<2>(main, d, idesc, acc0); break;
              case 3: issue_main<3>(main, d, idesc, acc0); break;
              default: issue_main<4>(main, d, idesc, acc0); break;
            }
            if (!ptx::mbar_wait(&full[s * NG + 1], ph, WAIT_NS)) { ok = false; break; }
            ptx::tc_fence_after();
            switch (ksteps) {
              case 1: issue_corr2<1>(corr, d, idesc, acc0); break;
              case 2: issue_corr2<2>(corr, d, idesc, acc0); break;
              case 3: issue_corr2<3>(corr, d, idesc, acc0); break;
              default: issue_corr2<4>(corr, d, idesc, acc0); break;
            }
          } else {
            // three pieces: the whole stage (waited above), then the six products of each K step
            // in turn (issuing them piece by piece measured 152 us against 133 us per 2048^2
            // launch)
            // DRAIN: each row group starts a fresh correction sum
            const uint32_t cacc0 = DRAIN ? (group_first ? 0u : 1u) : acc0;
            switch (ksteps) {
              case 1: issue_six<1>(main, corr, d, idesc, acc0, cacc0); break;
              case 2: issue_six<2>(main, corr, d, idesc, acc0, cacc0); break;
              case 3: issue_six<3>(main, corr, d, idesc, acc0, cacc0); break;
              default: issue_six<4>(main, corr, d, idesc, acc0, cacc0); break;
            }
          }
          ptx::mma_commit(&empty[s]);
          if (group_last) {
            ptx::mma_commit(&cf[cj]);
            ++kc;
            cj = cj == 2 ? 0 : cj + 1;
          }
          if (DRAIN) gpos = gpos + 1 == dr ? 0 : gpos + 1;
          if (++s == STAGES) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (ok) ptx::mma_commit(&accf[b]);
      }
      if (!ok) {
        atomicExch(err, ERR_TIMEOUT_MMA);
        s_abort = 1;
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int lane_base = 32 * (warp & 3);  // tcgen05.ld: a warp reaches lane quarter warp % 4
    const int row = lane_base + lane;       // TMEM lane = owner row within the M block
    const int half = (warp - 2) >> 2;       // this warp's 32-column blocks: 2 lb + half
    constexpr int NLB = BN / 64;            // 32-column blocks per warp
    int lt = 0, kc = 0;
    Cur cur = cur0;
    int u, kb0, kb1;
    for (; next_seg(cur, u, kb0, kb1); ++lt) {
      int lu;
      const GemmGeom& g = locate(u, lu)->g;
      if (kb1 < 0) kb1 = g.Wy;
      const int nbuf = DRAIN ? 1 : NBUF;
      const int b = lt % nbuf;
      float cs[DRAIN ? BN / 2 : 1];  // DRAIN: correction summed over row groups (this warp's columns)
      int fold = 0;                  // DRAIN: the correction buffer of the tile's last row group
      if constexpr (DRAIN) {
#pragma unroll
        for (int i = 0; i < BN / 2; ++i) cs[i] = 0.0f;
        bool ok = true;
        const int ngroups = (kb1 - kb0 + g.drain_rows - 1) / g.drain_rows;
        for (int gi = 0; gi < ngroups; ++gi, ++kc) {
          const int j = kc % 3;
          if (s_abort || !ptx::mbar_wait(&cf[j], (kc / 3) & 1, WAIT_NS)) { ok = false; break; }
          ptx::tc_fence_after();
          const uint32_t tc = tmem + (uint32_t(lane_base) << 16) + uint32_t((1 + j) * BN);
#pragma unroll
          for (int lb = 0; lb < NLB; ++lb) {  // 32 columns per load round trip
            const int col0 = (2 * lb + half) * 32;
            if (col0 >= g.bnp) break;        // (columns past bnp hold nothing of this unit)
            uint32_t r[32];
            ptx::tmem_ld_32x32b_x32(tc + col0, r);
#pragma unroll
            for (int i = 0; i < 32; ++i) cs[lb * 32 + i] = __fadd_rn(cs[lb * 32 + i], __uint_as_float(r[i]));
          }
          if (gi + 1 < ngroups) {  // the last buffer stays held: it receives the folded sum
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&ce[j]);
          } else {
            fold = j;
          }
        }
        if (!ok) {
          atomicExch(err, ERR_TIMEOUT_EPI);
          break;
        }
      }
      if (!ptx::mbar_wait(&accf[b], (lt / nbuf) & 1, WAIT_NS)) {
        atomicExch(err, ERR_TIMEOUT_EPI);
        break;
      }
      ptx::tc_fence_after();
      const uint32_t t_lane = tmem + (uint32_t(lane_base) << 16) + uint32_t(DRAIN ? 0 : b * 2 * BN);
      int m0, tx0, ty0;
      tile_of(g, lu, m0, tx0, ty0);
      const int ii = m0 + row;
      const bool row_in = ii < g.M;  // the last M block may extend past the owner rows
      const float oscale = pow2f(-((row_in ? g.eP[ii] : 0) + g.escale[parity]));
      const int iy = row_in ? ii / g.Tx : 0, ix = row_in ? ii % g.Tx : 0;
      const int rowbase = iy * g.nx + ix;
      float* __restrict__ uh = g.uh;
      float* __restrict__ ul = g.ul;
      // one batch of 16 windows (columns c0 .. c0 + 15): y = (main + corr) 2^-(eP_i + er) added
      // into the owner nodes
      auto batch = [&](int c0, const float (&vm)[16], const float (&vc)[16]) {
        // all 32 state loads of this batch go out before any store (the stores go through
        // the same pointers, so the compiler would otherwise keep them in program order)
        int node[16];
        float a[16], al[16];
        uint32_t inside = 0;  // windows of this batch that exist (blocks may overhang the grid)
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int n = c0 + i;
          const int ty = ty0 + (n >> g.lbx), tx = tx0 + (n & ((1 << g.lbx) - 1));
          const bool in = row_in && ty < g.nty && tx < g.ntx;
          inside |= uint32_t(in) << i;
          node[i] = in ? (ty * g.Ty) * g.nx + tx * g.Tx + rowbase : rowbase;
          a[i] = uh[node[i]];
          al[i] = ul[node[i]];
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float y = __fmul_rn(__fadd_rn(vm[i], vc[i]), oscale);
          // (u_hi, u_lo) += y in float-float
          const ffv s = two_sum(a[i], y);
          const float lo = __fadd_rn(al[i], s.l);
          const float hi2 = __fadd_rn(s.h, lo);
          if (inside >> i & 1u) {
            uh[node[i]] = hi2;
            ul[node[i]] = __fsub_rn(lo, __fsub_rn(hi2, s.h));
          }
        }
      };
      if constexpr (DRAIN) {
        // balance: a part that does not start the unit stores its folded sums for the CTA
        // holding the unit's first rows, which adds the later parts' sums (in row order)
        const bool whole = kb0 == 0 && kb1 == g.Wy;
        const int ew = warp - 2;  // this epilogue warp's flag
        if (!whole && kb0 > 0) {
          float* dst = g.part + int64_t(blockIdx.x) * BN * BM + row;
#pragma unroll
          for (int lb = 0; lb < NLB; ++lb) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              const int col0 = (2 * lb + half) * 32 + c * 16;
              if (col0 >= g.bnp) break;
              float vm[16];
              ptx::tmem_ld_32x32b_x16(t_lane + col0, vm);
#pragma unroll
              for (int i = 0; i < 16; ++i) dst[(col0 + i) * BM] = __fadd_rn(vm[i], cs[(lb * 32 + c * 16 + i) % (DRAIN ? BN / 2 : 1)]);
            }
          }
          ptx::tc_fence_before();
          __syncwarp();
          if (lane == 0) {
            ptx::mbar_arrive(&acce[b]);
            ptx::mbar_arrive(&ce[fold]);
          }
          __threadfence();
          __syncwarp();
          if (lane == 0) ptx::st_release_gpu(g.flags + blockIdx.x * EPI_WARPS + ew, epoch);
          continue;
        }
        // the CTAs holding this unit's later rows (balance, a part starting the unit)
        int partner0 = 0, npartners = 0;
        if (!whole) {
          const int64_t base = int64_t(u - tail0) * g.Wy;
          partner0 = int(blockIdx.x) + 1;
          // (every CTA's range holds at least one row: the host balances only then)
          for (int c = partner0; c < nunit_step && range_start(c) < base + g.Wy; ++c) {
            ++npartners;
            if (lane == 0 && !ptx::wait_flag_gpu(g.flags + c * EPI_WARPS + ew, epoch, WAIT_NS))
              atomicExch(err, ERR_TIMEOUT_EPI);
          }
          __syncwarp();
        }
        // fold main + correction (FP32, as without the drain) into the last row group's
        // correction buffer and free main at once, so the next tile's MMAs start during the
        // scatter below; that buffer is released after the scatter
        const uint32_t t_fold = tmem + (uint32_t(lane_base) << 16) + uint32_t((1 + fold) * BN);
#pragma unroll
        for (int lb = 0; lb < NLB; ++lb) {  // unrolled: cs is indexed statically
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int col0 = (2 * lb + half) * 32 + c * 16;
            if (col0 >= g.bnp) break;
            float vm[16];
            ptx::tmem_ld_32x32b_x16(t_lane + col0, vm);
#pragma unroll
            for (int i = 0; i < 16; ++i) vm[i] = __fadd_rn(vm[i], cs[(lb * 32 + c * 16 + i) % (DRAIN ? BN / 2 : 1)]);
            for (int p = 0; p < npartners; ++p) {
              const float* src = g.part + int64_t(partner0 + p) * BN * BM + row + int64_t(col0) * BM;
#pragma unroll
              for (int i = 0; i < 16; ++i) vm[i] = __fadd_rn(vm[i], __ldcg(src + i * BM));
            }
            ptx::tmem_st_32x32b_x16(t_fold + col0, vm);
          }
        }
        ptx::tmem_wait_st();
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&acce[b]);
        const float zero[16] = {};
#pragma unroll 1
        for (int lb = 0; lb < NLB; ++lb)
          for (int c = 0; c < 2; ++c) {
            const int col0 = (2 * lb + half) * 32 + c * 16;
            if (col0 >= g.bnp) break;
            float vm[16];
            ptx::tmem_ld_32x32b_x16(t_fold + col0, vm);
            batch(col0, vm, zero);
          }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&ce[fold]);
        continue;
      } else {
#pragma unroll 1
        for (int lb = 0; lb < NLB; ++lb)
          for (int c = 0; c < 2; ++c) {
            const int col0 = (2 * lb + half) * 32 + c * 16;
            if (col0 >= g.bnp) break;
            float vm[16], vc[16];
            ptx::tmem_ld_32x32b_x16(t_lane + col0, vm);
            ptx::tmem_ld_32x32b_x16(t_lane + BN + col0, vc);
            batch(col0, vm, vc);
          }
      }
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&acce[b]);
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, TMEM_COLS);
  }
}

using GemmKernel = void (*)(SplitProblem, const SplitProblem*, int, int, int, int*, unsigned);

int gemm_threads(int) { return GEMM_THREADS; }

// The instantiated (tile width, pieces) combinations: BN 256 with two pieces for large tile
// grids, BN 128 otherwise.
GemmKernel gemm_kernel_for(int bn, int np, bool multi = false) {
  if (multi) {
    if (np == 3) return split_gemm_kernel<128, 3, true>;
    return bn == 256 ? split_gemm_kernel<256, 2, true> : split_gemm_kernel<128, 2, true>;
  }
  if (np == 3) return split_gemm_kernel<128, 3, false>;
  return bn == 256 ? split_gemm_kernel<256, 2, false> : split_gemm_kernel<128, 2, false>;
}

}  // namespace

struct SplitPlan {
  int Ty = 0, Tx = 0, Hy = 0, Hx = 0, Wy = 0, Wx = 0, nty = 0, ntx = 0, M = 0, BNx = 0, BNy = 0;
  int pitch = 0, prow = 0, nsm = 0;
  int np = 2;        // FP16 pieces per operand: 2 (four products) or 3 (six products)
  int bn = 128;      // windows per CTA tile (256 for large tile grids with two pieces)
  int nbx = 0, nby = 0;  // window blocks per grid row / column (the last ones may overhang)
  ResParams rp{};
  float* d_uh = nullptr;
  float* d_ul = nullptr;
  __half* d_Rint = nullptr;
  __half* d_R2 = nullptr;
  __half* d_R3 = nullptr;
  __half* d_Pt = nullptr;  // P pieces as pre-swizzled tiles [M blocks][Wy][np][BM x KB]
  int* d_eP = nullptr;
  double* d_S = nullptr;
  unsigned* d_rmax = nullptr;
  int* d_escale = nullptr;
  int* d_err = nullptr;
  int* d_rb = nullptr;
  SplitProblem prob{};  // tensor maps and GEMM geometry
  float* d_part = nullptr;     // balance: per CTA, one stored tile part (BN x BM floats)
  unsigned* d_flags = nullptr; // balance: per CTA and epilogue warp, the epoch of its part
  unsigned epoch = 0;          // GEMM launches so far (the flags' values)
  int packed_gen = -1;
};

// log2 of a power of two
static int log2_exact(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

// Windows of a CTA tile form a BNx x BNy rectangle of the tile grid with BNx*BNy = bn (both
// powers of two). Blocks may overhang the grid at its right and bottom edges (TMA zero-fills
// those windows and the epilogue skips them), so the shape with the fewest blocks wins (ties:
// the wider one).
static void group_tiles(int64_t ntx, int64_t nty, int bn, int* bnx, int* bny) {
  int64_t best = -1;
  for (int x = bn; x >= 1; x /= 2) {
    const int y = bn / x;
    const int64_t blocks = ((ntx + x - 1) / x) * ((nty + y - 1) / y);
    if (best < 0 || blocks < best) {
      best = blocks;
      *bnx = x;
      *bny = y;
    }
  }
}

bool split_eligible(const lem_ctx* ctx) {
  const lem_problem_desc& d = ctx->desc;
  if (d.ndim != 2 || d.mode != LEM_MODE_PHI || d.reaction || d.coef_stride != 0) return false;
  if (d.bc[0] != LEM_BC_PERIODIC || d.bc[1] != LEM_BC_PERIODIC) return false;
  if (ctx->classes.size() != 1) return false;
  const int Ty = d.tile[0], Tx = d.tile[1], Hx = d.overlap[1];
  if (ctx->ny % Ty || ctx->nx % Tx) return false;
  const ClassDesc& c = ctx->classes[0];
  if (c.whole[0] || c.whole[1]) return false;
  const int Wx = Tx + 2 * Hx;
  if (Wx > KB || Tx % 8) return false;  // TMA: a window row fits one 128-byte row; 16-byte strides
  return true;
}

// cuTensorMapEncodeTiled, resolved through the runtime so that liblem.so does not link
// the driver library (it loads on machines without a GPU driver, e.g. for the host planner).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// FP16 tiled tensor map with a 128-byte (default) or 64-byte swizzle: the canonical K-major
// layouts of the tcgen05 operand tiles
lem_status encode_f16_map(CUtensorMap* m, void* base, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
                          const cuuint32_t* box, const char* what, int swizzle_bytes) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return fail(LEM_ECUDA, "cuTensorMapEncodeTiled unavailable");
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, cuuint32_t(rank), base, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE,
                  swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(LEM_ECUDA, std::string("cuTensorMapEncodeTiled failed for ") + what +
                                                    " (CUresult " + std::to_string(int(r)) + ")");
  return LEM_OK;
}

lem_status split_prepare(lem_ctx* ctx) {
  SplitPlan* sp = new SplitPlan();
  ctx->split = sp;
  const lem_problem_desc& d = ctx->desc;
  sp->Ty = d.tile[0]; sp->Tx = d.tile[1]; sp->Hy = d.overlap[0]; sp->Hx = d.overlap[1];
  sp->Wy = sp->Ty + 2 * sp->Hy; sp->Wx = sp->Tx + 2 * sp->Hx;
  sp->nty = int(ctx->ny / sp->Ty); sp->ntx = int(ctx->nx / sp->Tx);
  sp->M = sp->Ty * sp->Tx;
  sp->np = d.prec == LEM_PREC_SPLIT_FAST ? 2 : 3;
  // 256-wide tiles when they do not waste more than they save on mostly-empty edge blocks
  // (two pieces only: a stage of three 256-wide pieces leaves room for one stage)
  sp->bn = sp->np == 2 && int64_t(sp->ntx) * sp->nty >= 1024 ? 256 : 128;
  group_tiles(sp->ntx, sp->nty, sp->bn, &sp->BNx, &sp->BNy);
  sp->nbx = int((sp->ntx + sp->BNx - 1) / sp->BNx);
  sp->nby = int((sp->nty + sp->BNy - 1) / sp->BNy);
  LEM_CUDA_TRY(cudaDeviceGetAttribute(&sp->nsm, cudaDevAttrMultiProcessorCount, ctx->device));
  // padded residual: rows ny + 2Hy, row pitch covers the last 64-wide window row read
  sp->prow = int(ctx->ny) + 2 * sp->Hy;
  int need = std::max<int>(int(ctx->nx) + 2 * sp->Hx, (sp->ntx - 1) * sp->Tx + KB);
  sp->pitch = (need + 7) / 8 * 8;
  // stencil constants (dt-scaled) as float pairs
  const std::vector<double>& hc = ctx->h_coef;  // dt-scaled constant stencil
  double csum = 0.0;
  for (int k = 0; k < 5; ++k) {
    csum += hc[k];
    sp->rp.c_hi[k] = float(hc[k]);
    sp->rp.c_lo[k] = float(hc[k] - double(sp->rp.c_hi[k]));
  }
  sp->rp.csum_hi = float(csum);
  sp->rp.csum_lo = float(csum - double(sp->rp.csum_hi));
  sp->rp.has_lo = sp->rp.csum_lo != 0.0f;
  for (int k = 0; k < 5; ++k) sp->rp.has_lo |= sp->rp.c_lo[k] != 0.0f;
  sp->rp.ny = int(ctx->ny); sp->rp.nx = int(ctx->nx); sp->rp.Hy = sp->Hy; sp->rp.Hx = sp->Hx;
  sp->rp.pitch = sp->pitch; sp->rp.prow = sp->prow;
  sp->rp.rb = nullptr;  // device value, set from the packed propagator in split_pack
  const size_t npts = size_t(ctx->npts);
  const size_t rbytes = sizeof(__half) * size_t(sp->prow) * sp->pitch;
  // P pieces padded to whole 128-row M blocks (zero rows past Ty*Tx)
  const int Mpad = (sp->M + BM - 1) / BM * BM;
  const size_t pbytes = sizeof(__half) * size_t(Mpad) * sp->Wy * ((sp->Wx + 15) / 16 * 16) * sp->np;
  LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&sp->d_uh), sizeof(float) * npts));
  LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&sp->d_ul), sizeof(float) * npts));
  LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&sp->d_Rint), rbytes));
  LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&sp->d_R2), rbytes));
  LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&sp->d_Pt), pbytes));
  if (sp->np == 3) {
    LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&sp->d_R3), rbytes));
    LEM_CUDA_TRY(cudaMemsetAsync(sp->d_R3, 0, rbytes, ctx->stream));
  }
  LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&sp->d_eP), sizeof(int) * sp->M));
  LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&sp->d_S), sizeof(double) * sp->M));
  LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&sp->d_rmax), sizeof(unsigned) * 2));
  LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&sp->d_escale), sizeof(int) * 2));
  LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&sp->d_err), sizeof(int)));
  LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&sp->d_rb), sizeof(int)));
  sp->rp.rb = sp->d_rb;
  LEM_CUDA_TRY(cudaMemsetAsync(sp->d_Pt, 0, pbytes, ctx->stream));
  LEM_CUDA_TRY(cudaMemsetAsync(sp->d_Rint, 0, rbytes, ctx->stream));
  LEM_CUDA_TRY(cudaMemsetAsync(sp->d_R2, 0, rbytes, ctx->stream));
  LEM_CUDA_TRY(cudaMemsetAsync(sp->d_err, 0, sizeof(int), ctx->stream));
  LEM_CUDA_TRY(cudaFuncSetAttribute(gemm_kernel_for(sp->bn, sp->np), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    SMEM_BYTES));
  LEM_CUDA_TRY(cudaFuncSetAttribute(gemm_kernel_for(sp->bn, sp->np, true),
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
  // residual pieces through a 4D overlapping view of the padded array: (wx, tx, wy, ty) ->
  // R[ty*Ty + wy][tx*Tx + wx] (tm[3..5]; tm[0..2] unused: P tiles come by bulk copy)
  {
    SplitProblem& pr = sp->prob;
    // with two pieces the third map aliases the second (never loaded)
    __half* rbase[3] = {sp->d_Rint, sp->d_R2, sp->np == 3 ? sp->d_R3 : sp->d_R2};
    // only the window row's used columns: kx = Wx rounded up to 16 (a 96-byte box for 48-wide
    // windows lands at the same swizzled places as the first 48 columns of a 128-byte row)
    const cuuint32_t kx = cuuint32_t((sp->Wx + 15) / 16 * 16);
    cuuint64_t rd[4] = {KB, cuuint64_t(sp->ntx), cuuint64_t(sp->Wy), cuuint64_t(sp->nty)};
    cuuint64_t rs[3] = {cuuint64_t(sp->Tx) * 2, cuuint64_t(sp->pitch) * 2, cuuint64_t(sp->Ty) * sp->pitch * 2};
    cuuint32_t rbox[4] = {kx, cuuint32_t(sp->BNx), 1, cuuint32_t(sp->BNy)};
    for (int k = 0; k < 3; ++k) LEM_TRY(encode_f16_map(&pr.tm[3 + k], rbase[k], 4, rd, rs, rbox, "residual slice"));
  }
  GemmGeom& g = sp->prob.g;
  g.Wy = sp->Wy; g.Wx = sp->Wx; g.Ty = sp->Ty; g.Tx = sp->Tx; g.nx = int(ctx->nx);
  g.BNx = sp->BNx; g.BNy = sp->BNy; g.ntx = sp->ntx; g.nty = sp->nty; g.M = sp->M;
  g.lbx = log2_exact(sp->BNx);
  g.nbx = sp->nbx; g.nMB = (sp->M + BM - 1) / BM; g.nNB = sp->nbx * sp->nby; g.bnp = sp->bn;
  // three pieces: drain the correction after about 64 K elements (a 48- or 64-wide row, two
  // rows of up to 32, four of 16), so small windows do not pay a handshake per short row
  g.kx = (sp->Wx + 15) / 16 * 16;
  g.drain_rows = std::max(1, 64 / g.kx);
  if (const char* e = std::getenv("LEM_SPLIT_DRAIN_ROWS")) g.drain_rows = std::max(1, std::atoi(e));  // tuning knob
  g.unit0 = 0;
  {
    const char* f = std::getenv("LEM_FAULT");
    g.fault = f && std::strcmp(f, "timeout") == 0;
  }
  g.Pt = sp->d_Pt;
  // balance the last, partial wave (three pieces, at least one full wave, and at least 8 of its
  // window rows per CTA, so every CTA's range is a real part; LEM_SPLIT_BALANCE=0 keeps whole
  // units, for comparison)
  {
    const int units = g.nMB * g.nNB;
    const int64_t tail_rows = int64_t(units % sp->nsm) * g.Wy;
    const char* e = std::getenv("LEM_SPLIT_BALANCE");
    g.balance = sp->np == 3 && units > sp->nsm && units % sp->nsm != 0 && tail_rows >= int64_t(8) * sp->nsm &&
                !(e && std::strcmp(e, "0") == 0);
    g.part = nullptr;
    g.flags = nullptr;
    if (g.balance) {
      LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&sp->d_part), sizeof(float) * size_t(sp->nsm) * sp->bn * BM));
      LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&sp->d_flags), sizeof(unsigned) * size_t(sp->nsm) * EPI_WARPS));
      LEM_CUDA_TRY(cudaMemsetAsync(sp->d_flags, 0, sizeof(unsigned) * size_t(sp->nsm) * EPI_WARPS, ctx->stream));
      g.part = sp->d_part;
      g.flags = sp->d_flags;
    }
  }
  g.eP = sp->d_eP; g.escale = sp->d_escale; g.rmax = sp->d_rmax; g.uh = sp->d_uh; g.ul = sp->d_ul;
  cudaFuncAttributes fa{};
  LEM_CUDA_TRY(cudaFuncGetAttributes(&fa, gemm_kernel_for(sp->bn, sp->np)));
  if (fa.maxThreadsPerBlock < gemm_threads(sp->np))
    return fail(LEM_ECUDA, "split GEMM kernel cannot launch " + std::to_string(gemm_threads(sp->np)) + " threads (" +
                               std::to_string(fa.numRegs) + " registers per thread)");
  return LEM_OK;
}

// Pack the FP64 propagator into P_int + P2 and choose the residual integer range rb so that
// max_i sum_k |P_int[i,k]| * 2^rb < 2^24 (the main product's exactness bound).
static lem_status split_pack(lem_ctx* ctx) {
  SplitPlan* sp = ctx->split;
  cudaStream_t st = ctx->stream;
  pack_p_kernel<<<sp->M, 256, 0, st>>>(ctx->d_P, ctx->n_loc, sp->M, sp->Wy, sp->Wx, KB, sp->np, sp->prob.g.kx,
                                       sp->d_Pt, sp->d_eP, sp->d_S);
  choose_rb_kernel<<<1, 256, 0, st>>>(sp->d_S, sp->M, sp->d_rb, sp->d_err);
  LEM_CUDA_TRY(cudaGetLastError());
  sp->packed_gen = ctx->build_gen;
  return LEM_OK;
}

// nsteps LEM steps on a float-float state (uh, ul) already on the device. The scale of each
// step's residual pieces comes from the previous step's max|r|; the first step of a run takes
// its own (a measuring pass) unless carry_in, in which case d_carry holds the previous step's
// max|r| from an earlier run on the same state. With d_carry, the last step's max|r| is left
// there, so a run split into several calls gives the same result bit for bit as one call.
lem_status split_run(lem_ctx* ctx, float* uh, float* ul, int nsteps, unsigned* d_carry, bool carry_in,
                     const double* in64) {
  SplitPlan* sp = ctx->split;
  cudaStream_t st = ctx->stream;
  if (sp->packed_gen != ctx->build_gen) LEM_TRY(split_pack(ctx));
  const dim3 rgrid((int(ctx->nx) + 2 * sp->Hx + RTX - 1) / RTX, (sp->prow + RTY - 1) / RTY);
  LEM_CUDA_TRY(cudaMemsetAsync(sp->d_rmax, 0, sizeof(unsigned) * 2, st));
  if (carry_in && d_carry) {
    LEM_CUDA_TRY(cudaMemcpyAsync(sp->d_rmax, d_carry, sizeof(unsigned), cudaMemcpyDeviceToDevice, st));
  } else if (in64) {
    // the same measuring pass, on the FP64 state, which it converts to (uh, ul) as it goes
    residual_measure_f64_kernel<<<rgrid, 256, 0, st>>>(in64, uh, ul, sp->rp, sp->d_rmax, sp->d_escale);
    LEM_CUDA_TRY(cudaGetLastError());
  } else {
    // measure max|r| of the first step into rmax[0] (the measuring pass reads rmax[1] only
    // to form a scale it never uses)
    residual_split_kernel<<<rgrid, 256, 0, st>>>(uh, ul, sp->d_Rint, sp->d_R2, sp->d_R3, sp->rp, sp->d_rmax,
                                                 sp->d_escale, 1, 1);
    LEM_CUDA_TRY(cudaGetLastError());
  }
  SplitProblem prob = sp->prob;  // the GEMM's epilogue adds into this state
  prob.g.uh = uh;
  prob.g.ul = ul;
  // residual and GEMM launches alternate with programmatic stream serialization: each may
  // start its set-up while the previous one finishes (both kernels wait for their input)
  cudaLaunchAttribute pdl[1];
  pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  pdl[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg{};
  cfg.blockDim = dim3(gemm_threads(sp->np));
  cfg.dynamicSmemBytes = SMEM_BYTES;
  cfg.stream = st;
  cfg.gridDim = dim3(std::min(prob.g.nMB * prob.g.nNB, sp->nsm));
  cfg.attrs = pdl;
  cfg.numAttrs = 1;
  cudaLaunchConfig_t rcfg{};
  rcfg.blockDim = dim3(256);
  rcfg.gridDim = rgrid;
  rcfg.stream = st;
  rcfg.attrs = pdl;
  rcfg.numAttrs = 1;
  for (int k = 0; k < nsteps; ++k) {
    const int parity = k & 1;
    LEM_CUDA_TRY(cudaLaunchKernelEx(&rcfg, residual_split_kernel, static_cast<const float*>(uh),
                                    static_cast<const float*>(ul), sp->d_Rint, sp->d_R2, sp->d_R3, sp->rp, sp->d_rmax,
                                    sp->d_escale, parity, 0));
    cudaEvent_t stop;
    LEM_CUDA_TRY(ctx->timing_begin(&stop));
    LEM_CUDA_TRY(cudaLaunchKernelEx(&cfg, gemm_kernel_for(sp->bn, sp->np), prob,
                                    static_cast<const SplitProblem*>(nullptr), 1, 0, parity, sp->d_err, ++sp->epoch));
    ctx->timing_end(stop);
  }
  LEM_CUDA_TRY(cudaGetLastError());
  // the last step (parity (nsteps - 1) & 1) accumulated its max|r| into rmax[nsteps & 1]
  if (d_carry && nsteps > 0)
    LEM_CUDA_TRY(cudaMemcpyAsync(d_carry, sp->d_rmax + (nsteps & 1), sizeof(unsigned), cudaMemcpyDeviceToDevice, st));
  return LEM_OK;
}

// FP64 state <-> float-float state on the context stream (every float-float state the split
// kernels leave is normalised, |ul| <= ulp(uh) / 2, so the conversion to float-float of a value
// they wrote returns the same pair).
// (eight 256-thread blocks per SM)
lem_status split_to_ff(lem_ctx* ctx, const double* d_u, float* uh, float* ul) {
  f64_to_ff_kernel<<<8 * ctx->split->nsm, 256, 0, ctx->stream>>>(d_u, uh, ul, ctx->npts);
  LEM_CUDA_TRY(cudaGetLastError());
  return LEM_OK;
}

lem_status split_from_ff(lem_ctx* ctx, const float* uh, const float* ul, double* d_u) {
  ff_to_f64_kernel<<<8 * ctx->split->nsm, 256, 0, ctx->stream>>>(uh, ul, d_u, ctx->npts);
  LEM_CUDA_TRY(cudaGetLastError());
  return LEM_OK;
}

lem_status split_step(lem_ctx* ctx, double* d_u, int nsteps, bool fuse_io) {
  SplitPlan* sp = ctx->split;
  if (fuse_io && nsteps > 0) {
    LEM_TRY(split_run(ctx, sp->d_uh, sp->d_ul, nsteps, nullptr, false, d_u));
  } else {
    LEM_TRY(split_to_ff(ctx, d_u, sp->d_uh, sp->d_ul));
    LEM_TRY(split_run(ctx, sp->d_uh, sp->d_ul, nsteps, nullptr, false));
  }
  return split_from_ff(ctx, sp->d_uh, sp->d_ul, d_u);
}

// ------------------------------------------------------------------ multi-problem steps
// Every problem of a batch advances one LEM step with one residual launch and one persistent
// GEMM launch (units of all problems, the heaviest problems' units first).
struct SplitBatch {
  int n = 0, np = 2, bn = 128, nunits = 0, res_blocks = 0, conv_blocks = 0, grid = 0;
  double executed_flops = 0.0;  // MMA work of one fused GEMM launch, padding included
  SplitProblem first{};  // by-value kernel argument (unused when the array is given)
  SplitProblem* d_probs = nullptr;
  ResProblem* d_res = nullptr;
  int* d_res_first = nullptr;
  ConvProblem* d_conv = nullptr;
  int* d_conv_first = nullptr;
  int* d_err = nullptr;
};

bool split_batch_eligible(lem_ctx* const* ctxs, int n) {
  if (n <= 0 || !ctxs[0]->split) return false;
  for (int i = 0; i < n; ++i) {
    const SplitPlan* sp = ctxs[i]->split;
    if (!sp || sp->np != ctxs[0]->split->np || sp->bn != ctxs[0]->split->bn) return false;
    if (ctxs[i]->apply_path != LEM_APPLY_TC_SPLIT) return false;  // e.g. truncated propagators
    if (ctxs[i]->device != ctxs[0]->device) return false;
  }
  return true;
}

void split_batch_destroy(SplitBatch* b) {
  if (!b) return;
  cudaFree(b->d_probs); cudaFree(b->d_res); cudaFree(b->d_res_first);
  cudaFree(b->d_conv); cudaFree(b->d_conv_first); cudaFree(b->d_err);
  delete b;
}

// Windows per block of one problem in a multi-problem launch: the power of two in [16, cap]
// (cap 0: the context's own width) whose blocks cost the fewest operand bytes, NP P pieces
// plus NP residual pieces of bnp window rows per stage and block (ties: the wider). Small
// tile grids then take narrow N blocks instead of mostly empty 128-window ones.
static int batch_block_width(const SplitPlan* sp, int cap) {
  if (cap <= 0) return sp->bn;
  cap = std::min(cap, sp->bn);
  int best = sp->bn;
  int64_t best_cost = -1;
  for (int w = 16; w <= cap; w *= 2) {
    int bx = 0, by = 0;
    group_tiles(sp->ntx, sp->nty, w, &bx, &by);
    const int64_t blocks = int64_t((sp->ntx + bx - 1) / bx) * ((sp->nty + by - 1) / by);
    const int64_t kx = (sp->Wx + 15) / 16 * 16;
    const int64_t cost = blocks * int64_t(sp->np) * (BM + int64_t(w)) * kx * 2;
    if (best_cost < 0 || cost <= best_cost) {
      best_cost = cost;
      best = w;
    }
  }
  return best;
}

lem_status split_batch_prepare(lem_ctx* const* ctxs, double* const* d_states, int n, int cap, SplitBatch** out) {
  *out = nullptr;
  if (!split_batch_eligible(ctxs, n)) return fail(LEM_EINVAL, "batch is not one tensor-core split tier");
  for (int i = 0; i < n; ++i)
    if (ctxs[i]->split->packed_gen != ctxs[i]->build_gen) return fail(LEM_ENOTREADY, "split propagator not packed");
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  auto work = [&](int i) {
    const SplitPlan* sp = ctxs[i]->split;
    return int64_t(sp->Wy) * ((sp->Wx + 15) / 16);
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return work(a) > work(c); });
  SplitBatch* b = new SplitBatch();
  b->n = n;
  b->np = ctxs[0]->split->np;
  b->bn = ctxs[0]->split->bn;
  std::vector<SplitProblem> probs(n);
  std::vector<ResProblem> res(n);
  std::vector<ConvProblem> conv(n);
  std::vector<int> res_first(n), conv_first(n);
  for (int k = 0; k < n; ++k) {
    const lem_ctx* c = ctxs[order[k]];
    const SplitPlan* sp = c->split;
    probs[k] = sp->prob;
    GemmGeom& g = probs[k].g;
    const int w = batch_block_width(sp, cap);
    if (w != sp->bn) {  // narrower window blocks: their own residual tensor maps
      int bx = 0, by = 0;
      group_tiles(sp->ntx, sp->nty, w, &bx, &by);
      g.BNx = bx; g.BNy = by; g.bnp = w;
      g.lbx = log2_exact(bx);
      g.nbx = (sp->ntx + bx - 1) / bx;
      g.nNB = g.nbx * ((sp->nty + by - 1) / by);
      __half* rbase[3] = {sp->d_Rint, sp->d_R2, sp->np == 3 ? sp->d_R3 : sp->d_R2};
      cuuint64_t rd[4] = {KB, cuuint64_t(sp->ntx), cuuint64_t(sp->Wy), cuuint64_t(sp->nty)};
      cuuint64_t rs[3] = {cuuint64_t(sp->Tx) * 2, cuuint64_t(sp->pitch) * 2, cuuint64_t(sp->Ty) * sp->pitch * 2};
      cuuint32_t rbox[4] = {cuuint32_t(g.kx), cuuint32_t(bx), 1, cuuint32_t(by)};
      for (int q = 0; q < 3; ++q) {
        const lem_status e = encode_f16_map(&probs[k].tm[3 + q], rbase[q], 4, rd, rs, rbox, "residual slice");
        if (e != LEM_OK) {
          delete b;
          return e;
        }
      }
    }
    g.unit0 = b->nunits;
    b->nunits += g.nMB * g.nNB;
    b->executed_flops += 2.0 * sp->np * 2.0 * double(g.nMB) * BM * double(sp->Wy) * ((sp->Wx + 15) / 16 * 16) *
                         double(g.nNB) * g.bnp;
    ResProblem& r = res[k];
    r.p = sp->rp;
    r.uh = sp->d_uh; r.ul = sp->d_ul; r.Rint = sp->d_Rint; r.R2 = sp->d_R2; r.R3 = sp->d_R3;
    r.rmax = sp->d_rmax; r.escale = sp->d_escale;
    r.gx = (int(c->nx) + 2 * sp->Hx + RTX - 1) / RTX;
    r.block0 = res_first[k] = b->res_blocks;
    b->res_blocks += r.gx * ((sp->prow + RTY - 1) / RTY);
    ConvProblem& v = conv[k];
    v.u = d_states[order[k]]; v.uh = sp->d_uh; v.ul = sp->d_ul; v.rmax = sp->d_rmax; v.n = c->npts;
    v.block0 = conv_first[k] = b->conv_blocks;
    b->conv_blocks += int((c->npts + CONV_CHUNK - 1) / CONV_CHUNK);
  }
  b->first = probs[0];
  b->grid = std::min(b->nunits, ctxs[0]->split->nsm);
  auto upload = [&](void** d, const void* h, size_t bytes) -> lem_status {
    if (cudaMalloc(d, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(LEM_ENOMEM, "batch tables");
    }
    LEM_CUDA_TRY(cudaMemcpy(*d, h, bytes, cudaMemcpyHostToDevice));
    return LEM_OK;
  };
  lem_status st = upload(reinterpret_cast<void**>(&b->d_probs), probs.data(), sizeof(SplitProblem) * n);
  if (st == LEM_OK) st = upload(reinterpret_cast<void**>(&b->d_res), res.data(), sizeof(ResProblem) * n);
  if (st == LEM_OK) st = upload(reinterpret_cast<void**>(&b->d_res_first), res_first.data(), sizeof(int) * n);
  if (st == LEM_OK) st = upload(reinterpret_cast<void**>(&b->d_conv), conv.data(), sizeof(ConvProblem) * n);
  if (st == LEM_OK) st = upload(reinterpret_cast<void**>(&b->d_conv_first), conv_first.data(), sizeof(int) * n);
  const int zero = 0;
  if (st == LEM_OK) st = upload(reinterpret_cast<void**>(&b->d_err), &zero, sizeof(int));
  if (st != LEM_OK) {
    split_batch_destroy(b);
    return st;
  }
  *out = b;
  return LEM_OK;
}

lem_status split_batch_step(SplitBatch* b, int nsteps, cudaStream_t st, cudaEvent_t* ev) {
  // ev (not under capture): 2 * nsteps + 2 events bracketing [conversion + measure],
  // then each step's residual and GEMM
  convert_multi_kernel<<<b->conv_blocks, 256, 0, st>>>(b->d_conv, b->d_conv_first, b->n, 1);
  residual_multi_kernel<<<b->res_blocks, 256, 0, st>>>(b->d_res, b->d_res_first, b->n, 1, 1);
  LEM_CUDA_TRY(cudaGetLastError());
  if (ev) LEM_CUDA_TRY(cudaEventRecord(ev[0], st));
  cudaLaunchConfig_t cfg{};
  cfg.blockDim = dim3(gemm_threads(b->np));
  cfg.dynamicSmemBytes = SMEM_BYTES;
  cfg.stream = st;
  cfg.gridDim = dim3(b->grid);
  for (int k = 0; k < nsteps; ++k) {
    const int parity = k & 1;
    residual_multi_kernel<<<b->res_blocks, 256, 0, st>>>(b->d_res, b->d_res_first, b->n, parity, 0);
    if (ev) LEM_CUDA_TRY(cudaEventRecord(ev[1 + 2 * k], st));
    LEM_CUDA_TRY(cudaLaunchKernelEx(&cfg, gemm_kernel_for(b->bn, b->np, true), b->first,
                                    static_cast<const SplitProblem*>(b->d_probs), b->n, b->nunits, parity, b->d_err,
                                    0u));
    if (ev) LEM_CUDA_TRY(cudaEventRecord(ev[2 + 2 * k], st));
  }
  convert_multi_kernel<<<b->conv_blocks, 256, 0, st>>>(b->d_conv, b->d_conv_first, b->n, 0);
  LEM_CUDA_TRY(cudaGetLastError());
  return LEM_OK;
}

double split_batch_executed_flops(const SplitBatch* b) { return b->executed_flops; }

// Algorithmic FLOPs of one fused GEMM launch: products x 2 x owner rows x window nodes, summed
// over every window of every problem.
double split_batch_gemm_flops(const SplitBatch* b, lem_ctx* const* ctxs) {
  double f = 0.0;
  for (int i = 0; i < b->n; ++i) {
    const SplitPlan* sp = ctxs[i]->split;
    f += 2.0 * sp->np * 2.0 * sp->M * double(sp->Wy) * sp->Wx * double(sp->ntx) * sp->nty;
  }
  return f;
}

lem_status split_batch_check_error(SplitBatch* b) {
  int e = 0;
  LEM_CUDA_TRY(cudaMemcpy(&e, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e != 0) {
    cudaMemset(b->d_err, 0, sizeof(int));
    if (e == ERR_NUMERIC) return fail(LEM_ENUMERIC, "split path: propagator rows too heavy for an exact integer product");
    return fail(LEM_ETIMEOUT, "tensor-core kernel gave up waiting on an mbarrier (code " + std::to_string(e) + ")");
  }
  return LEM_OK;
}

lem_status split_check_error(lem_ctx* ctx) {
  if (!ctx->split) return LEM_OK;
  int e = 0;
  LEM_CUDA_TRY(cudaMemcpy(&e, ctx->split->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e != 0) {
    cudaMemset(ctx->split->d_err, 0, sizeof(int));
    if (e == ERR_NUMERIC) return fail(LEM_ENUMERIC, "split path: propagator rows too heavy for an exact integer product");
    return fail(LEM_ETIMEOUT, "tensor-core kernel gave up waiting on an mbarrier (code " + std::to_string(e) + ")");
  }
  return LEM_OK;
}

void split_destroy(lem_ctx* ctx) {
  SplitPlan* sp = ctx->split;
  if (!sp) return;
  for (void* p : {static_cast<void*>(sp->d_uh), static_cast<void*>(sp->d_ul), static_cast<void*>(sp->d_Rint),
                  static_cast<void*>(sp->d_R2), static_cast<void*>(sp->d_Pt),
                  static_cast<void*>(sp->d_eP), static_cast<void*>(sp->d_S),
                  static_cast<void*>(sp->d_R3), static_cast<void*>(sp->d_rmax), static_cast<void*>(sp->d_escale),
                  static_cast<void*>(sp->d_err), static_cast<void*>(sp->d_rb), static_cast<void*>(sp->d_part),
                  static_cast<void*>(sp->d_flags)})
    if (p) cudaFreeAsync(p, ctx->stream);  // stream-ordered (the memory came from cudaMallocAsync)
  delete sp;
  ctx->split = nullptr;
}

}  // namespace lem
