// Split-precision LEM step on the tcgen05 tensor cores (Sec. 3 steps 1-3, Eq. lem) for
// problems whose windows all share one local operator (constant coefficients, periodic 2D
// mesh, tiles dividing the mesh). One step is two kernels:
//
//  1. residual_split_kernel: r = dt A u^n from the float-float state, written as a scaled
//     FP16 pair r*2^er = r_hi + r_lo into a ghost-padded [ny + 2Hy][pitch] array (the
//     periodic halo is materialised here, so every window is a plain rectangle of it).
//  2. split_gemm_kernel: Y = P R, M = Ty*Tx owner rows, N = tiles, K = window nodes, with
//     P*2^eP = P_hi + P_lo. Each K block is one window row (Wx nodes, padded to 64 in the
//     P layout): TMA loads P_hi/P_lo tiles and the 128 windows' rows straight from the
//     padded residual through a 4D tensor map (the halo gather happens inside TMA). One
//     thread issues tcgen05.mma: per window row the small products P_hi r_lo, P_lo r_hi,
//     P_lo r_lo and then P_hi r_hi into one TMEM accumulator (two buffers alternate). The
//     tensor pipe's FP32 accumulation is not correctly rounded, so each row's partial is
//     drained into registers and summed there with Kahan compensation. The epilogue scales
//     by 2^-(eP + er) and adds Y into the owner nodes of the float-float state (scatter).
//
// The float-float state (u_hi + u_lo, about 48 bits) is converted from/to the caller's
// FP64 buffer once per lem_step call. max|u| is tracked by the epilogue for the next
// step's residual scale (|r| <= K_r max|u| with K_r = 2 sum_nbr |c| + |sum c|).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "lem_internal.h"
#include "tc_ptx.cuh"

namespace lem {

namespace {

constexpr int BM = 128;            // owner rows per CTA tile (TMEM lanes)
constexpr int BN = 128;            // windows per CTA tile (TMEM columns per accumulator)
constexpr int KB = 64;             // fp16 elements per 128-byte K row
constexpr int STAGES = 3;
constexpr int TILE_BYTES = BM * KB * 2;  // 16 KB (A and B tiles have 128 rows each)
constexpr int STAGE_BYTES = 4 * TILE_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr uint32_t TMEM_COLS = 256;  // two row accumulators of BN fp32 columns
constexpr int EPI_WARPS = 8;           // two warps per TMEM lane quarter
constexpr int EPI_COLS = BN / 2;       // columns drained by one epilogue thread
constexpr int GEMM_THREADS = 64 + 32 * EPI_WARPS;
constexpr uint64_t WAIT_NS = 2000000000ull;  // 2 s bound on every mbarrier wait

enum : int { ERR_TIMEOUT_PRODUCER = 1, ERR_TIMEOUT_MMA = 2, ERR_TIMEOUT_EPI = 3 };

struct GemmParams {
  int Wy, Wx, Ty, Tx, nx, BNx, BNy, ntx, eP;
  float Kr;
  unsigned* umax;
  int* err;
  int parity;
};

struct ResParams {
  int ny, nx, Hy, Hx, pitch, prow;
  float c_hi[5], c_lo[5];   // dt-scaled C, W, E, S, N as float pairs
  float csum_hi, csum_lo;   // sum of all five
  float Kr;
};

__device__ __forceinline__ float pow2f(int e) {  // exact 2^e for -126 <= e <= 127
  return __int_as_float((127 + e) << 23);
}

__device__ __forceinline__ int residual_exponent(float Kr, unsigned umax_bits) {
  const float v = Kr * __uint_as_float(umax_bits);
  if (!(v > 0.0f)) return 0;
  int e;
  frexpf(v, &e);  // v < 2^e, so |r| 2^(14-e) < 2^14 < fp16 max
  return 14 - e;
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

// acc += (ch + cl) * d, keeping the product's rounding error (exact through the FMA)
__device__ __forceinline__ void ff_mac(ffv& acc, float ch, float cl, ffv d) {
  const float p = __fmul_rn(ch, d.h);
  float pe = fmaf(ch, d.h, -p);
  pe = fmaf(ch, d.l, fmaf(cl, d.h, pe));
  const ffv s = two_sum(acc.h, p);
  acc.h = s.h;
  acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, pe));
}

__global__ void __launch_bounds__(256) residual_split_kernel(const float* __restrict__ uh,
                                                             const float* __restrict__ ul,
                                                             __half* __restrict__ Rhi,
                                                             __half* __restrict__ Rlo, ResParams p,
                                                             unsigned* umax, int parity) {
  const int er = residual_exponent(p.Kr, umax[parity]);
  const float scale = pow2f(er);
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) umax[parity ^ 1] = 0u;
  const int xp = blockIdx.x * blockDim.x + threadIdx.x;  // padded column
  const int wpad = p.nx + 2 * p.Hx;
  if (xp >= wpad) return;
  for (int yp = blockIdx.y; yp < p.prow; yp += gridDim.y) {
    int y = yp - p.Hy, x = xp - p.Hx;
    y = (y % p.ny + p.ny) % p.ny;
    x = (x % p.nx + p.nx) % p.nx;
    const int64_t c = int64_t(y) * p.nx + x;
    const int xw = x == 0 ? p.nx - 1 : x - 1, xe = x == p.nx - 1 ? 0 : x + 1;
    const int ys = y == 0 ? p.ny - 1 : y - 1, yn = y == p.ny - 1 ? 0 : y + 1;
    const int64_t iw = int64_t(y) * p.nx + xw, ie = int64_t(y) * p.nx + xe;
    const int64_t is = int64_t(ys) * p.nx + x, in = int64_t(yn) * p.nx + x;
    const float ch = uh[c], cl = ul[c];
    // r = sum_nbr c_j (u_j - u_C) + (sum_all c) u_C, every term and the sum in float-float:
    // the W/E (S/N) differences of a smooth field nearly cancel, so a float sum would
    // lose about log2(|c d| / |r|) bits of r.
    ffv acc{0.0f, 0.0f};
    ff_mac(acc, p.c_hi[1], p.c_lo[1], ff_sub(uh[iw], ul[iw], ch, cl));
    ff_mac(acc, p.c_hi[2], p.c_lo[2], ff_sub(uh[ie], ul[ie], ch, cl));
    ff_mac(acc, p.c_hi[3], p.c_lo[3], ff_sub(uh[is], ul[is], ch, cl));
    ff_mac(acc, p.c_hi[4], p.c_lo[4], ff_sub(uh[in], ul[in], ch, cl));
    ff_mac(acc, p.csum_hi, p.csum_lo, ffv{ch, cl});
    const float r = __fadd_rn(acc.h, acc.l);
    const float rs = __fmul_rn(r, scale);
    const __half h = __float2half_rn(rs);
    const __half l = __float2half_rn(__fsub_rn(rs, __half2float(h)));
    const int64_t o = int64_t(yp) * p.pitch + xp;
    Rhi[o] = h;
    Rlo[o] = l;
  }
}

__global__ void f64_to_ff_kernel(const double* __restrict__ u, float* __restrict__ uh,
                                 float* __restrict__ ul, int64_t n, unsigned* umax) {
  float m = 0.0f;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double v = u[i];
    const float h = __double2float_rn(v);
    const float l = __double2float_rn(v - double(h));
    uh[i] = h;
    ul[i] = l;
    m = fmaxf(m, fabsf(h));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(umax, __float_as_uint(m));
}

__global__ void ff_to_f64_kernel(const float* __restrict__ uh, const float* __restrict__ ul,
                                 double* __restrict__ u, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    u[i] = double(uh[i]) + double(ul[i]);
}

__global__ void absmax_f64_kernel(const double* __restrict__ x, int64_t n, unsigned long long* out) {
  double m = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    m = fmax(m, fabs(x[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// P (FP64, n_int x n_loc, window row-major) -> P*2^eP = hi + lo in the [M][Wy*64] K layout
__global__ void pack_p_kernel(const double* __restrict__ P, int64_t n_loc, int M, int Wy, int Wx, int eP,
                              __half* __restrict__ Phi, __half* __restrict__ Plo) {
  const int64_t total = int64_t(M) * Wy * KB;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int i = int(e / (int64_t(Wy) * KB));
    const int col = int(e % (int64_t(Wy) * KB));
    const int wy = col / KB, wx = col % KB;
    const double v = wx < Wx ? P[int64_t(i) * n_loc + int64_t(wy) * Wx + wx] : 0.0;
    const double x = ldexp(v, eP);
    const __half h = __double2half(x);
    const __half l = __double2half(x - double(__half2float(h)));
    Phi[e] = h;
    Plo[e] = l;
  }
}

__global__ void __launch_bounds__(GEMM_THREADS, 1)
    split_gemm_kernel(const __grid_constant__ CUtensorMap tmAhi, const __grid_constant__ CUtensorMap tmAlo,
                      const __grid_constant__ CUtensorMap tmBhi, const __grid_constant__ CUtensorMap tmBlo,
                      float* __restrict__ uh, float* __restrict__ ul, GemmParams g) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* tiles = smem;  // [stage][A_hi, A_lo, B_hi, B_lo] 16 KB each
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* full = bars;                 // [STAGES] stage loaded
  uint64_t* empty = bars + STAGES;       // [STAGES] stage consumed by the MMAs
  uint64_t* accf = bars + 2 * STAGES;    // [2] row accumulator ready
  uint64_t* acce = accf + 2;             // [2] row accumulator drained
  uint64_t* done = acce + 2;             // every MMA finished
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ volatile int s_abort;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int m0 = blockIdx.x * BM;
  const int nbx = g.ntx / g.BNx;
  const int tx0 = (blockIdx.y % nbx) * g.BNx;
  const int ty0 = (blockIdx.y / nbx) * g.BNy;
  const int nk = g.Wy;

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < STAGES; ++s) { ptx::mbar_init(&full[s], 1); ptx::mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { ptx::mbar_init(&accf[b], 1); ptx::mbar_init(&acce[b], EPI_WARPS); }
    ptx::mbar_init(done, 1);
    ptx::fence_barrier_init();
    ptx::tma_prefetch_desc(&tmAhi); ptx::tma_prefetch_desc(&tmAlo);
    ptx::tma_prefetch_desc(&tmBhi); ptx::tma_prefetch_desc(&tmBlo);
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, TMEM_COLS);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int issued = 0;
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES;
        const uint32_t use = kb / STAGES;
        if (kb >= STAGES && !ptx::mbar_wait(&empty[s], (use & 1) ^ 1, WAIT_NS)) {
          atomicExch(g.err, ERR_TIMEOUT_PRODUCER);
          s_abort = 1;
          break;
        }
        if (s_abort) break;
        uint8_t* st = tiles + s * STAGE_BYTES;
        ptx::mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
        ptx::tma_load_2d(st, &tmAhi, &full[s], kb * KB, m0);
        ptx::tma_load_2d(st + TILE_BYTES, &tmAlo, &full[s], kb * KB, m0);
        ptx::tma_load_4d(st + 2 * TILE_BYTES, &tmBhi, &full[s], 0, tx0, kb, ty0);
        ptx::tma_load_4d(st + 3 * TILE_BYTES, &tmBlo, &full[s], 0, tx0, kb, ty0);
        issued = kb + 1;
      }
      // every copy this thread issued has landed before the CTA may exit
      for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
        ptx::mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1, WAIT_NS);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = ptx::idesc_f16_f32(BM, BN);
      bool ok = true;
      for (int kb = 0; kb < nk; ++kb) {
        const int buf = kb & 1;
        if (kb >= 2) {
          if (!ptx::mbar_wait(&acce[buf], ((kb >> 1) - 1) & 1, WAIT_NS)) { ok = false; break; }
          ptx::tc_fence_after();
        }
        const int s = kb % STAGES;
        if (!ptx::mbar_wait(&full[s], (kb / STAGES) & 1, WAIT_NS)) { ok = false; break; }
        ptx::tc_fence_after();
        const uint32_t base = ptx::smem_u32(tiles + s * STAGE_BYTES);
        const uint64_t dAh = ptx::sw128_kmajor_desc(base);
        const uint64_t dAl = ptx::sw128_kmajor_desc(base + TILE_BYTES);
        const uint64_t dBh = ptx::sw128_kmajor_desc(base + 2 * TILE_BYTES);
        const uint64_t dBl = ptx::sw128_kmajor_desc(base + 3 * TILE_BYTES);
        const uint32_t d = tmem + buf * BN;
        // the three small products first, the large P_hi r_hi last: the tensor pipe's
        // accumulation error scales with the accumulator's size when each term is added
        for (int kk = 0; kk < g.Wx / 16; ++kk) {
          const uint64_t adv = uint64_t(kk * 32) >> 4;  // 16 fp16 = 32 B along K
          ptx::mma_f16(d, dAh + adv, dBl + adv, idesc, kk > 0 ? 1u : 0u);
          ptx::mma_f16(d, dAl + adv, dBh + adv, idesc, 1u);
          ptx::mma_f16(d, dAl + adv, dBl + adv, idesc, 1u);
        }
        for (int kk = 0; kk < g.Wx / 16; ++kk) {
          const uint64_t adv = uint64_t(kk * 32) >> 4;
          ptx::mma_f16(d, dAh + adv, dBh + adv, idesc, 1u);
        }
        ptx::mma_commit(&empty[s]);
        ptx::mma_commit(&accf[buf]);
      }
      if (!ok) {
        atomicExch(g.err, ERR_TIMEOUT_MMA);
        s_abort = 1;
      }
      ptx::mma_commit(done);
      ptx::mbar_wait(done, 0, WAIT_NS);  // no MMA may still run when TMEM is released
    }
  } else {
    // ------------------------------------------------------------ epilogue (8 warps)
    // warp w reads TMEM lanes 32*(w%4)..+31 (its owner rows) and 64 of the 128 columns
    const int lane_base = 32 * (warp & 3);
    const int half = (warp - 2) >> 2;
    const int row = lane_base + lane;
    const uint32_t t_lane = tmem + (uint32_t(lane_base) << 16) + uint32_t(half * EPI_COLS);
    // Kahan sum over the window rows; the compensation (a few ulp of acc) is kept in packed
    // bf16 pairs, which have FP32 range and enough bits for a correction term
    float acc[EPI_COLS];
    __nv_bfloat162 comp[EPI_COLS / 2];
#pragma unroll
    for (int i = 0; i < EPI_COLS; ++i) acc[i] = 0.0f;
#pragma unroll
    for (int i = 0; i < EPI_COLS / 2; ++i) comp[i] = __floats2bfloat162_rn(0.0f, 0.0f);
    bool ok = true;
    for (int kb = 0; kb < nk; ++kb) {
      const int buf = kb & 1;
      if (!ptx::mbar_wait(&accf[buf], (kb >> 1) & 1, WAIT_NS)) { ok = false; break; }
      ptx::tc_fence_after();
#pragma unroll
      for (int q = 0; q < EPI_COLS / 16; ++q) {
        float v[16];
        ptx::tmem_ld_32x32b_x16(t_lane + buf * BN + q * 16, v);
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
          const int j = q * 16 + i;
          const float2 c = __bfloat1622float2(comp[j / 2]);
          const float y0 = __fsub_rn(v[i], c.x), y1 = __fsub_rn(v[i + 1], c.y);
          const float t0 = __fadd_rn(acc[j], y0), t1 = __fadd_rn(acc[j + 1], y1);
          comp[j / 2] = __floats2bfloat162_rn(__fsub_rn(__fsub_rn(t0, acc[j]), y0),
                                              __fsub_rn(__fsub_rn(t1, acc[j + 1]), y1));
          acc[j] = t0;
          acc[j + 1] = t1;
        }
      }
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&acce[buf]);
    }
    if (!ok) {
      atomicExch(g.err, ERR_TIMEOUT_EPI);
    } else {
      const int er = residual_exponent(g.Kr, g.umax[g.parity]);
      const float oscale = pow2f(-(g.eP + er));
      const int ii = m0 + row;
      const int iy = ii / g.Tx, ix = ii % g.Tx;
      float umax_local = 0.0f;
#pragma unroll
      for (int j = 0; j < EPI_COLS; ++j) {
        const int n = half * EPI_COLS + j;
        const int ty = ty0 + n / g.BNx, tx = tx0 + n % g.BNx;
        const int64_t node = int64_t(ty * g.Ty + iy) * g.nx + tx * g.Tx + ix;
        const float2 cc = __bfloat1622float2(comp[j / 2]);
        const float y = __fmul_rn(__fsub_rn(acc[j], (j & 1) ? cc.y : cc.x), oscale);
        // (u_hi, u_lo) += y in float-float
        const ffv s = two_sum(uh[node], y);
        const float lo = __fadd_rn(ul[node], s.l);
        const float hi2 = __fadd_rn(s.h, lo);
        const float lo2 = __fsub_rn(lo, __fsub_rn(hi2, s.h));
        uh[node] = hi2;
        ul[node] = lo2;
        umax_local = fmaxf(umax_local, fabsf(hi2));
      }
      for (int o = 16; o > 0; o >>= 1) umax_local = fmaxf(umax_local, __shfl_xor_sync(0xffffffffu, umax_local, o));
      if (lane == 0) atomicMax(g.umax + (g.parity ^ 1), __float_as_uint(umax_local));
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, TMEM_COLS);
  }
}

// -------------------------------------------------------------------- host helpers
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

}  // namespace

struct SplitPlan {
  int Ty = 0, Tx = 0, Hy = 0, Hx = 0, Wy = 0, Wx = 0, nty = 0, ntx = 0, M = 0, BNx = 0, BNy = 0;
  int pitch = 0, prow = 0, eP = 0;
  float Kr = 0.0f;
  ResParams rp{};
  float* d_uh = nullptr;
  float* d_ul = nullptr;
  __half* d_Rhi = nullptr;
  __half* d_Rlo = nullptr;
  __half* d_Phi = nullptr;
  __half* d_Plo = nullptr;
  unsigned* d_umax = nullptr;
  int* d_err = nullptr;
  unsigned long long* d_pmax = nullptr;
  CUtensorMap tmAhi, tmAlo, tmBhi, tmBlo;
  int packed_gen = -1;
};

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
  if (Wx > KB || Wx % 16 || Tx % 8) return false;
  if ((Ty * Tx) % BM) return false;
  const int64_t ntx = ctx->nx / Tx, nty = ctx->ny / Ty;
  if (ntx >= BN) { if (ntx % BN) return false; }
  else if (BN % ntx || nty % (BN / ntx)) return false;
  return true;
}

static lem_status encode(CUtensorMap* m, void* base, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
                         const cuuint32_t* box, const char* what) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return fail(LEM_ECUDA, "cuTensorMapEncodeTiled unavailable");
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, cuuint32_t(rank), base, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
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
  sp->BNx = sp->ntx >= BN ? BN : sp->ntx;
  sp->BNy = BN / sp->BNx;
  // padded residual: rows ny + 2Hy, row pitch covers the last 64-wide window row read
  sp->prow = int(ctx->ny) + 2 * sp->Hy;
  int need = std::max<int>(int(ctx->nx) + 2 * sp->Hx, (sp->ntx - 1) * sp->Tx + KB);
  sp->pitch = (need + 7) / 8 * 8;
  // stencil constants (dt-scaled) as float pairs; bound K_r for the residual scale
  double c[5], csum = 0.0, babs = 0.0;
  std::vector<double> hc(5);
  LEM_CUDA_TRY(cudaMemcpy(hc.data(), ctx->d_coef, sizeof(double) * 5, cudaMemcpyDeviceToHost));
  for (int k = 0; k < 5; ++k) {
    c[k] = hc[k];
    csum += c[k];
    if (k > 0) babs += 2.0 * std::fabs(c[k]);
    sp->rp.c_hi[k] = float(c[k]);
    sp->rp.c_lo[k] = float(c[k] - double(sp->rp.c_hi[k]));
  }
  sp->rp.csum_hi = float(csum);
  sp->rp.csum_lo = float(csum - double(sp->rp.csum_hi));
  sp->Kr = float((babs + std::fabs(csum)) * 1.001);
  sp->rp.Kr = sp->Kr;
  sp->rp.ny = int(ctx->ny); sp->rp.nx = int(ctx->nx); sp->rp.Hy = sp->Hy; sp->rp.Hx = sp->Hx;
  sp->rp.pitch = sp->pitch; sp->rp.prow = sp->prow;
  const size_t npts = size_t(ctx->npts);
  const size_t rbytes = sizeof(__half) * size_t(sp->prow) * sp->pitch;
  const size_t pbytes = sizeof(__half) * size_t(sp->M) * sp->Wy * KB;
  LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&sp->d_uh), sizeof(float) * npts));
  LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&sp->d_ul), sizeof(float) * npts));
  LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&sp->d_Rhi), rbytes));
  LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&sp->d_Rlo), rbytes));
  LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&sp->d_Phi), pbytes));
  LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&sp->d_Plo), pbytes));
  LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&sp->d_umax), sizeof(unsigned) * 2));
  LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&sp->d_err), sizeof(int)));
  LEM_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&sp->d_pmax), sizeof(unsigned long long)));
  LEM_CUDA_TRY(cudaMemset(sp->d_Rhi, 0, rbytes));
  LEM_CUDA_TRY(cudaMemset(sp->d_Rlo, 0, rbytes));
  LEM_CUDA_TRY(cudaMemset(sp->d_err, 0, sizeof(int)));
  // tensor maps: A = [M][Wy*64] fp16, box 64 x 128 ; B = 4D overlapping view of the
  // padded residual: (wx, tx, wy, ty) -> R[ty*Ty + wy][tx*Tx + wx], box 64 x BNx x 1 x BNy
  {
    cuuint64_t dims[2] = {cuuint64_t(sp->Wy) * KB, cuuint64_t(sp->M)};
    cuuint64_t str[1] = {cuuint64_t(sp->Wy) * KB * 2};
    cuuint32_t box[2] = {KB, BM};
    LEM_TRY(encode(&sp->tmAhi, sp->d_Phi, 2, dims, str, box, "P_hi"));
    LEM_TRY(encode(&sp->tmAlo, sp->d_Plo, 2, dims, str, box, "P_lo"));
  }
  {
    cuuint64_t dims[4] = {KB, cuuint64_t(sp->ntx), cuuint64_t(sp->Wy), cuuint64_t(sp->nty)};
    cuuint64_t str[3] = {cuuint64_t(sp->Tx) * 2, cuuint64_t(sp->pitch) * 2, cuuint64_t(sp->Ty) * sp->pitch * 2};
    cuuint32_t box[4] = {KB, cuuint32_t(sp->BNx), 1, cuuint32_t(sp->BNy)};
    LEM_TRY(encode(&sp->tmBhi, sp->d_Rhi, 4, dims, str, box, "R_hi"));
    LEM_TRY(encode(&sp->tmBlo, sp->d_Rlo, 4, dims, str, box, "R_lo"));
  }
  LEM_CUDA_TRY(cudaFuncSetAttribute(split_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
  cudaFuncAttributes fa{};
  LEM_CUDA_TRY(cudaFuncGetAttributes(&fa, split_gemm_kernel));
  if (fa.maxThreadsPerBlock < GEMM_THREADS)
    return fail(LEM_ECUDA, "split GEMM kernel cannot launch " + std::to_string(GEMM_THREADS) + " threads (" +
                               std::to_string(fa.numRegs) + " registers per thread)");
  return LEM_OK;
}

static lem_status split_pack(lem_ctx* ctx) {
  SplitPlan* sp = ctx->split;
  cudaStream_t st = ctx->stream;
  const int64_t np = ctx->n_int * ctx->n_loc;
  LEM_CUDA_TRY(cudaMemsetAsync(sp->d_pmax, 0, sizeof(unsigned long long), st));
  absmax_f64_kernel<<<256, 256, 0, st>>>(ctx->d_P, np, sp->d_pmax);
  LEM_CUDA_TRY(cudaGetLastError());
  unsigned long long bits = 0;
  LEM_CUDA_TRY(cudaMemcpyAsync(&bits, sp->d_pmax, sizeof(bits), cudaMemcpyDeviceToHost, st));
  LEM_CUDA_TRY(cudaStreamSynchronize(st));
  double pmax;
  std::memcpy(&pmax, &bits, sizeof(pmax));
  int e = 0;
  if (pmax > 0.0) std::frexp(pmax, &e);
  sp->eP = pmax > 0.0 ? 14 - e : 0;
  pack_p_kernel<<<1024, 256, 0, st>>>(ctx->d_P, ctx->n_loc, sp->M, sp->Wy, sp->Wx, sp->eP, sp->d_Phi, sp->d_Plo);
  LEM_CUDA_TRY(cudaGetLastError());
  sp->packed_gen = ctx->build_gen;
  return LEM_OK;
}

lem_status split_step(lem_ctx* ctx, double* d_u, int nsteps) {
  SplitPlan* sp = ctx->split;
  cudaStream_t st = ctx->stream;
  if (sp->packed_gen != ctx->build_gen) LEM_TRY(split_pack(ctx));
  const int64_t npts = ctx->npts;
  LEM_CUDA_TRY(cudaMemsetAsync(sp->d_umax, 0, sizeof(unsigned) * 2, st));
  f64_to_ff_kernel<<<1024, 256, 0, st>>>(d_u, sp->d_uh, sp->d_ul, npts, sp->d_umax);
  LEM_CUDA_TRY(cudaGetLastError());
  GemmParams g{};
  g.Wy = sp->Wy; g.Wx = sp->Wx; g.Ty = sp->Ty; g.Tx = sp->Tx; g.nx = int(ctx->nx);
  g.BNx = sp->BNx; g.BNy = sp->BNy; g.ntx = sp->ntx; g.eP = sp->eP;
  g.Kr = sp->Kr; g.umax = sp->d_umax; g.err = sp->d_err;
  const dim3 rgrid((int(ctx->nx) + 2 * sp->Hx + 255) / 256, std::min(sp->prow, 4096));
  const dim3 ggrid(sp->M / BM, unsigned(ctx->tiles.size() / BN));
  for (int k = 0; k < nsteps; ++k) {
    const int parity = k & 1;
    residual_split_kernel<<<rgrid, 256, 0, st>>>(sp->d_uh, sp->d_ul, sp->d_Rhi, sp->d_Rlo, sp->rp, sp->d_umax,
                                                 parity);
    g.parity = parity;
    cudaEvent_t stop;
    LEM_CUDA_TRY(ctx->timing_begin(&stop));
    split_gemm_kernel<<<ggrid, GEMM_THREADS, SMEM_BYTES, st>>>(sp->tmAhi, sp->tmAlo, sp->tmBhi, sp->tmBlo, sp->d_uh,
                                                       sp->d_ul, g);
    ctx->timing_end(stop);
  }
  LEM_CUDA_TRY(cudaGetLastError());
  ff_to_f64_kernel<<<1024, 256, 0, st>>>(sp->d_uh, sp->d_ul, d_u, npts);
  LEM_CUDA_TRY(cudaGetLastError());
  return LEM_OK;
}

lem_status split_check_error(lem_ctx* ctx) {
  if (!ctx->split) return LEM_OK;
  int e = 0;
  LEM_CUDA_TRY(cudaMemcpy(&e, ctx->split->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e != 0) {
    cudaMemset(ctx->split->d_err, 0, sizeof(int));
    return fail(LEM_ETIMEOUT, "tensor-core kernel gave up waiting on an mbarrier (code " + std::to_string(e) + ")");
  }
  return LEM_OK;
}

void split_destroy(lem_ctx* ctx) {
  SplitPlan* sp = ctx->split;
  if (!sp) return;
  cudaFree(sp->d_uh); cudaFree(sp->d_ul); cudaFree(sp->d_Rhi); cudaFree(sp->d_Rlo);
  cudaFree(sp->d_Phi); cudaFree(sp->d_Plo); cudaFree(sp->d_umax); cudaFree(sp->d_err); cudaFree(sp->d_pmax);
  delete sp;
  ctx->split = nullptr;
}

}  // namespace lem
