// Dense FP64 matrix products of the propagator build on the tcgen05 tensor cores, for the
// split-precision tiers (Sec. 1, Sec. 4: Pade-13 products and the squarings of scaling and
// squaring). The FP64 tier keeps the FP64 GEMM; the Pade denominator solve stays in FP64.
//
// The products are exact sums of integer slice products (an Ozaki-type splitting). Each row i
// of A is scaled by 2^-e_i (max |A_i,:| < 2^e_i) and cut into OZ_S slices of OZ_BITS bits,
//   A_ik 2^-e_i = sum_s a_s 2^-(7(s+1)) (+ remainder < 2^-49),  a_s integers, |a_s| <= 128,
// and each column j of B likewise with 2^-f_j. Slices are FP16 (integers up to 2048 are exact).
// For every level L = s + t <= OZ_S - 1 the MMA accumulates sum_k a_s b_t over a K chunk of
// 128 into one TMEM accumulator: at most 7 pairs x 128 terms x 2^14 < 2^24, so every partial
// sum is an integer FP32 holds exactly, whatever the tensor pipe's rounding. After each chunk
// the epilogue adds sum_L acc_L 2^-7L into a float-float accumulator (about 48 bits), and at
// the end C_ij = alpha 2^(e_i + f_j - 14) (hi + lo) + beta C_ij in FP64. The dropped terms
// (L >= OZ_S, slice remainders) are below 2^-48 of sum_k |A_ik| |B_kj|.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "lem_internal.h"
#include "tc_ptx.cuh"

namespace lem {

namespace {

constexpr int OZ_S = 7;     // slices per operand
constexpr int OZ_BM = 128;  // output rows per CTA (TMEM lanes)
constexpr int OZ_BN = 64;   // output columns per CTA
constexpr int OZ_KB = 32;   // K elements per block
constexpr int OZ_CHUNK = 4;  // K blocks per exact chunk (K = 128)
constexpr int OZ_A_BYTES = OZ_BM * OZ_KB * 2;
constexpr int OZ_B_BYTES = OZ_BN * OZ_KB * 2;
constexpr int OZ_STAGE = OZ_S * (OZ_A_BYTES + OZ_B_BYTES);  // 84 KB: all slices of one K block
constexpr int OZ_STAGES = 2;
constexpr int OZ_SMEM = OZ_STAGES * OZ_STAGE + 1024 + 256;
constexpr int OZ_THREADS = 192;                             // producer, MMA issuer, 4 epilogue warps
constexpr uint64_t OZ_WAIT_NS = 2000000000ull;

// x 2^E as a double, built from the bits of the float x with integer operations only (x normal
// or zero; GB300 runs FP64 conversions and multiplies at a small fraction of its FP32 rate).
__device__ __forceinline__ double f32_scaled_to_f64(float x, int E) {
  const uint32_t b = __float_as_uint(x);
  const int e8 = static_cast<int>((b >> 23) & 0xFF);
  const int ed = e8 - 127 + E + 1023;
  if (e8 == 0 || ed <= 0) return 0.0;
  const unsigned long long sign = static_cast<unsigned long long>(b >> 31) << 63;
  if (ed >= 2047) return __longlong_as_double(static_cast<long long>(sign | 0x7FF0000000000000ull));
  return __longlong_as_double(static_cast<long long>(sign | (static_cast<unsigned long long>(ed) << 52) |
                                                     (static_cast<unsigned long long>(b & 0x7FFFFF) << 29)));
}

// Biased exponent field of a double (0 for zero and subnormals, which the slices treat as 0).
__device__ __forceinline__ int exp_field(double x) {
  return static_cast<int>((static_cast<unsigned long long>(__double_as_longlong(x)) >> 52) & 0x7FF);
}

// The scale exponent of a row or column with largest biased exponent field E: every entry
// has |x| < 2^(E - 1022).
__device__ __forceinline__ int scale_exp(int E) { return E - 1022; }

// Slices of x 2^-e (|x| < 2^e) as 7 balanced base-128 digits, most significant first:
// x 2^-e = sum_s d_s 2^-7(s+1) + rem, |d_0| <= 128, |d_s| <= 64 (s > 0), |rem| <= 2^-50.
// Integer arithmetic on the bits of x: N = round(x 2^(49 - e)) is the mantissa shifted right
// by sh = 1026 + e - E >= 4 (sh >= 54 gives 0), and the digits are N's balanced base-128
// digits (round to nearest at each step).
__device__ __forceinline__ void slice_digits(double x, int e, __half (&d)[OZ_S]) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(x));
  const int E = static_cast<int>((bits >> 52) & 0x7FF);
  long long N = 0;
  const int sh = 1026 + e - E;
  if (E != 0 && sh < 54) {
    const long long m = static_cast<long long>((bits & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
    N = (m + (1ll << (sh - 1))) >> sh;
    if (bits >> 63) N = -N;
  }
#pragma unroll
  for (int s = 0; s < OZ_S - 1; ++s) {
    const int p = 7 * (OZ_S - 1 - s);
    const long long q = (N + (1ll << (p - 1))) >> p;  // arithmetic shift: floor
    N -= q << p;
    d[s] = __int2half_rn(static_cast<int>(q));
  }
  d[OZ_S - 1] = __int2half_rn(static_cast<int>(N));
}

// Strided batch of row-major FP64 matrices: element (q, r, c) at p + map(q) stride + r ld + c.
struct Mat {
  const double* p;
  int64_t ld, stride;
};
struct MatOut {
  double* p;
  int64_t ld, stride;
};

// Matrix q of a product batch is matrix map[q] of the caller's arrays (map null: q itself);
// slices and exponents are stored at q.
__device__ __forceinline__ int mat_of(const int* map, int q) { return map ? map[q] : q; }

// Slice planes are stored as the operand tiles the MMA reads, each one contiguous: for slice s
// of matrix q, tile (row block, K block) of R x OZ_KB halves (R = 128 for A, 64 for B) in the
// tcgen05 K-major layout without swizzle: 8-row x 8-element core matrices of 128 contiguous
// bytes, core matrices along K 128 B apart, along the rows 512 B apart. Element (r, k) of a
// tile sits at half offset (r / 8) 256 + (k / 8) 64 + (r % 8) 8 + k % 8.
__device__ __forceinline__ size_t tile_off(int r, int k8) {  // k8: first of 8 consecutive K elements
  return size_t(r / 8) * 256 + size_t(k8 / 8) * 64 + size_t(r % 8) * 8;
}

__device__ __forceinline__ void store8(__half* dst, const __half (&v)[8]) {
  uint4 u;
  u.x = uint32_t(__half_as_ushort(v[0])) | (uint32_t(__half_as_ushort(v[1])) << 16);
  u.y = uint32_t(__half_as_ushort(v[2])) | (uint32_t(__half_as_ushort(v[3])) << 16);
  u.z = uint32_t(__half_as_ushort(v[4])) | (uint32_t(__half_as_ushort(v[5])) << 16);
  u.w = uint32_t(__half_as_ushort(v[6])) | (uint32_t(__half_as_ushort(v[7])) << 16);
  *reinterpret_cast<uint4*>(dst) = u;
}

// Row exponents and row slices of A (rows x kdim): e[q][i], and the A tiles of every slice
// (zero padding to rows_pad x k_pad). One block per row; a thread cuts 8 consecutive K.
__global__ void oz_slice_rows_kernel(Mat A, int rows, int kdim, int rows_pad, int k_pad, int nb,
                                     const int* __restrict__ map, int* __restrict__ e,
                                     __half* __restrict__ out) {
  const int i = blockIdx.x, q = blockIdx.y;
  const double* row = A.p + mat_of(map, q) * A.stride + int64_t(i) * A.ld;
  __shared__ int red[256];
  int E = 0;
  if (i < rows)
    for (int k = threadIdx.x; k < kdim; k += blockDim.x) E = max(E, exp_field(row[k]));
  red[threadIdx.x] = E;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = max(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  const int ex = scale_exp(red[0]);
  if (threadIdx.x == 0) e[size_t(q) * rows_pad + i] = ex;
  const size_t plane = size_t(nb) * rows_pad * k_pad;
  const int kt = k_pad / OZ_KB;
  __half* tile_row = out + (size_t(q) * (rows_pad / OZ_BM) + i / OZ_BM) * kt * (OZ_BM * OZ_KB);
  for (int k8 = threadIdx.x * 8; k8 < k_pad; k8 += blockDim.x * 8) {
    __half d[8][OZ_S];
#pragma unroll
    for (int u = 0; u < 8; ++u) slice_digits((i < rows && k8 + u < kdim) ? row[k8 + u] : 0.0, ex, d[u]);
    __half* dst = tile_row + size_t(k8 / OZ_KB) * (OZ_BM * OZ_KB) + tile_off(i % OZ_BM, k8 % OZ_KB);
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
      __half v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = d[u][s];
      store8(dst + s * plane, v);
    }
  }
}

// f[q][j]: the scale exponent of column j of B (kdim x cols); columns past cols get 0's.
__global__ void oz_colexp_kernel(Mat B, int kdim, int cols, int cols_pad, const int* __restrict__ map,
                                 int* __restrict__ f) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
  if (j >= cols_pad) return;
  const double* col = B.p + mat_of(map, q) * B.stride + j;
  int E = 0;
  if (j < cols) {
#pragma unroll 8
    for (int k = 0; k < kdim; ++k) E = max(E, exp_field(col[int64_t(k) * B.ld]));
  }
  f[size_t(q) * cols_pad + j] = scale_exp(E);
}

// Column slices of B, transposed into the B tiles (row j of a tile = column j of B). A block
// takes 32 columns x 32 K through shared memory (coalesced reads along j); a thread then cuts
// 8 consecutive K of one column.
__global__ void oz_slice_cols_kernel(Mat B, int kdim, int cols, int k_pad, int cols_pad, int nb,
                                     const int* __restrict__ map, const int* __restrict__ f,
                                     __half* __restrict__ out) {
  __shared__ double tile[32][33];
  const int j0 = blockIdx.x * 32, k0 = blockIdx.y * 32, q = blockIdx.z;
  const double* base = B.p + mat_of(map, q) * B.stride;
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int r = e / 32, c = e % 32;  // r: K, c: column
    const int k = k0 + r, j = j0 + c;
    tile[r][c] = (k < kdim && j < cols) ? base[int64_t(k) * B.ld + j] : 0.0;
  }
  __syncthreads();
  const size_t plane = size_t(nb) * cols_pad * k_pad;
  const int kt = k_pad / OZ_KB;
  const int c = threadIdx.x % 32, k8 = (threadIdx.x / 32) * 8;  // blockDim 128: 32 columns x 4 chunks
  const int j = j0 + c;
  const int fx = f[size_t(q) * cols_pad + j];
  __half d[8][OZ_S];
#pragma unroll
  for (int u = 0; u < 8; ++u) slice_digits(tile[k8 + u][c], fx, d[u]);
  __half* dst = out + ((size_t(q) * (cols_pad / OZ_BN) + j / OZ_BN) * kt + k0 / OZ_KB) * (OZ_BN * OZ_KB) +
                tile_off(j % OZ_BN, k8);
#pragma unroll
  for (int t = 0; t < OZ_S; ++t) {
    __half v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = d[u][t];
    store8(dst + t * plane, v);
  }
}

struct OzParams {
  int M, N;                  // output rows and columns
  int m_pad, n_pad, k_pad;   // padded to 128 / 64 / 64
  int mt, nt;                // 128-row / 64-column tiles per matrix
  const __half* sa;          // A tiles [OZ_S][batch][mt][kt][OZ_BM x OZ_KB]
  const __half* sb;          // B tiles [OZ_S][batch][nt][kt][OZ_BN x OZ_KB]
  size_t planeA, planeB;     // halves per slice plane
  const int* map;            // batch index -> matrix of C and D (null: identity)
  const int* e;              // [batch][m_pad] row exponents of A
  const int* f;              // [batch][n_pad] column exponents of B
  Mat D;                     // addend (may alias C; p null: none)
  int zr0, zr1;              // rows [zr0, zr1) of D read as zero
  MatOut C;
  int* err;
};

__device__ __forceinline__ void ff_add(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  hi = s;
  lo = __fadd_rn(lo, e);
}

// One 128 x 64 output tile of one matrix per CTA. K blocks of 32 (all slices of A and B: 84 KB)
// go through a two-stage ring, so the copies of one block overlap the MMAs of the other; every
// OZ_CHUNK blocks (a 128-wide exact chunk) the epilogue drains the OZ_S level accumulators into
// float-float registers level by level, and the MMAs of the next chunk start on a level as
// soon as it has been drained.
__global__ void __launch_bounds__(OZ_THREADS, 1)
    oz_gemm_kernel(const __grid_constant__ OzParams p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // (offset arithmetic on the shared array keeps the pointers in the shared address space)
  uint8_t* smem = smem_raw + ((1024u - (ptx::smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + OZ_STAGES * OZ_STAGE);
  uint64_t* full = bars;                   // [OZ_STAGES] stage loaded
  uint64_t* empty = bars + OZ_STAGES;      // [OZ_STAGES] stage consumed by the MMAs
  uint64_t* accf = bars + 2 * OZ_STAGES;   // chunk accumulators ready
  uint64_t* acce = accf + 1;               // [OZ_S] level drained
  uint32_t* tslot = reinterpret_cast<uint32_t*>(acce + OZ_S);
  __shared__ volatile int s_abort;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int t = blockIdx.x;
  const int b = t / (p.mt * p.nt), rem = t % (p.mt * p.nt);  // b: index within the product batch
  const int mb = rem / p.nt, nbk = rem % p.nt;
  const int nkb = p.k_pad / OZ_KB;
  const int nchunk = (nkb + OZ_CHUNK - 1) / OZ_CHUNK;

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int q = 0; q < OZ_STAGES; ++q) {
      ptx::mbar_init(&full[q], 1);
      ptx::mbar_init(&empty[q], 1);
    }
    ptx::mbar_init(accf, 1);
    for (int L = 0; L < OZ_S; ++L) ptx::mbar_init(&acce[L], 4);
    ptx::fence_barrier_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(tslot, 512);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tslot;
  const __half* tA = p.sa + (size_t(b) * p.mt + mb) * nkb * (OZ_BM * OZ_KB);  // slice 0, K block 0
  const __half* tB = p.sb + (size_t(b) * p.nt + nbk) * nkb * (OZ_BN * OZ_KB);

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int kb = 0; kb < nkb && !s_abort; ++kb) {
        const int q = kb % OZ_STAGES, use = kb / OZ_STAGES;
        if (use > 0 && !ptx::mbar_wait(&empty[q], (use - 1) & 1, OZ_WAIT_NS)) {
          atomicExch(p.err, 1);
          s_abort = 1;
          break;
        }
        uint8_t* st = smem + q * OZ_STAGE;
        ptx::mbar_arrive_expect_tx(&full[q], OZ_STAGE);
#pragma unroll
        for (int s = 0; s < OZ_S; ++s) {
          ptx::bulk_load(st + s * OZ_A_BYTES, tA + s * p.planeA + size_t(kb) * (OZ_BM * OZ_KB), OZ_A_BYTES, &full[q]);
          ptx::bulk_load(st + OZ_S * OZ_A_BYTES + s * OZ_B_BYTES, tB + s * p.planeB + size_t(kb) * (OZ_BN * OZ_KB),
                         OZ_B_BYTES, &full[q]);
        }
        issued = kb + 1;
      }
      // every copy issued has landed before the CTA can exit
      for (int kb = std::max(0, issued - OZ_STAGES); kb < issued; ++kb)
        ptx::mbar_wait(&full[kb % OZ_STAGES], (kb / OZ_STAGES) & 1, OZ_WAIT_NS);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = ptx::idesc_f16_f32(OZ_BM, OZ_BN);
      bool ok = true;
      for (int kb = 0; kb < nkb && ok; ++kb) {
        const int q = kb % OZ_STAGES, use = kb / OZ_STAGES;
        const int c = kb / OZ_CHUNK;
        const bool first = kb % OZ_CHUNK == 0, last = kb % OZ_CHUNK == OZ_CHUNK - 1 || kb == nkb - 1;
        if (!ptx::mbar_wait(&full[q], use & 1, OZ_WAIT_NS)) { ok = false; break; }
        ptx::tc_fence_after();
        const uint32_t base = ptx::smem_u32(smem + q * OZ_STAGE);
        for (int L = 0; L < OZ_S && ok; ++L) {
          // the first block of a chunk overwrites level L: wait until the epilogue drained it
          if (first && c > 0) {
            if (!ptx::mbar_wait(&acce[L], (c - 1) & 1, OZ_WAIT_NS)) { ok = false; break; }
            ptx::tc_fence_after();
          }
          const uint32_t acc = tmem + L * OZ_BN;
          for (int s = 0; s <= L; ++s) {
            const uint64_t dA = ptx::plain_kmajor_desc(base + s * OZ_A_BYTES, 128, 512);
            const uint64_t dB = ptx::plain_kmajor_desc(base + OZ_S * OZ_A_BYTES + (L - s) * OZ_B_BYTES, 128, 512);
#pragma unroll
            for (int kk = 0; kk < OZ_KB / 16; ++kk) {
              const uint64_t adv = uint64_t(kk * 256) >> 4;  // 16 K = two core matrices = 256 B
              ptx::mma_f16(acc, dA + adv, dB + adv, idesc, (first && s == 0 && kk == 0) ? 0u : 1u);
            }
          }
        }
        if (!ok) break;
        ptx::mma_commit(&empty[q]);
        if (last) ptx::mma_commit(accf);
      }
      if (!ok) {
        atomicExch(p.err, 2);
        s_abort = 1;
      }
    }
  } else {
    // Thread = output row (TMEM lane); hi/lo hold the float-float running sum of its 64 columns.
    const int lane_base = 32 * (warp & 3);
    {  // bring this thread's row of the addend tile into L2 while the MMAs run
      const int i = mb * OZ_BM + lane_base + lane;
      if (p.D.p && i < p.M && (i < p.zr0 || i >= p.zr1)) {
        const double* drow = p.D.p + mat_of(p.map, b) * p.D.stride + int64_t(i) * p.D.ld + nbk * OZ_BN;
        const int ncol = min(OZ_BN, p.N - nbk * OZ_BN);
        for (int j = 0; j < ncol; j += 16) asm volatile("prefetch.global.L2 [%0];" ::"l"(drow + j));
      }
    }
    float hi[OZ_BN], lo[OZ_BN];
#pragma unroll
    for (int j = 0; j < OZ_BN; ++j) hi[j] = lo[j] = 0.0f;
    bool ok = true;
    for (int c = 0; c < nchunk; ++c) {
      if (s_abort || !ptx::mbar_wait(accf, c & 1, OZ_WAIT_NS)) { ok = false; break; }
      ptx::tc_fence_after();
#pragma unroll 1
      for (int L = 0; L < OZ_S; ++L) {
        const float sc = __int_as_float((127 - 7 * L) << 23);  // 2^-7L: exact scaling
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t r[32];
          ptx::tmem_ld_32x32b_x32(tmem + (uint32_t(lane_base) << 16) + uint32_t(L * OZ_BN + 32 * h), r);
          if (h == 1) {  // level L is in registers: the MMAs of the next chunk may overwrite it
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&acce[L]);
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) ff_add(hi[32 * h + j], lo[32 * h + j], __fmul_rn(__uint_as_float(r[j]), sc));
        }
      }
    }
    if (!ok) {
      atomicExch(p.err, 3);
    } else {
      // Every MMA has completed (the last accf phase), so the stage buffer is free: each warp
      // stages its 32 rows x 64 columns there (hi, lo as floats; the addend tile in FP64) and
      // writes C row by row, coalesced. C = (hi + lo) 2^(e_i + f_j - 14) + D: the scaled
      // doubles come from the float bits, leaving one or two FP64 adds per element.
      const int cb = mat_of(p.map, b);
      const int i = mb * OZ_BM + lane_base + lane;
      const int ei = (i < p.M ? p.e[size_t(b) * p.m_pad + i] : 0) - 14;
      float2* stile = reinterpret_cast<float2*>(smem) + (warp & 3) * 32 * (OZ_BN + 1);
      double* sd = reinterpret_cast<double*>(smem + 4 * 32 * (OZ_BN + 1) * sizeof(float2)) + (warp & 3) * 32 * OZ_BN;
#pragma unroll
      for (int j = 0; j < OZ_BN; ++j) stile[lane * (OZ_BN + 1) + j] = make_float2(hi[j], lo[j]);
      if (p.D.p) {  // loads only, 8 rows in flight at a time (C may alias D)
#pragma unroll 1
        for (int r0 = 0; r0 < 32; r0 += 8) {
          double t[8][2];
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const int ir = mb * OZ_BM + lane_base + r0 + r;
            const bool use = ir < p.M && (ir < p.zr0 || ir >= p.zr1);
            const double* drow = p.D.p + cb * p.D.stride + int64_t(ir) * p.D.ld;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int jj = nbk * OZ_BN + 32 * h + lane;
              t[r][h] = (use && jj < p.N) ? drow[jj] : 0.0;
            }
          }
#pragma unroll
          for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int h = 0; h < 2; ++h) sd[(r0 + r) * OZ_BN + 32 * h + lane] = t[r][h];
        }
      }
      __syncwarp();
      int fj[2];  // column exponents of this lane's two columns
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int jj = nbk * OZ_BN + 32 * h + lane;
        fj[h] = jj < p.N ? p.f[size_t(b) * p.n_pad + jj] : 0;
      }
#pragma unroll 2
      for (int r = 0; r < 32; ++r) {
        const int ir = mb * OZ_BM + lane_base + r;
        const int er = __shfl_sync(0xffffffffu, ei, r);
        if (ir < p.M) {
          double* crow = p.C.p + cb * p.C.stride + int64_t(ir) * p.C.ld;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int jj = nbk * OZ_BN + 32 * h + lane;
            const float2 v = stile[r * (OZ_BN + 1) + 32 * h + lane];
            double c = f32_scaled_to_f64(v.x, er + fj[h]) + f32_scaled_to_f64(v.y, er + fj[h]);
            if (p.D.p) c += sd[r * OZ_BN + 32 * h + lane];
            if (jj < p.N) crow[jj] = c;
          }
        }
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 512);
  }
}

}  // namespace

// Workspace for the sliced products of one build batch: slice planes of A and B, exponents.
struct TcGemm {
  int nb = 0;
  size_t a_cap = 0, b_cap = 0, e_cap = 0, f_cap = 0;  // elements
  __half* sa = nullptr;
  __half* sb = nullptr;
  int* e = nullptr;
  int* f = nullptr;
  int* err = nullptr;
};

static inline int pad_to(int x, int m) { return (x + m - 1) / m * m; }

namespace {
struct Caps {
  size_t a, b, e, f;
};
// Room for square n x n products and for the rank-64 updates of an n x gjcols elimination
// (K padded to OZ_KB <= 64 <= the 64-padded n).
Caps caps_for(int n, int nb, int gjcols) {
  const size_t mp = pad_to(n, OZ_BM), np = pad_to(std::max(n, 64), OZ_BN), gp = pad_to(std::max(gjcols, 1), OZ_BN);
  return {size_t(OZ_S) * nb * mp * np, size_t(OZ_S) * nb * std::max(np * np, gp * 64), size_t(nb) * mp,
          size_t(nb) * std::max(np, gp)};
}
}  // namespace

size_t tc_gemm_bytes(int n, int nb, int gjcols) {
  const Caps c = caps_for(n, nb, gjcols);
  return sizeof(__half) * (c.a + c.b) + sizeof(int) * (c.e + c.f) + 16;
}

void tc_gemm_destroy(TcGemm* g, cudaStream_t st) {
  if (!g) return;
  for (void* q : {static_cast<void*>(g->sa), static_cast<void*>(g->sb), static_cast<void*>(g->e),
                  static_cast<void*>(g->f), static_cast<void*>(g->err)})
    if (q) cudaFreeAsync(q, st);
  delete g;
}

lem_status tc_gemm_create(int n, int nb, int gjcols, cudaStream_t st, TcGemm** out) {
  *out = nullptr;
  // the shared-memory attribute is per device (cheap to set again)
  if (cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM) != cudaSuccess)
    return cuda_fail(cudaGetLastError(), "oz_gemm_kernel attributes");
  TcGemm* g = new TcGemm();
  const Caps c = caps_for(n, nb, gjcols);
  g->nb = nb;
  g->a_cap = c.a;
  g->b_cap = c.b;
  g->e_cap = c.e;
  g->f_cap = c.f;
  auto alloc = [&](void** p, size_t bytes) -> bool {
    if (cudaMallocAsync(p, bytes, st) == cudaSuccess) return true;
    cudaGetLastError();
    return false;
  };
  if (!alloc(reinterpret_cast<void**>(&g->sa), sizeof(__half) * c.a) ||
      !alloc(reinterpret_cast<void**>(&g->sb), sizeof(__half) * c.b) ||
      !alloc(reinterpret_cast<void**>(&g->e), sizeof(int) * c.e) ||
      !alloc(reinterpret_cast<void**>(&g->f), sizeof(int) * c.f) ||
      !alloc(reinterpret_cast<void**>(&g->err), sizeof(int))) {
    tc_gemm_destroy(g, st);
    return fail(LEM_ENOMEM, "tensor-core build workspace");
  }
  if (cudaMemsetAsync(g->err, 0, sizeof(int), st) != cudaSuccess) {
    tc_gemm_destroy(g, st);
    return cuda_fail(cudaGetLastError(), "tensor-core build workspace");
  }
  *out = g;
  return LEM_OK;
}

// C[m] = A[m] B[m] + D[m] (D null: no addend; D rows [zr0, zr1) taken as zero) for
// m = map[q], q < nbatch (map a device array, or null for m = q): A is M x K, B is K x N, C and
// D M x N, all row-major FP64 with the given leading dimensions and batch strides. A and B are
// sliced before the product runs, so C may overlap them; D may alias C.
lem_status tc_gemm_ex(TcGemm* g, int nbatch, const int* map, int M, int N, int K, const double* A, int64_t lda,
                      int64_t sA, const double* B, int64_t ldb, int64_t sB, const double* D, int64_t ldd,
                      int64_t sD, int zr0, int zr1, double* C, int64_t ldc, int64_t sC, cudaStream_t st) {
  if (nbatch <= 0 || M <= 0 || N <= 0) return LEM_OK;
  const int m_pad = pad_to(M, OZ_BM), n_pad = pad_to(N, OZ_BN), k_pad = pad_to(std::max(K, 1), OZ_KB);
  if (nbatch > g->nb || size_t(OZ_S) * g->nb * m_pad * k_pad > g->a_cap ||
      size_t(OZ_S) * g->nb * n_pad * k_pad > g->b_cap || size_t(nbatch) * m_pad > g->e_cap ||
      size_t(nbatch) * n_pad > g->f_cap)
    return fail(LEM_EINVAL, "tensor-core product larger than its workspace");
  const Mat mA{A, lda, sA}, mB{B, ldb, sB};
  oz_slice_rows_kernel<<<dim3(m_pad, nbatch), 256, 0, st>>>(mA, M, K, m_pad, k_pad, g->nb, map, g->e, g->sa);
  oz_colexp_kernel<<<dim3((n_pad + 127) / 128, nbatch), 128, 0, st>>>(mB, K, N, n_pad, map, g->f);
  oz_slice_cols_kernel<<<dim3(n_pad / 32, k_pad / 32, nbatch), 128, 0, st>>>(mB, K, N, k_pad, n_pad, g->nb, map,
                                                                              g->f, g->sb);
  LEM_CUDA_TRY(cudaGetLastError());
  OzParams p{};
  p.M = M;
  p.N = N;
  p.m_pad = m_pad;
  p.n_pad = n_pad;
  p.k_pad = k_pad;
  p.mt = m_pad / OZ_BM;
  p.nt = n_pad / OZ_BN;
  p.sa = g->sa;
  p.sb = g->sb;
  p.planeA = size_t(g->nb) * m_pad * k_pad;
  p.planeB = size_t(g->nb) * n_pad * k_pad;
  p.map = map;
  p.e = g->e;
  p.f = g->f;
  p.D = Mat{D, ldd, sD};
  p.zr0 = zr0;
  p.zr1 = zr1;
  p.C = MatOut{C, ldc, sC};
  p.err = g->err;
  oz_gemm_kernel<<<nbatch * p.mt * p.nt, OZ_THREADS, OZ_SMEM, st>>>(p);
  LEM_CUDA_TRY(cudaGetLastError());
  return LEM_OK;
}

// Square n x n matrices stored back to back.
lem_status tc_gemm(TcGemm* g, int n, int nbatch, const int* map, const double* A, const double* B, const double* D,
                   double* C, cudaStream_t st) {
  const int64_t nn = int64_t(n) * n;
  return tc_gemm_ex(g, nbatch, map, n, n, n, A, n, nn, B, n, nn, D, n, nn, 0, 0, C, n, nn, st);
}

// Error flag of the workspace's products (reads it after synchronising st).
lem_status tc_gemm_check(TcGemm* g, cudaStream_t st) {
  int e = 0;
  LEM_CUDA_TRY(cudaMemcpyAsync(&e, g->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  LEM_CUDA_TRY(cudaStreamSynchronize(st));
  if (e != 0) {
    cudaMemsetAsync(g->err, 0, sizeof(int), st);
    return fail(LEM_ETIMEOUT, "tensor-core build product gave up waiting on an mbarrier (code " +
                                  std::to_string(e) + ")");
  }
  return LEM_OK;
}

}  // namespace lem
