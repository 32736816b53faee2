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
constexpr int OZ_KB = 64;   // K elements per block (one 128-byte swizzled row)
constexpr int OZ_A_BYTES = OZ_BM * OZ_KB * 2;
constexpr int OZ_B_BYTES = OZ_BN * OZ_KB * 2;
constexpr int OZ_STAGE = OZ_S * (OZ_A_BYTES + OZ_B_BYTES);  // 168 KB: one stage
constexpr int OZ_SMEM = OZ_STAGE + 1024 + 256;
constexpr int OZ_THREADS = 192;                             // producer, MMA issuer, 4 epilogue warps
constexpr uint64_t OZ_WAIT_NS = 2000000000ull;

// 2^e as a double (built from its bits in the normal range).
__device__ __forceinline__ double pow2d(int e) {
  return (e >= -1022 && e <= 1023) ? __longlong_as_double(static_cast<long long>(e + 1023) << 52) : ldexp(1.0, e);
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

// Row exponents and row slices of A (rows x kdim): e[q][i] and out[s][q][i][k] (K contiguous,
// rows_pad x k_pad per (s, q), zero padding). One block per row.
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
  for (int k = threadIdx.x; k < k_pad; k += blockDim.x) {
    __half d[OZ_S];
    slice_digits((i < rows && k < kdim) ? row[k] : 0.0, ex, d);
    const size_t o = (size_t(q) * rows_pad + i) * k_pad + k;
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) out[s * plane + o] = d[s];
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

// Column slices of B, transposed: out[t][q][j][k] = slice t of B[k][j] 2^-f_j. 32 x 32 tiles
// through shared memory keep both the reads (along j) and the writes (along k) coalesced.
__global__ void oz_slice_cols_kernel(Mat B, int kdim, int cols, int k_pad, int cols_pad, int nb,
                                     const int* __restrict__ map, const int* __restrict__ f,
                                     __half* __restrict__ out) {
  __shared__ double tile[32][33];
  const int j0 = blockIdx.x * 32, k0 = blockIdx.y * 32, q = blockIdx.z;
  const double* base = B.p + mat_of(map, q) * B.stride;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int k = k0 + r, j = j0 + tx;
    tile[r][tx] = (k < kdim && j < cols) ? base[int64_t(k) * B.ld + j] : 0.0;
  }
  __syncthreads();
  const size_t plane = size_t(nb) * cols_pad * k_pad;
  for (int r = ty; r < 32; r += 8) {
    const int j = j0 + r, k = k0 + tx;
    __half d[OZ_S];
    slice_digits(tile[tx][r], f[size_t(q) * cols_pad + j], d);
    const size_t o = (size_t(q) * cols_pad + j) * k_pad + k;
#pragma unroll
    for (int t = 0; t < OZ_S; ++t) out[t * plane + o] = d[t];
  }
}

struct OzParams {
  int M, N;                  // output rows and columns
  int m_pad, n_pad, k_pad;   // padded to 128 / 64 / 64
  int mt, nt;                // 128-row / 64-column tiles per matrix
  int planeA, planeB;        // rows of one slice plane in the A / B tensor maps
  const int* map;            // batch index -> matrix of C and D (null: identity)
  const int* e;              // [batch][m_pad] row exponents of A
  const int* f;              // [batch][n_pad] column exponents of B
  Mat D;                     // addend (may alias C; p null: none)
  int zr0, zr1;              // rows [zr0, zr1) of D read as zero
  MatOut C;
  double alpha, beta;
  int* err;
};

__device__ __forceinline__ void ff_add(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  hi = s;
  lo = __fadd_rn(lo, e);
}

// One 128 x 64 output tile of one matrix per CTA. K blocks of 64 are loaded one at a time
// (all slices of A and B: 168 KB); every 2 K blocks (a 128-wide exact chunk) the epilogue
// drains the OZ_S level accumulators into float-float registers.
__global__ void __launch_bounds__(OZ_THREADS, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, OzParams p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + OZ_STAGE);
  uint64_t* full = bars;       // stage loaded
  uint64_t* empty = bars + 1;  // stage consumed by the MMAs
  uint64_t* accf = bars + 2;   // chunk accumulators ready
  uint64_t* acce = bars + 3;   // chunk accumulators drained
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 4);
  __shared__ volatile int s_abort;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int t = blockIdx.x;
  const int b = t / (p.mt * p.nt), rem = t % (p.mt * p.nt);  // b: index within the product batch
  const int mb = rem / p.nt, nbk = rem % p.nt;
  const int nkb = p.k_pad / OZ_KB;
  const int nchunk = (nkb + 1) / 2;

  if (threadIdx.x == 0) {
    s_abort = 0;
    ptx::mbar_init(full, 1);
    ptx::mbar_init(empty, 1);
    ptx::mbar_init(accf, 1);
    ptx::mbar_init(acce, 4);
    ptx::fence_barrier_init();
    ptx::tma_prefetch_desc(&tmA);
    ptx::tma_prefetch_desc(&tmB);
  }
  if (warp == 1) {
    ptx::tmem_alloc(tslot, 512);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tslot;
  const int rowA = b * p.m_pad + mb * OZ_BM;  // row of the (s = 0) slice plane
  const int rowB = b * p.n_pad + nbk * OZ_BN;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int kb = 0; kb < nkb && !s_abort; ++kb) {
        if (kb > 0 && !ptx::mbar_wait(empty, (kb - 1) & 1, OZ_WAIT_NS)) {
          atomicExch(p.err, 1);
          s_abort = 1;
          break;
        }
        ptx::mbar_arrive_expect_tx(full, OZ_STAGE);
#pragma unroll
        for (int s = 0; s < OZ_S; ++s) {
          ptx::tma_load_2d(smem + s * OZ_A_BYTES, &tmA, full, kb * OZ_KB, s * p.planeA + rowA);
          ptx::tma_load_2d(smem + OZ_S * OZ_A_BYTES + s * OZ_B_BYTES, &tmB, full, kb * OZ_KB, s * p.planeB + rowB);
        }
        issued = kb + 1;
      }
      if (issued > 0) ptx::mbar_wait(full, (issued - 1) & 1, OZ_WAIT_NS);  // the last copies landed
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = ptx::idesc_f16_f32(OZ_BM, OZ_BN);
      bool ok = true;
      for (int kb = 0; kb < nkb && ok; ++kb) {
        const int c = kb / 2;
        const bool first = kb % 2 == 0, last = kb % 2 == 1 || kb == nkb - 1;
        if (first && c > 0 && !ptx::mbar_wait(acce, (c - 1) & 1, OZ_WAIT_NS)) { ok = false; break; }
        if (!ptx::mbar_wait(full, kb & 1, OZ_WAIT_NS)) { ok = false; break; }
        ptx::tc_fence_after();
        const uint32_t base = ptx::smem_u32(smem);
        for (int L = 0; L < OZ_S; ++L) {
          const uint32_t acc = tmem + L * OZ_BN;
          for (int s = 0; s <= L; ++s) {
            const int tt = L - s;
            const uint64_t dA = ptx::sw128_kmajor_desc(base + s * OZ_A_BYTES);
            const uint64_t dB = ptx::sw128_kmajor_desc(base + OZ_S * OZ_A_BYTES + tt * OZ_B_BYTES);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t adv = uint64_t(kk * 32) >> 4;
              ptx::mma_f16(acc, dA + adv, dB + adv, idesc, (first && s == 0 && kk == 0) ? 0u : 1u);
            }
          }
        }
        ptx::mma_commit(empty);
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
#pragma unroll
          for (int j = 0; j < 32; ++j) ff_add(hi[32 * h + j], lo[32 * h + j], __fmul_rn(__uint_as_float(r[j]), sc));
        }
      }
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(acce);
    }
    if (!ok) {
      atomicExch(p.err, 3);
    } else {
      // Every MMA has completed (the last accf phase), so the stage buffer is free: each warp
      // stages its 32 rows x 64 columns of C there and writes them row by row, coalesced.
      const int cb = mat_of(p.map, b);
      const int i = mb * OZ_BM + lane_base + lane;
      const double rs = pow2d((i < p.M ? p.e[size_t(b) * p.m_pad + i] : 0) - 14);  // row scale
      double* stile = reinterpret_cast<double*>(smem) + (warp & 3) * 32 * (OZ_BN + 1);
#pragma unroll
      for (int j = 0; j < OZ_BN; ++j) stile[lane * (OZ_BN + 1) + j] = (double(hi[j]) + double(lo[j])) * rs;
      __syncwarp();
      double cs[2];  // column scales of this lane's two columns
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int jj = nbk * OZ_BN + 32 * h + lane;
        cs[h] = pow2d(jj < p.N ? p.f[size_t(b) * p.n_pad + jj] : 0) * p.alpha;
      }
      for (int r = 0; r < 32; ++r) {
        const int ir = mb * OZ_BM + lane_base + r;
        if (ir >= p.M) break;
        double* crow = p.C.p + cb * p.C.stride + int64_t(ir) * p.C.ld;
        const double* drow =
            (p.D.p && (ir < p.zr0 || ir >= p.zr1)) ? p.D.p + cb * p.D.stride + int64_t(ir) * p.D.ld : nullptr;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int jj = nbk * OZ_BN + 32 * h + lane;
          if (jj < p.N) {
            const double v = stile[r * (OZ_BN + 1) + 32 * h + lane] * cs[h];
            crow[jj] = drow ? fma(p.beta, drow[jj], v) : v;
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
// Room for square n x n products and for the rank-64 updates of an n x gjcols elimination.
Caps caps_for(int n, int nb, int gjcols) {
  const size_t mp = pad_to(n, OZ_BM), np = pad_to(n, OZ_BN), gp = pad_to(std::max(gjcols, 1), OZ_BN);
  return {size_t(OZ_S) * nb * mp * np, size_t(OZ_S) * nb * std::max(np * np, gp * OZ_KB), size_t(nb) * mp,
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
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM) != cudaSuccess)
      return cuda_fail(cudaGetLastError(), "oz_gemm_kernel attributes");
    attr_set = true;
  }
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

// C[m] = alpha A[m] B[m] + beta D[m] (D rows [zr0, zr1) taken as zero) for m = map[q],
// q < nbatch (map a device array, or null for m = q): A is M x K, B is K x N, C and D M x N,
// all row-major FP64 with the given leading dimensions and batch strides. D may alias C
// (each element is read before it is written by the same thread); C must not overlap A or B.
lem_status tc_gemm_ex(TcGemm* g, int nbatch, const int* map, int M, int N, int K, const double* A, int64_t lda,
                      int64_t sA, const double* B, int64_t ldb, int64_t sB, const double* D, int64_t ldd,
                      int64_t sD, int zr0, int zr1, double* C, int64_t ldc, int64_t sC, double alpha, double beta,
                      cudaStream_t st) {
  if (nbatch <= 0 || M <= 0 || N <= 0) return LEM_OK;
  const int m_pad = pad_to(M, OZ_BM), n_pad = pad_to(N, OZ_BN), k_pad = pad_to(std::max(K, 1), OZ_KB);
  if (nbatch > g->nb || size_t(OZ_S) * g->nb * m_pad * k_pad > g->a_cap ||
      size_t(OZ_S) * g->nb * n_pad * k_pad > g->b_cap || size_t(nbatch) * m_pad > g->e_cap ||
      size_t(nbatch) * n_pad > g->f_cap)
    return fail(LEM_EINVAL, "tensor-core product larger than its workspace");
  const Mat mA{A, lda, sA}, mB{B, ldb, sB};
  oz_slice_rows_kernel<<<dim3(m_pad, nbatch), 256, 0, st>>>(mA, M, K, m_pad, k_pad, g->nb, map, g->e, g->sa);
  oz_colexp_kernel<<<dim3((n_pad + 127) / 128, nbatch), 128, 0, st>>>(mB, K, N, n_pad, map, g->f);
  oz_slice_cols_kernel<<<dim3(n_pad / 32, k_pad / 32, nbatch), 256, 0, st>>>(mB, K, N, k_pad, n_pad, g->nb, map,
                                                                              g->f, g->sb);
  LEM_CUDA_TRY(cudaGetLastError());
  // slice planes: A [OZ_S][nb][m_pad][k_pad], B [OZ_S][nb][n_pad][k_pad] (fp16, K contiguous)
  CUtensorMap tmA, tmB;
  const cuuint64_t dimsA[2] = {cuuint64_t(k_pad), cuuint64_t(OZ_S) * g->nb * m_pad};
  const cuuint64_t dimsB[2] = {cuuint64_t(k_pad), cuuint64_t(OZ_S) * g->nb * n_pad};
  const cuuint64_t strides[1] = {cuuint64_t(k_pad) * 2};
  const cuuint32_t boxA[2] = {OZ_KB, OZ_BM}, boxB[2] = {OZ_KB, OZ_BN};
  LEM_TRY(encode_f16_map(&tmA, g->sa, 2, dimsA, strides, boxA, "A slices"));
  LEM_TRY(encode_f16_map(&tmB, g->sb, 2, dimsB, strides, boxB, "B slices"));
  OzParams p{};
  p.M = M;
  p.N = N;
  p.m_pad = m_pad;
  p.n_pad = n_pad;
  p.k_pad = k_pad;
  p.mt = m_pad / OZ_BM;
  p.nt = n_pad / OZ_BN;
  p.planeA = g->nb * m_pad;
  p.planeB = g->nb * n_pad;
  p.map = map;
  p.e = g->e;
  p.f = g->f;
  p.D = Mat{beta != 0.0 ? D : nullptr, ldd, sD};
  p.zr0 = zr0;
  p.zr1 = zr1;
  p.C = MatOut{C, ldc, sC};
  p.alpha = alpha;
  p.beta = beta;
  p.err = g->err;
  oz_gemm_kernel<<<nbatch * p.mt * p.nt, OZ_THREADS, OZ_SMEM, st>>>(tmA, tmB, p);
  LEM_CUDA_TRY(cudaGetLastError());
  return LEM_OK;
}

// Square n x n matrices stored back to back.
lem_status tc_gemm(TcGemm* g, int n, int nbatch, const int* map, const double* A, const double* B, const double* D,
                   double* C, double alpha, double beta, cudaStream_t st) {
  const int64_t nn = int64_t(n) * n;
  return tc_gemm_ex(g, nbatch, map, n, n, n, A, n, nn, B, n, nn, D, n, nn, 0, 0, C, n, nn, alpha, beta, st);
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
