// FP64 batched GEMM for the propagator builder and the plain FP64 apply.
//   C[b](m, n) = alpha * sum_k A[b](m, k) * B[b](k, n) + beta * C[b](m, n)
// Row-major operands. transB = 1 reads B(k, n) from B[n * ldb + k] (B stored N x K).
// An optional row index maps A row m and C row m to rowidx[m] (gathered rows), which the
// step uses to apply one class propagator to the tiles of that class.
// GB300 runs FP64 at about 1.2 TFLOP/s (two DFMA per clock per SM), so this kernel is
// bound by the FP64 pipe: 64 x 64 CTA tile, 4 x 4 outputs per thread, 16-deep K slabs
// staged in shared memory; loads are guarded so any M, N, K works.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lem {

struct DgemmArgs {
  int M, N, K;
  const double* A; int64_t lda; int64_t sA;
  const double* B; int64_t ldb; int64_t sB; int transB;
  double* C; int64_t ldc; int64_t sC;
  double alpha, beta;
  const int32_t* rowidx;  // optional (nullptr): A/C row m -> rowidx[m]
};

constexpr int DG_BM = 64, DG_BN = 64, DG_BK = 16;

static __global__ void __launch_bounds__(256) dgemm_kernel(DgemmArgs g) {
  __shared__ double As[DG_BK][DG_BM + 1];
  __shared__ double Bs[DG_BK][DG_BN + 1];
  const int b = blockIdx.z;
  const double* A = g.A + b * g.sA;
  const double* B = g.B + b * g.sB;
  double* C = g.C + b * g.sC;
  const int m0 = blockIdx.y * DG_BM, n0 = blockIdx.x * DG_BN;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < g.K; k0 += DG_BK) {
    // A slab: 64 rows x 16 k -> 1024 values, 4 per thread (k fastest for coalescing)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int e = tid + r * 256;
      int mm = e / DG_BK, kk = e % DG_BK;
      int m = m0 + mm, k = k0 + kk;
      double v = 0.0;
      if (m < g.M && k < g.K) {
        int64_t row = g.rowidx ? int64_t(g.rowidx[m]) : int64_t(m);
        v = A[row * g.lda + k];
      }
      As[kk][mm] = v;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int e = tid + r * 256;
      int nn, kk;
      if (g.transB) { nn = e / DG_BK; kk = e % DG_BK; } else { kk = e / DG_BN; nn = e % DG_BN; }
      int n = n0 + nn, k = k0 + kk;
      double v = 0.0;
      if (n < g.N && k < g.K) v = g.transB ? B[int64_t(n) * g.ldb + k] : B[int64_t(k) * g.ldb + n];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < DG_BK; ++kk) {
      double a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int m = m0 + ty + 16 * i;
    if (m >= g.M) continue;
    int64_t row = g.rowidx ? int64_t(g.rowidx[m]) : int64_t(m);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int n = n0 + tx + 16 * j;
      if (n >= g.N) continue;
      double* c = C + row * g.ldc + n;
      double v = g.alpha * acc[i][j];
      if (g.beta != 0.0) v = fma(g.beta, *c, v);
      *c = v;
    }
  }
}

inline cudaError_t dgemm(const DgemmArgs& g, int batch, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || batch <= 0) return cudaSuccess;
  dim3 grid((g.N + DG_BN - 1) / DG_BN, (g.M + DG_BM - 1) / DG_BM, batch);
  dgemm_kernel<<<grid, 256, 0, st>>>(g);
  return cudaGetLastError();
}

// C = alpha * A * B + beta * C on batches of square n x n row-major matrices.
inline cudaError_t dgemm_sq(int n, int batch, const double* A, const double* B, double* C,
                            double alpha, double beta, cudaStream_t st, int ldb_cols = -1,
                            int ncols = -1) {
  DgemmArgs g{};
  g.M = n; g.K = n;
  g.N = ncols < 0 ? n : ncols;
  int64_t ld = ldb_cols < 0 ? n : ldb_cols;
  g.A = A; g.lda = n; g.sA = int64_t(n) * n;
  g.B = B; g.ldb = ld; g.sB = int64_t(n) * ld; g.transB = 0;
  g.C = C; g.ldc = ld; g.sC = int64_t(n) * ld;
  g.alpha = alpha; g.beta = beta; g.rowidx = nullptr;
  return dgemm(g, batch, st);
}

}  // namespace lem
