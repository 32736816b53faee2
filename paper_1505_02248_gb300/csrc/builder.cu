// Local propagator builder (Sec. 3 step 2; Pade approximation with scaling and squaring
// as named in Sec. 1 and Sec. 4), batched over propagator classes, in FP64. For the
// split-precision tiers the matrix products run on the tensor cores as exact sums of FP16
// slice products (builder_tc.cu, about 2^-45 relative to the operands' scale); the Pade
// denominator solve stays in FP64 either way.
//
// For each class the local matrix X = dt A_M (principal submatrix on the window, i.e.
// Dirichlet data at the artificial boundary; plus dt diag(1 - 3u^2) with the reaction, or
// times diag(phi'(u)) on the right for the porous-medium equation) is
// assembled in a zero-padded n x n frame (padding is an exact block-diagonal embedding).
//   EXP:  P = R_D exp(X)
//   PHI:  P = R_D phi_1(X), the top-right block of exp(Z), Z = [[X, I], [0, 0]].
// The PHI path never forms the 2n x 2n matrix Z: every power and polynomial of Z has the
// form (T, B; beta) = [[T, B], [0, beta I]], and products of such pairs need two n x n
// products. Degree-13 Pade (Higham 2005 coefficients b_j = (2m-j)! m! / ((2m)! j! (m-j)!)),
// s = smallest integer >= 0 with ||Z||_1 / 2^s <= theta_13 from the exact 1-norm,
// (V - U) R = (V + U) by Gauss-Jordan elimination with partial pivoting, then s squarings.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <numeric>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "dgemm.cuh"
#include "lem_internal.h"

namespace lem {

namespace {

constexpr double kTheta13 = 5.371920351148152;

// b_j for m = 13 as exact rationals (numerator integers / 64764752532480000).
const double kPadeInt[14] = {64764752532480000.0, 32382376266240000.0, 7771770303897600.0,
                             1187353796428800.0,  129060195264000.0,   10559470521600.0,
                             670442572800.0,      33522128640.0,       1323241920.0,
                             40840800.0,          960960.0,            16380.0,
                             182.0,               1.0};

struct BatchClass {
  TileDesc rep;      // representative tile (window geometry)
  int32_t whole[2];
};

// ---------------------------------------------------------------- assembly
// nonlin 1: + dt diag(1 - 3u^2); nonlin 2 (porous medium): X diag(phi'(u)) with
// phi'(u) = m |u|^(m-1), each entry scaled by phi' at its column's node.
__global__ void assemble_local_kernel(double* X, int n, const BatchClass* bc, int nb,
                                      const double* coef, int64_t cstride, int64_t ny,
                                      int64_t nx, int ndim, const double* u, double dt,
                                      int nonlin, double pm) {
  const int b = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb || k >= n) return;
  double* row = X + (int64_t(b) * n + k) * n;
  for (int j = 0; j < n; ++j) row[j] = 0.0;
  const BatchClass c = bc[b];
  const int wy = c.rep.wext[0], wx = c.rep.wext[1];
  if (k >= wy * wx) return;  // padding row
  const int a = k / wx, bb = k % wx;
  int64_t gy = (int64_t(c.rep.org[0]) + a) % ny;
  if (gy < 0) gy += ny;
  int64_t gx = (int64_t(c.rep.org[1]) + bb) % nx;
  if (gx < 0) gx += nx;
  const int64_t p = gy * nx + gx;
  const int64_t npts = ny * nx;
  auto cf = [&](int which) { return coef[which * (cstride ? npts : 1) + (cstride ? p : 0)]; };
  const bool porous = u && nonlin == 2;
  // phi'(u) at global node q (1 unless porous)
  auto dphi = [&](int64_t q) { return porous ? pm * pow(fabs(u[q]), pm - 1.0) : 1.0; };
  // the four neighbours' global nodes (wrapped; a window never holds a node beyond a wall)
  const int64_t qw = gy * nx + (gx + nx - 1) % nx, qe = gy * nx + (gx + 1) % nx;
  const int64_t qs = ((gy + ny - 1) % ny) * nx + gx, qn = ((gy + 1) % ny) * nx + gx;
  double diag = cf(0);
  if (u && nonlin == 1) diag += dt * (1.0 - 3.0 * u[p] * u[p]);
  row[k] += diag * dphi(p);
  // W (x - 1) and E (x + 1): inside the window, or wrapped when it spans the periodic axis
  if (bb >= 1) row[k - 1] += cf(1) * dphi(qw);
  else if (c.whole[1]) row[k + wx - 1] += cf(1) * dphi(qw);
  if (bb + 1 < wx) row[k + 1] += cf(2) * dphi(qe);
  else if (c.whole[1]) row[k + 1 - wx] += cf(2) * dphi(qe);
  if (ndim == 2) {
    if (a >= 1) row[k - wx] += cf(3) * dphi(qs);
    else if (c.whole[0]) row[k + (wy - 1) * wx] += cf(3) * dphi(qs);
    if (a + 1 < wy) row[k + wx] += cf(4) * dphi(qn);
    else if (c.whole[0]) row[k - (wy - 1) * wx] += cf(4) * dphi(qn);
  }
}

// Complex problems: the real embedding [[Re X, -Im X], [Im X, Re X]] of X = dt A_M (n = twice
// the window nodes): row k carries the real part of node k's equation, row n/2 + k the
// imaginary part. Coefficients: real parts at coef[w], imaginary parts at coef[5 + w].
__global__ void assemble_local_complex_kernel(double* X, int n, const BatchClass* bc, int nb, const double* coef,
                                              int64_t cstride, int64_t ny, int64_t nx, int ndim) {
  const int b = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int h = n / 2;
  if (b >= nb || k >= h) return;
  double* rr = X + (int64_t(b) * n + k) * n;
  double* ri = X + (int64_t(b) * n + h + k) * n;
  for (int j = 0; j < n; ++j) rr[j] = ri[j] = 0.0;
  const BatchClass c = bc[b];
  const int wy = c.rep.wext[0], wx = c.rep.wext[1];
  if (k >= wy * wx) return;  // padding node
  const int a = k / wx, bb = k % wx;
  int64_t gy = (int64_t(c.rep.org[0]) + a) % ny;
  if (gy < 0) gy += ny;
  int64_t gx = (int64_t(c.rep.org[1]) + bb) % nx;
  if (gx < 0) gx += nx;
  const int64_t p = gy * nx + gx, npts = ny * nx;
  auto add = [&](int col, int w) {
    const int64_t o = cstride ? p : 0;
    const double cr = coef[int64_t(w) * (cstride ? npts : 1) + o];
    const double ci = coef[int64_t(5 + w) * (cstride ? npts : 1) + o];
    rr[col] += cr;
    rr[h + col] -= ci;
    ri[col] += ci;
    ri[h + col] += cr;
  };
  add(k, 0);
  if (bb >= 1) add(k - 1, 1);
  else if (c.whole[1]) add(k + wx - 1, 1);
  if (bb + 1 < wx) add(k + 1, 2);
  else if (c.whole[1]) add(k + 1 - wx, 2);
  if (ndim == 2) {
    if (a >= 1) add(k - wx, 3);
    else if (c.whole[0]) add(k + (wy - 1) * wx, 3);
    if (a + 1 < wy) add(k + wx, 4);
    else if (c.whole[0]) add(k - (wy - 1) * wx, 4);
  }
}

// column 1-norms -> per-matrix max (non-negative doubles order like their bit patterns)
__global__ void norm1_kernel(const double* X, int n, unsigned long long* out) {
  const int b = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double* M = X + int64_t(b) * n * n;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += fabs(M[int64_t(i) * n + j]);
  atomicMax(out + b, (unsigned long long)__double_as_longlong(s));
}

// out[b] = sum_t w_t in_t[b] + diag * dscale[b] * I   (dscale may be null: 1)
struct Lin {
  const double* in[4];
  double w[4];
  int nin;
  double diag;
  const double* dscale;
  const double* wscale0;  // optional per-batch multiplier of w[0]
};

__global__ void lincomb_kernel(double* out, int n, int64_t ld, int ncols, Lin L) {
  const int b = blockIdx.y;
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= int64_t(n) * ncols) return;
  const int i = int(e / ncols), j = int(e % ncols);
  const int64_t off = int64_t(b) * n * ld + int64_t(i) * ld + j;
  double v = 0.0;
  for (int t = 0; t < L.nin; ++t) {
    double w = L.w[t];
    if (t == 0 && L.wscale0) w *= L.wscale0[b];
    v += w * L.in[t][off];
  }
  if (i == j && L.diag != 0.0) v += L.diag * (L.dscale ? L.dscale[b] : 1.0);
  out[off] = v;
}

// Gauss-Jordan elimination with partial pivoting on G = [Q | RHS] (n x (n + m), row-major).
// Step k: pick the largest |G[i][k]|, i >= k; swap rows; normalise row k by the pivot.
__global__ void gj_pivot_kernel(double* G, int n, int ncols, int k, int* status) {
  const int b = blockIdx.x;
  double* M = G + int64_t(b) * n * ncols;
  __shared__ double sv[256];
  __shared__ int si[256];
  double best = -1.0;
  int bi = k;
  for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
    double v = fabs(M[int64_t(i) * ncols + k]);
    if (v > best) { best = v; bi = i; }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      double o = sv[threadIdx.x + s];
      int oi = si[threadIdx.x + s];
      if (o > sv[threadIdx.x] || (o == sv[threadIdx.x] && oi < si[threadIdx.x])) {
        sv[threadIdx.x] = o;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const int p = si[0];
  const double pv = M[int64_t(p) * ncols + k];
  __syncthreads();  // every thread holds pv before row k / row p are rewritten
  if (!(sv[0] > 0.0) || !isfinite(pv)) {
    if (threadIdx.x == 0) atomicExch(status, int(LEM_ENUMERIC));
    return;
  }
  for (int j = threadIdx.x; j < ncols; j += blockDim.x) {
    double a = M[int64_t(k) * ncols + j];
    double c = M[int64_t(p) * ncols + j];
    if (p != k) M[int64_t(p) * ncols + j] = a;
    M[int64_t(k) * ncols + j] = c / pv;
  }
}

// eliminate column k from every row i != k:  G[i][j] -= G[i][k] * G[k][j], j > k
__global__ void gj_update_kernel(double* G, int n, int ncols, int k) {
  const int b = blockIdx.z;
  double* M = G + int64_t(b) * n * ncols;
  const int i = blockIdx.y;
  if (i == k) return;
  const double f = M[int64_t(i) * ncols + k];
  if (f == 0.0) return;
  for (int j = k + 1 + blockIdx.x * blockDim.x + threadIdx.x; j < ncols; j += gridDim.x * blockDim.x)
    M[int64_t(i) * ncols + j] = fma(-f, M[int64_t(k) * ncols + j], M[int64_t(i) * ncols + j]);
}

// ---------------------------------------------------------------- blocked Gauss-Jordan
// For the tensor-core build the elimination runs in panels of GJ_KB columns. The panel's
// GJ_KB pivot steps (partial pivoting, FP64) are applied to the panel columns and to a tracker
// Y (n x GJ_KB): at step c, right after the row swap, Y[k0 + c][c] = 1 is injected, and every
// later swap, scaling and elimination acts on Y too. At the end of the panel the composite row
// operation is M = T Pi with T = I + W E_K^T (Pi: the panel's swaps, K: rows k0 .. k0 + kb),
// and Y = T[:, K], so the trailing columns become
//   rows K:      Y_K (Pi G)[K, :]
//   other rows:  (Pi G)[i, :] + Y_i (Pi G)[K, :],
// one rank-kb product C = Y B + D with B the permuted pivot rows and D the permuted trailing
// columns with rows K taken as zero. The FP64 work drops from n^2 gjcols to about 2 n^2 GJ_KB.
constexpr int GJ_KB = 64;

__global__ void bgj_pivot_kernel(double* G, int n, int ld, int k0, int c, int kb, double* Y, int* piv,
                                 int* status) {
  const int b = blockIdx.x;
  double* M = G + int64_t(b) * n * ld;
  double* Yb = Y + int64_t(b) * n * GJ_KB;
  const int col = k0 + c, r = k0 + c;
  __shared__ double sv[256];
  __shared__ int si[256];
  double best = -1.0;
  int bi = r;
  for (int i = r + threadIdx.x; i < n; i += blockDim.x) {
    const double v = fabs(M[int64_t(i) * ld + col]);
    if (v > best) { best = v; bi = i; }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double o = sv[threadIdx.x + s];
      const int oi = si[threadIdx.x + s];
      if (o > sv[threadIdx.x] || (o == sv[threadIdx.x] && oi < si[threadIdx.x])) {
        sv[threadIdx.x] = o;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const int p = si[0];
  const double pv = M[int64_t(p) * ld + col];
  __syncthreads();  // every thread holds pv before rows r / p are rewritten
  if (!(sv[0] > 0.0) || !isfinite(pv)) {
    if (threadIdx.x == 0) atomicExch(status, int(LEM_ENUMERIC));
    return;
  }
  if (threadIdx.x == 0) piv[b * GJ_KB + c] = p;
  const double inv = 1.0 / pv;
  // panel columns col .. k0 + kb - 1 of rows r and p, then the tracker rows
  for (int j = col + threadIdx.x; j < k0 + kb; j += blockDim.x) {
    const double a = M[int64_t(r) * ld + j], q = M[int64_t(p) * ld + j];
    if (p != r) M[int64_t(p) * ld + j] = a;
    M[int64_t(r) * ld + j] = q * inv;
  }
  for (int j = threadIdx.x; j < kb; j += blockDim.x) {
    const double a = Yb[int64_t(r) * GJ_KB + j], q = Yb[int64_t(p) * GJ_KB + j];
    if (p != r) Yb[int64_t(p) * GJ_KB + j] = a;
    Yb[int64_t(r) * GJ_KB + j] = (j == c ? 1.0 : q) * inv;  // inject the unit column, then scale
  }
}

// Eliminate panel column k0 + c from every row but the pivot row: 4 rows per block, thread t
// of a row updates panel column k0 + c + 1 + t and tracker column t.
__global__ void bgj_elim_kernel(double* G, int n, int ld, int k0, int c, int kb, double* Y) {
  const int b = blockIdx.y;
  const int i = blockIdx.x * 4 + threadIdx.x / 64, t = threadIdx.x % 64;
  const int r = k0 + c, col = k0 + c;
  if (i >= n || i == r) return;
  double* M = G + int64_t(b) * n * ld;
  double* Yb = Y + int64_t(b) * n * GJ_KB;
  const double f = M[int64_t(i) * ld + col];
  if (f == 0.0) return;
  const int j = col + 1 + t;
  if (j < k0 + kb) M[int64_t(i) * ld + j] = fma(-f, M[int64_t(r) * ld + j], M[int64_t(i) * ld + j]);
  if (t < kb) Yb[int64_t(i) * GJ_KB + t] = fma(-f, Yb[int64_t(r) * GJ_KB + t], Yb[int64_t(i) * GJ_KB + t]);
}

// The panel's row swaps, in order, on the trailing columns j >= k0 + kb.
__global__ void bgj_swap_kernel(double* G, int n, int ld, int k0, int kb, const int* piv) {
  const int b = blockIdx.y;
  const int j = k0 + kb + blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ld) return;
  double* M = G + int64_t(b) * n * ld;
  for (int c = 0; c < kb; ++c) {
    const int p = piv[b * GJ_KB + c];
    if (p == k0 + c) continue;
    const double a = M[int64_t(k0 + c) * ld + j];
    M[int64_t(k0 + c) * ld + j] = M[int64_t(p) * ld + j];
    M[int64_t(p) * ld + j] = a;
  }
}

// rows of the owner tile D inside the window, from the squared result R (n x ld, col0)
__global__ void extract_rows_kernel(double* P, int64_t n_int, int64_t n_loc, const double* R,
                                    int n, int64_t ld, int col0, const BatchClass* bc) {
  const int b = blockIdx.y;
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= n_int * n_loc) return;
  const int i = int(e / n_loc), k = int(e % n_loc);
  const BatchClass c = bc[b];
  const int ie = c.rep.iext[0] * c.rep.iext[1];
  const int wl = c.rep.wext[0] * c.rep.wext[1];
  double v = 0.0;
  if (i < ie && k < wl && k < n) {
    const int row = (c.rep.iofs[0] + i / c.rep.iext[1]) * c.rep.wext[1] + c.rep.iofs[1] + i % c.rep.iext[1];
    v = R[int64_t(b) * n * ld + int64_t(row) * ld + col0 + k];
  }
  P[int64_t(b) * n_int * n_loc + e] = v;
}

// Complex problems: owner rows of the embedded result R (n x n, n = 2 x window nodes) into P
// (n_int x n_loc, both embedded sizes): rows [0, n_int/2) the real parts, [n_int/2, n_int) the
// imaginary parts of the owner nodes; columns as in R (real parts, then imaginary parts).
__global__ void extract_rows_complex_kernel(double* P, int64_t n_int, int64_t n_loc, const double* R, int n,
                                            const BatchClass* bc) {
  const int b = blockIdx.y;
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= n_int * n_loc) return;
  const int i = int(e / n_loc), k = int(e % n_loc);
  const int hi = int(n_int / 2), hn = n / 2;
  const int comp = i / hi, io = i % hi;
  const BatchClass c = bc[b];
  const int ie = c.rep.iext[0] * c.rep.iext[1];
  double v = 0.0;
  if (io < ie && k < n) {
    const int row = (c.rep.iofs[0] + io / c.rep.iext[1]) * c.rep.wext[1] + c.rep.iofs[1] + io % c.rep.iext[1];
    v = R[int64_t(b) * n * n + int64_t(comp * hn + row) * n + k];
  }
  P[int64_t(b) * n_int * n_loc + e] = v;
}

__global__ void copy_cols_kernel(double* dst, int64_t ldd, int dcol0, const double* src, int64_t lds,
                                 int scol0, int n, int ncols) {
  const int b = blockIdx.y;
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= int64_t(n) * ncols) return;
  const int i = int(e / ncols), j = int(e % ncols);
  dst[int64_t(b) * n * ldd + int64_t(i) * ldd + dcol0 + j] = src[int64_t(b) * n * lds + int64_t(i) * lds + scol0 + j];
}

// Builder scratch from cudaMallocAsync. It is freed after the build has synchronised its
// stream, on the legacy stream: that waits for no non-blocking stream, where cudaFree would
// wait for the whole device.
struct Buf {
  double* p = nullptr;
  ~Buf() { if (p) cudaFreeAsync(p, 0); }
};

inline dim3 grid1(int64_t total, int by) { return dim3(unsigned((total + 255) / 256), by); }

}  // namespace

bool builder_uses_tc(int prec) {
  if (prec == LEM_PREC_FP64) return false;
  const char* e = std::getenv("LEM_BUILD_PRODUCTS");  // "fp64": FP64 products in every tier
  return !(e && std::string(e) == "fp64");
}

namespace {
struct TcGuard {
  TcGemm* g = nullptr;
  cudaStream_t st = nullptr;
  ~TcGuard() { tc_gemm_destroy(g, st); }
};
}  // namespace

// Gauss-Jordan elimination of G = [Q | RHS] (nb matrices of n x gjcols): on exit the RHS
// columns hold Q^{-1} RHS. With a tensor-core workspace the blocked form (FP64 panels,
// rank-GJ_KB trailing products on tcgen05); otherwise one FP64 pivot step at a time.
static lem_status solve_gj(lem_ctx* ctx, TcGemm* tcg, double* G, int n, int gjcols, int nb, Buf& ybuf, Buf& pivbuf) {
  cudaStream_t st = ctx->stream;
  if (tcg) {
    LEM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&ybuf.p), sizeof(double) * nb * n * GJ_KB, st));
    LEM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&pivbuf.p), sizeof(int) * nb * GJ_KB, st));
    double* Y = ybuf.p;
    int* piv = reinterpret_cast<int*>(pivbuf.p);
    for (int k0 = 0; k0 < n; k0 += GJ_KB) {
      const int kb = std::min(GJ_KB, n - k0);
      LEM_CUDA_TRY(cudaMemsetAsync(Y, 0, sizeof(double) * nb * n * GJ_KB, st));
      for (int c = 0; c < kb; ++c) {
        bgj_pivot_kernel<<<nb, 256, 0, st>>>(G, n, gjcols, k0, c, kb, Y, piv, ctx->d_status);
        bgj_elim_kernel<<<dim3((n + 3) / 4, nb), 256, 0, st>>>(G, n, gjcols, k0, c, kb, Y);
      }
      const int m_r = gjcols - (k0 + kb);
      bgj_swap_kernel<<<dim3((m_r + 255) / 256, nb), 256, 0, st>>>(G, n, gjcols, k0, kb, piv);
      LEM_CUDA_TRY(cudaGetLastError());
      double* T = G + (k0 + kb);  // trailing columns
      const int64_t sG = int64_t(n) * gjcols;
      LEM_TRY(tc_gemm_ex(tcg, nb, nullptr, n, m_r, kb, Y, GJ_KB, int64_t(n) * GJ_KB,  // A = Y
                         T + int64_t(k0) * gjcols, gjcols, sG,                         // B = pivot rows
                         T, gjcols, sG, k0, k0 + kb,                                   // D, rows K zero
                         T, gjcols, sG, st));
    }
  } else {
    for (int k = 0; k < n; ++k) {
      gj_pivot_kernel<<<nb, 256, 0, st>>>(G, n, gjcols, k, ctx->d_status);
      int bx = std::max(1, std::min(8, (gjcols - k - 1 + 255) / 256));
      gj_update_kernel<<<dim3(bx, n, nb), 256, 0, st>>>(G, n, gjcols, k);
    }
  }
  LEM_CUDA_TRY(cudaGetLastError());
  return LEM_OK;
}

// Build the propagators of classes [c0, c0 + nb) into P (nb x n_int x n_loc).
static lem_status build_batch(lem_ctx* ctx, int c0, int nb, const double* d_state) {
  cudaStream_t st = ctx->stream;
  const int n = int(ctx->n_loc);
  const bool phi = ctx->desc.mode == LEM_MODE_PHI;
  const int64_t nn = int64_t(n) * n;
  std::vector<BatchClass> hbc(nb);
  for (int b = 0; b < nb; ++b) {
    const ClassDesc& c = ctx->classes[c0 + b];
    hbc[b].rep = ctx->tiles[c.rep_tile];
    hbc[b].whole[0] = c.whole[0];
    hbc[b].whole[1] = c.whole[1];
  }
  // device scratch for this batch (freed at return)
  const int nmat = phi ? 16 : 9;
  const int gjcols = phi ? 3 * n : 2 * n;
  Buf scratch, bcbuf, normbuf, scalebuf;
  size_t bytes = sizeof(double) * (size_t(nmat) * nn + size_t(n) * gjcols) * nb;
  LEM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&scratch.p), bytes, st));
  LEM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&bcbuf.p), sizeof(BatchClass) * nb, st));
  LEM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&normbuf.p), sizeof(double) * nb, st));
  LEM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&scalebuf.p), sizeof(double) * 2 * nb, st));
  BatchClass* d_bc = reinterpret_cast<BatchClass*>(bcbuf.p);
  LEM_CUDA_TRY(cudaMemcpyAsync(d_bc, hbc.data(), sizeof(BatchClass) * nb, cudaMemcpyHostToDevice, st));
  double* S = scratch.p;
  auto M = [&](int i) { return S + size_t(i) * nn * nb; };
  double* Xs = M(0); double* T2 = M(1); double* T4 = M(2); double* T6 = M(3);
  double* TW = M(4); double* T3 = M(5); double* UT = M(6); double* VT = M(7); double* RT2 = M(8);
  double *B2 = nullptr, *B4 = nullptr, *B6 = nullptr, *BW = nullptr, *B3 = nullptr, *UB = nullptr,
         *VB = nullptr;
  if (phi) { B2 = M(9); B4 = M(10); B6 = M(11); BW = M(12); B3 = M(13); UB = M(14); VB = M(15); }
  double* G = S + size_t(nmat) * nn * nb;  // n x gjcols per batch entry

  // X = dt A_M (+ reaction Jacobian)
  const double* u = ctx->desc.reaction ? d_state : nullptr;
  if (ctx->cplx)  // the real embedding of the complex window matrix
    assemble_local_complex_kernel<<<dim3((n / 2 + 127) / 128, nb), 128, 0, st>>>(
        Xs, n, d_bc, nb, ctx->d_coef, ctx->desc.coef_stride, ctx->ny, ctx->nx, ctx->desc.ndim);
  else
    assemble_local_kernel<<<dim3((n + 127) / 128, nb), 128, 0, st>>>(
        Xs, n, d_bc, nb, ctx->d_coef, ctx->desc.coef_stride, ctx->ny, ctx->nx, ctx->desc.ndim, u,
        ctx->desc.dt, ctx->desc.reaction, ctx->desc.porous_m);
  LEM_CUDA_TRY(cudaGetLastError());
  // exact 1-norms -> s per class (host decides, same rule as theta_13 scaling)
  LEM_CUDA_TRY(cudaMemsetAsync(normbuf.p, 0, sizeof(double) * nb, st));
  norm1_kernel<<<dim3((n + 127) / 128, nb), 128, 0, st>>>(
      Xs, n, reinterpret_cast<unsigned long long*>(normbuf.p));
  LEM_CUDA_TRY(cudaGetLastError());
  std::vector<double> norms(nb), scales(2 * nb);
  LEM_CUDA_TRY(cudaMemcpyAsync(norms.data(), normbuf.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
  LEM_CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<int> s(nb);
  int smax = 0;
  for (int b = 0; b < nb; ++b) {
    double nz = phi ? std::max(norms[b], 1.0) : norms[b];  // ||[[X, I], [0, 0]]||_1
    int sb = 0;
    while (nz > kTheta13 * std::ldexp(1.0, sb)) ++sb;
    s[b] = sb;
    smax = std::max(smax, sb);
    ctx->squarings[c0 + b] = sb;
    scales[b] = std::ldexp(1.0, -sb);                       // c = 2^-s
    scales[nb + b] = std::ldexp(1.0, -sb) * (kPadeInt[1] / kPadeInt[0]);  // c * b1
  }
  double* d_c = scalebuf.p;
  double* d_cb1 = scalebuf.p + nb;
  LEM_CUDA_TRY(cudaMemcpyAsync(d_c, scales.data(), sizeof(double) * 2 * nb, cudaMemcpyHostToDevice, st));

  double bj[14];
  for (int j = 0; j < 14; ++j) bj[j] = kPadeInt[j] / kPadeInt[0];
  const dim3 gsq = grid1(nn, nb);
  auto lin = [&](double* out, std::initializer_list<std::pair<const double*, double>> terms,
                 double diag, const double* dscale, const double* wscale0) -> lem_status {
    Lin L{};
    L.nin = 0;
    for (auto& t : terms) { L.in[L.nin] = t.first; L.w[L.nin] = t.second; ++L.nin; }
    L.diag = diag; L.dscale = dscale; L.wscale0 = wscale0;
    lincomb_kernel<<<gsq, 256, 0, st>>>(out, n, n, n, L);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LEM_OK : cuda_fail(e, "lincomb_kernel");
  };
  TcGuard tc;
  tc.st = st;
  if (ctx->build_tc) LEM_TRY(tc_gemm_create(n, nb, gjcols, st, &tc.g));
  // C = A B + beta C for every class of the batch
  auto mm = [&](const double* A, const double* B, double* C, double beta) -> lem_status {
    if (tc.g) return tc_gemm(tc.g, n, nb, nullptr, A, B, beta != 0.0 ? C : nullptr, C, st);
    LEM_CUDA_TRY(dgemm_sq(n, nb, A, B, C, 1.0, beta, st));
    return LEM_OK;
  };
  // Xs = X / 2^s   (per class)
  LEM_TRY(lin(Xs, {{Xs, 1.0}}, 0.0, nullptr, d_c));
  LEM_TRY(mm(Xs, Xs, T2, 0.0));
  LEM_TRY(mm(T2, T2, T4, 0.0));
  LEM_TRY(mm(T4, T2, T6, 0.0));
  if (phi) {
    LEM_TRY(lin(B2, {{Xs, 1.0}}, 0.0, nullptr, d_c));  // Z^2 top-right = c Xs
    LEM_TRY(mm(T2, B2, B4, 0.0));
    LEM_TRY(mm(T4, B2, B6, 0.0));
  }
  // W1 = b13 Z6 + b11 Z4 + b9 Z2 ;  W3 = Z6 W1 + b7 Z6 + b5 Z4 + b3 Z2 + b1 I ; U = Z W3
  LEM_TRY(lin(TW, {{T6, bj[13]}, {T4, bj[11]}, {T2, bj[9]}}, 0.0, nullptr, nullptr));
  LEM_TRY(lin(T3, {{T6, bj[7]}, {T4, bj[5]}, {T2, bj[3]}}, bj[1], nullptr, nullptr));
  LEM_TRY(mm(T6, TW, T3, 1.0));
  LEM_TRY(mm(Xs, T3, UT, 0.0));
  if (phi) {
    LEM_TRY(lin(BW, {{B6, bj[13]}, {B4, bj[11]}, {B2, bj[9]}}, 0.0, nullptr, nullptr));
    LEM_TRY(lin(B3, {{B6, bj[7]}, {B4, bj[5]}, {B2, bj[3]}}, 0.0, nullptr, nullptr));
    LEM_TRY(mm(T6, BW, B3, 1.0));
    LEM_TRY(lin(UB, {}, 1.0, d_cb1, nullptr));  // c b1 I (from Z's top-right c I times b1)
    LEM_TRY(mm(Xs, B3, UB, 1.0));
  }
  // V = Z6 (b12 Z6 + b10 Z4 + b8 Z2) + b6 Z6 + b4 Z4 + b2 Z2 + b0 I
  LEM_TRY(lin(TW, {{T6, bj[12]}, {T4, bj[10]}, {T2, bj[8]}}, 0.0, nullptr, nullptr));
  LEM_TRY(lin(VT, {{T6, bj[6]}, {T4, bj[4]}, {T2, bj[2]}}, bj[0], nullptr, nullptr));
  LEM_TRY(mm(T6, TW, VT, 1.0));
  if (phi) {
    LEM_TRY(lin(BW, {{B6, bj[12]}, {B4, bj[10]}, {B2, bj[8]}}, 0.0, nullptr, nullptr));
    LEM_TRY(lin(VB, {{B6, bj[6]}, {B4, bj[4]}, {B2, bj[2]}}, 0.0, nullptr, nullptr));
    LEM_TRY(mm(T6, BW, VB, 1.0));
  }
  // G = [V_T - U_T | V_T + U_T | (V_B + U_B) - (V_B - U_B) = 2 U_B]
  {
    Lin L{};
    L.nin = 2; L.in[0] = VT; L.in[1] = UT; L.w[0] = 1.0; L.w[1] = -1.0;
    lincomb_kernel<<<gsq, 256, 0, st>>>(T2, n, n, n, L);  // T2 reused as scratch
    L.w[1] = 1.0;
    lincomb_kernel<<<gsq, 256, 0, st>>>(T4, n, n, n, L);
    LEM_CUDA_TRY(cudaGetLastError());
    copy_cols_kernel<<<gsq, 256, 0, st>>>(G, gjcols, 0, T2, n, 0, n, n);
    copy_cols_kernel<<<gsq, 256, 0, st>>>(G, gjcols, n, T4, n, 0, n, n);
    if (phi) {
      Lin L2{};
      L2.nin = 1; L2.in[0] = UB; L2.w[0] = 2.0;
      lincomb_kernel<<<gsq, 256, 0, st>>>(T6, n, n, n, L2);
      copy_cols_kernel<<<gsq, 256, 0, st>>>(G, gjcols, 2 * n, T6, n, 0, n, n);
    }
    LEM_CUDA_TRY(cudaGetLastError());
  }
  LEM_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
  Buf ybuf, pivbuf;  // freed after the final synchronisation
  LEM_TRY(solve_gj(ctx, tc.g, G, n, gjcols, nb, ybuf, pivbuf));
  LEM_CUDA_TRY(cudaGetLastError());
  // R_T -> RT2 (ping) ; R_B -> B2 (ping) ; squarings per class (s differs per class:
  // classes that need fewer squarings are squared by a masked update; simplest: square each
  // batch entry separately when the counts differ).
  copy_cols_kernel<<<gsq, 256, 0, st>>>(RT2, n, 0, G, gjcols, n, n, n);
  if (phi) copy_cols_kernel<<<gsq, 256, 0, st>>>(B2, n, 0, G, gjcols, 2 * n, n, n);
  LEM_CUDA_TRY(cudaGetLastError());
  double* RT = RT2; double* RTn = T4;
  double* RB = B2;  double* RBn = B4;
  bool uniform = true;
  for (int b = 0; b < nb; ++b) uniform = uniform && (s[b] == s[0]);
  Buf mapbuf;
  if (tc.g && !uniform) {
    // Classes sorted by s, descending: at squaring q the classes still squaring (s > q) are a
    // prefix of the order, so one index map serves every squaring.
    std::vector<int> order(nb);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return s[a] > s[b]; });
    LEM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&mapbuf.p), sizeof(int) * nb, st));
    const int* d_map = reinterpret_cast<const int*>(mapbuf.p);
    LEM_CUDA_TRY(cudaMemcpyAsync(mapbuf.p, order.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));
    for (int q = 0; q < smax; ++q) {
      int nact = 0;
      while (nact < nb && s[order[nact]] > q) ++nact;
      if (phi) LEM_TRY(tc_gemm(tc.g, n, nact, d_map, RT, RB, RB, RBn, st));  // R_T R_B + R_B
      LEM_TRY(tc_gemm(tc.g, n, nact, d_map, RT, RT, nullptr, RTn, st));
      std::swap(RT, RTn);
      if (phi) std::swap(RB, RBn);
    }
    // a class that stopped squaring an odd number of steps early holds its result in the
    // other buffer of the pair
    for (int b = 0; b < nb; ++b) {
      if ((smax - s[b]) % 2 == 0) continue;
      LEM_CUDA_TRY(cudaMemcpyAsync(RT + b * nn, RTn + b * nn, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
      if (phi)
        LEM_CUDA_TRY(cudaMemcpyAsync(RB + b * nn, RBn + b * nn, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
    }
  } else if (uniform) {
    for (int q = 0; q < s[0]; ++q) {
      if (phi) {  // (R_T, R_B)^2 = (R_T^2, R_T R_B + R_B)
        if (tc.g) {
          LEM_TRY(tc_gemm(tc.g, n, nb, nullptr, RT, RB, RB, RBn, st));
        } else {
          LEM_CUDA_TRY(cudaMemcpyAsync(RBn, RB, sizeof(double) * nn * nb, cudaMemcpyDeviceToDevice, st));
          LEM_TRY(mm(RT, RB, RBn, 1.0));
        }
        std::swap(RB, RBn);
      }
      LEM_TRY(mm(RT, RT, RTn, 0.0));
      std::swap(RT, RTn);
    }
  } else {
    for (int b = 0; b < nb; ++b) {
      double* rt = RT + b * nn; double* rtn = RTn + b * nn;
      double* rb = phi ? RB + b * nn : nullptr; double* rbn = phi ? RBn + b * nn : nullptr;
      for (int q = 0; q < s[b]; ++q) {
        if (phi) {
          LEM_CUDA_TRY(cudaMemcpyAsync(rbn, rb, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
          LEM_CUDA_TRY(dgemm_sq(n, 1, rt, rb, rbn, 1.0, 1.0, st));
          std::swap(rb, rbn);
        }
        LEM_CUDA_TRY(dgemm_sq(n, 1, rt, rt, rtn, 1.0, 0.0, st));
        std::swap(rt, rtn);
      }
      // move the result into the batch-uniform buffer position of RT/RB
      if (rt != RT + b * nn) LEM_CUDA_TRY(cudaMemcpyAsync(RT + b * nn, rt, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
      if (phi && rb != RB + b * nn) LEM_CUDA_TRY(cudaMemcpyAsync(RB + b * nn, rb, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
    }
  }
  const double* R = phi ? RB : RT;
  double* Pout = ctx->d_P + size_t(c0) * ctx->n_int * ctx->n_loc;
  if (ctx->cplx)
    extract_rows_complex_kernel<<<grid1(ctx->n_int * ctx->n_loc, nb), 256, 0, st>>>(Pout, ctx->n_int, ctx->n_loc, R,
                                                                                    n, d_bc);
  else
    extract_rows_kernel<<<grid1(ctx->n_int * ctx->n_loc, nb), 256, 0, st>>>(
        Pout, ctx->n_int, ctx->n_loc, R, n, n, 0, d_bc);
  LEM_CUDA_TRY(cudaGetLastError());
  int status = 0;
  LEM_CUDA_TRY(cudaMemcpyAsync(&status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  LEM_CUDA_TRY(cudaStreamSynchronize(st));
  // scratch is released by the Buf destructors (stream-ordered frees are unnecessary
  // after the synchronisation above)
  if (status != 0) return fail(LEM_ENUMERIC, "singular Pade denominator (V - U) in the propagator build");
  if (tc.g) LEM_TRY(tc_gemm_check(tc.g, st));
  return LEM_OK;
}

// ---------------------------------------------------------------- phi_1 and phi_3 together
// For the third-order Rosenbrock step each class needs phi_1(X) and phi_3(X). Both are blocks
// of exp(Z), Z = [[X, I, 0, 0], [0, 0, I, 0], [0, 0, 0, I], [0, 0, 0, 0]] (top block row:
// e^X, phi_1, phi_2, phi_3). Every polynomial in Z, and its inverse, has the form
//   [[T, B0, B1, B2], [0, b0 I, b1 I, b2 I], [0, 0, b0 I, b1 I], [0, 0, 0, b0 I]]
// (an "augmented" element: T and B_j n x n, b a scalar upper-triangular Toeplitz part), with
//   (A C).T = A.T C.T,  (A C).B_j = A.T C.B_j + sum_{a <= j} c.b_{j-a} A.B_a,  b = a.b * c.b.
// The scaling is moved onto the functions: with Xs = X / 2^s, the Pade-13 approximant runs on
// Z(Xs) (unit identity blocks, so every weight and the Toeplitz parts are the same for every
// class), and s doublings 2^k phi_k(2Y) = e^Y phi_k(Y) + sum_{j=1..k} phi_j(Y) / (k - j)!
// bring phi_k(Xs) back to phi_k(X). s follows the same rule as the phi_1 build (the 1-norm of
// the augmented matrix is max(|X|_1, 1)).
struct Aug {
  double* m[4];  // T, B0, B1, B2
  double b[3];   // Toeplitz part (class independent)
};

static lem_status build_batch_phi3(lem_ctx* ctx, int c0, int nb, const double* d_state) {
  cudaStream_t st = ctx->stream;
  const int n = int(ctx->n_loc);
  const int64_t nn = int64_t(n) * n;
  std::vector<BatchClass> hbc(nb);
  for (int b = 0; b < nb; ++b) {
    const ClassDesc& c = ctx->classes[c0 + b];
    hbc[b].rep = ctx->tiles[c.rep_tile];
    hbc[b].whole[0] = c.whole[0];
    hbc[b].whole[1] = c.whole[1];
  }
  constexpr int NAUG = 10;  // Z, Z2, Z4, Z6, W, W3, U, V, R, Rn
  const int gjcols = 5 * n;
  Buf scratch, bcbuf, normbuf, scalebuf, ybuf, pivbuf, mapbuf;
  const size_t bytes = sizeof(double) * (size_t(NAUG) * 4 * nn + size_t(n) * gjcols) * nb;
  LEM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&scratch.p), bytes, st));
  LEM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&bcbuf.p), sizeof(BatchClass) * nb, st));
  LEM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&normbuf.p), sizeof(double) * nb, st));
  LEM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&scalebuf.p), sizeof(double) * nb, st));
  BatchClass* d_bc = reinterpret_cast<BatchClass*>(bcbuf.p);
  LEM_CUDA_TRY(cudaMemcpyAsync(d_bc, hbc.data(), sizeof(BatchClass) * nb, cudaMemcpyHostToDevice, st));
  double* S = scratch.p;
  auto aug = [&](int i) {
    Aug a;
    for (int q = 0; q < 4; ++q) a.m[q] = S + (size_t(i) * 4 + q) * nn * nb;
    a.b[0] = a.b[1] = a.b[2] = 0.0;
    return a;
  };
  Aug Z = aug(0), Z2 = aug(1), Z4 = aug(2), Z6 = aug(3), W = aug(4), W3 = aug(5), U = aug(6), V = aug(7),
      R = aug(8), Rn = aug(9);
  double* G = S + size_t(NAUG) * 4 * nn * nb;

  // X = dt J_M, the 1-norms, s per class
  const double* u = ctx->desc.reaction ? d_state : nullptr;
  assemble_local_kernel<<<dim3((n + 127) / 128, nb), 128, 0, st>>>(
      Z.m[0], n, d_bc, nb, ctx->d_coef, ctx->desc.coef_stride, ctx->ny, ctx->nx, ctx->desc.ndim, u, ctx->desc.dt,
      ctx->desc.reaction, ctx->desc.porous_m);
  LEM_CUDA_TRY(cudaMemsetAsync(normbuf.p, 0, sizeof(double) * nb, st));
  norm1_kernel<<<dim3((n + 127) / 128, nb), 128, 0, st>>>(Z.m[0], n,
                                                           reinterpret_cast<unsigned long long*>(normbuf.p));
  LEM_CUDA_TRY(cudaGetLastError());
  std::vector<double> norms(nb), scales(nb);
  LEM_CUDA_TRY(cudaMemcpyAsync(norms.data(), normbuf.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
  LEM_CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<int> s(nb);
  int smax = 0;
  for (int b = 0; b < nb; ++b) {
    const double nz = std::max(norms[b], 1.0);
    int sb = 0;
    while (nz > kTheta13 * std::ldexp(1.0, sb)) ++sb;
    s[b] = sb;
    smax = std::max(smax, sb);
    ctx->squarings[c0 + b] = sb;
    scales[b] = std::ldexp(1.0, -sb);
  }
  LEM_CUDA_TRY(cudaMemcpyAsync(scalebuf.p, scales.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, st));

  const dim3 gsq = grid1(nn, nb);
  auto lin = [&](double* out, std::initializer_list<std::pair<const double*, double>> terms, double diag,
                 const double* wscale0) -> lem_status {
    Lin L{};
    L.nin = 0;
    for (auto& t : terms) {
      if (t.second == 0.0) continue;  // never read a buffer that is not needed (it may be unset)
      L.in[L.nin] = t.first;
      L.w[L.nin] = t.second;
      ++L.nin;
    }
    L.diag = diag;
    L.dscale = nullptr;
    L.wscale0 = wscale0;
    lincomb_kernel<<<gsq, 256, 0, st>>>(out, n, n, n, L);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LEM_OK : cuda_fail(e, "lincomb_kernel");
  };
  TcGuard tc;
  tc.st = st;
  if (ctx->build_tc) LEM_TRY(tc_gemm_create(n, nb, gjcols, st, &tc.g));
  auto mm = [&](const double* A, const double* B, double* C, const double* D) -> lem_status {
    if (tc.g) return tc_gemm(tc.g, n, nb, nullptr, A, B, D, C, st);
    if (D && D != C) LEM_CUDA_TRY(cudaMemcpyAsync(C, D, sizeof(double) * nn * nb, cudaMemcpyDeviceToDevice, st));
    LEM_CUDA_TRY(dgemm_sq(n, nb, A, B, C, 1.0, D ? 1.0 : 0.0, st));
    return LEM_OK;
  };
  // C = A * B (C distinct from A and B)
  auto amul = [&](const Aug& A, const Aug& B, Aug& C) -> lem_status {
    LEM_TRY(mm(A.m[0], B.m[0], C.m[0], nullptr));
    for (int j = 0; j < 3; ++j) {
      LEM_TRY(mm(A.m[0], B.m[1 + j], C.m[1 + j], nullptr));
      const double w0 = B.b[j], w1 = j >= 1 ? B.b[j - 1] : 0.0, w2 = j >= 2 ? B.b[j - 2] : 0.0;
      if (w0 != 0.0 || w1 != 0.0 || w2 != 0.0)  // + sum_{a <= j} B.b[j - a] A.B_a
        LEM_TRY(lin(C.m[1 + j], {{C.m[1 + j], 1.0}, {A.m[1], w0}, {A.m[2], w1}, {A.m[3], w2}}, 0.0, nullptr));
    }
    for (int j = 0; j < 3; ++j) {
      double v = 0.0;
      for (int a = 0; a <= j; ++a) v += A.b[a] * B.b[j - a];
      C.b[j] = v;
    }
    return LEM_OK;
  };
  // C = sum w_i A_i + d I (C may be one of the A_i)
  auto alin = [&](Aug& C, std::initializer_list<std::pair<const Aug*, double>> terms, double d) -> lem_status {
    double nb3[3] = {d, 0.0, 0.0};
    for (int q = 0; q < 4; ++q) {
      Lin L{};
      L.nin = 0;
      for (auto& t : terms) {
        L.in[L.nin] = t.first->m[q];
        L.w[L.nin] = t.second;
        ++L.nin;
      }
      L.diag = q == 0 ? d : 0.0;
      lincomb_kernel<<<gsq, 256, 0, st>>>(C.m[q], n, n, n, L);
    }
    LEM_CUDA_TRY(cudaGetLastError());
    for (auto& t : terms)
      for (int j = 0; j < 3; ++j) nb3[j] += t.second * t.first->b[j];
    for (int j = 0; j < 3; ++j) C.b[j] = nb3[j];
    return LEM_OK;
  };

  // Z(Xs): T = X / 2^s, B = (I, 0, 0), Toeplitz part N (b = (0, 1, 0))
  LEM_TRY(lin(Z.m[0], {{Z.m[0], 1.0}}, 0.0, scalebuf.p));
  LEM_TRY(lin(Z.m[1], {}, 1.0, nullptr));
  LEM_CUDA_TRY(cudaMemsetAsync(Z.m[2], 0, sizeof(double) * nn * nb, st));
  LEM_CUDA_TRY(cudaMemsetAsync(Z.m[3], 0, sizeof(double) * nn * nb, st));
  Z.b[0] = 0.0; Z.b[1] = 1.0; Z.b[2] = 0.0;
  double bj[14];
  for (int j = 0; j < 14; ++j) bj[j] = kPadeInt[j] / kPadeInt[0];
  LEM_TRY(amul(Z, Z, Z2));
  LEM_TRY(amul(Z2, Z2, Z4));
  LEM_TRY(amul(Z4, Z2, Z6));
  // U = Z (Z6 (b13 Z6 + b11 Z4 + b9 Z2) + b7 Z6 + b5 Z4 + b3 Z2 + b1 I)
  LEM_TRY(alin(W, {{&Z6, bj[13]}, {&Z4, bj[11]}, {&Z2, bj[9]}}, 0.0));
  LEM_TRY(amul(Z6, W, W3));
  LEM_TRY(alin(W3, {{&W3, 1.0}, {&Z6, bj[7]}, {&Z4, bj[5]}, {&Z2, bj[3]}}, bj[1]));
  LEM_TRY(amul(Z, W3, U));
  // V = Z6 (b12 Z6 + b10 Z4 + b8 Z2) + b6 Z6 + b4 Z4 + b2 Z2 + b0 I
  LEM_TRY(alin(W, {{&Z6, bj[12]}, {&Z4, bj[10]}, {&Z2, bj[8]}}, 0.0));
  LEM_TRY(amul(Z6, W, V));
  LEM_TRY(alin(V, {{&V, 1.0}, {&Z6, bj[6]}, {&Z4, bj[4]}, {&Z2, bj[2]}}, bj[0]));
  // R = (V - U)^{-1} (V + U). With M = V - U = [[Ma, Mc], [0, Md]] and P = V + U likewise:
  // R.T = Ma^{-1} Pa, R.B = Ma^{-1} (Pc - Mc g), g = Md^{-1} Pd (a Toeplitz solve).
  LEM_TRY(alin(W, {{&V, 1.0}, {&U, -1.0}}, 0.0));   // M
  LEM_TRY(alin(W3, {{&V, 1.0}, {&U, 1.0}}, 0.0));   // P
  double g[3];
  g[0] = W3.b[0] / W.b[0];
  g[1] = (W3.b[1] - W.b[1] * g[0]) / W.b[0];
  g[2] = (W3.b[2] - W.b[1] * g[1] - W.b[2] * g[0]) / W.b[0];
  for (int j = 0; j < 3; ++j) {  // Pc_j - sum_{a <= j} Mc_a g_{j-a}
    const double w0 = g[j], w1 = j >= 1 ? g[j - 1] : 0.0, w2 = j >= 2 ? g[j - 2] : 0.0;
    LEM_TRY(lin(W3.m[1 + j], {{W3.m[1 + j], 1.0}, {W.m[1], -w0}, {W.m[2], -w1}, {W.m[3], -w2}}, 0.0, nullptr));
  }
  copy_cols_kernel<<<gsq, 256, 0, st>>>(G, gjcols, 0, W.m[0], n, 0, n, n);
  for (int q = 0; q < 4; ++q) copy_cols_kernel<<<gsq, 256, 0, st>>>(G, gjcols, (1 + q) * n, W3.m[q], n, 0, n, n);
  LEM_CUDA_TRY(cudaGetLastError());
  LEM_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
  LEM_TRY(solve_gj(ctx, tc.g, G, n, gjcols, nb, ybuf, pivbuf));
  for (int q = 0; q < 4; ++q) copy_cols_kernel<<<gsq, 256, 0, st>>>(R.m[q], n, 0, G, gjcols, (1 + q) * n, n, n);
  LEM_CUDA_TRY(cudaGetLastError());

  // s doublings of (E, phi_1, phi_2, phi_3) per class. The scaled copies H_k = phi_k / 2^k and
  // the addends D_k go to free scratch first, then phi_k' = E H_k + D_k and E' = E E.
  double* H1 = Z2.m[0]; double* H2 = Z2.m[1]; double* H3 = Z2.m[2];
  double* D2 = Z4.m[0]; double* D3 = Z4.m[1];
  auto prep = [&](const Aug& X) -> lem_status {  // on every class (harmless for finished ones)
    LEM_TRY(lin(H1, {{X.m[1], 0.5}}, 0.0, nullptr));
    LEM_TRY(lin(H2, {{X.m[2], 0.25}}, 0.0, nullptr));
    LEM_TRY(lin(H3, {{X.m[3], 0.125}}, 0.0, nullptr));
    LEM_TRY(lin(D2, {{X.m[1], 0.25}, {X.m[2], 0.25}}, 0.0, nullptr));
    LEM_TRY(lin(D3, {{X.m[1], 0.0625}, {X.m[2], 0.125}, {X.m[3], 0.125}}, 0.0, nullptr));
    return LEM_OK;
  };
  std::vector<int> order(nb);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return s[a] > s[b]; });
  const bool uniform = s[order.front()] == s[order.back()];
  if (tc.g) {
    const int* d_map = nullptr;
    if (!uniform) {
      LEM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&mapbuf.p), sizeof(int) * nb, st));
      LEM_CUDA_TRY(cudaMemcpyAsync(mapbuf.p, order.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));
      d_map = reinterpret_cast<const int*>(mapbuf.p);
    }
    for (int q = 0; q < smax; ++q) {
      int nact = 0;
      while (nact < nb && s[order[nact]] > q) ++nact;
      LEM_TRY(prep(R));
      LEM_TRY(tc_gemm(tc.g, n, nact, d_map, R.m[0], H1, H1, Rn.m[1], st));
      LEM_TRY(tc_gemm(tc.g, n, nact, d_map, R.m[0], H2, D2, Rn.m[2], st));
      LEM_TRY(tc_gemm(tc.g, n, nact, d_map, R.m[0], H3, D3, Rn.m[3], st));
      LEM_TRY(tc_gemm(tc.g, n, nact, d_map, R.m[0], R.m[0], nullptr, Rn.m[0], st));
      std::swap(R, Rn);
    }
    for (int b = 0; b < nb; ++b) {  // classes that stopped an odd number of steps early
      if ((smax - s[b]) % 2 == 0) continue;
      for (int q = 0; q < 4; ++q)
        LEM_CUDA_TRY(cudaMemcpyAsync(R.m[q] + b * nn, Rn.m[q] + b * nn, sizeof(double) * nn,
                                     cudaMemcpyDeviceToDevice, st));
    }
  } else {
    for (int q = 0; q < smax; ++q) {
      LEM_TRY(prep(R));
      for (int b = 0; b < nb; ++b) {
        if (s[b] <= q) {  // finished: carry it into the other buffer
          for (int k = 0; k < 4; ++k)
            LEM_CUDA_TRY(cudaMemcpyAsync(Rn.m[k] + b * nn, R.m[k] + b * nn, sizeof(double) * nn,
                                         cudaMemcpyDeviceToDevice, st));
          continue;
        }
        const int64_t o = b * nn;
        LEM_CUDA_TRY(cudaMemcpyAsync(Rn.m[1] + o, H1 + o, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
        LEM_CUDA_TRY(cudaMemcpyAsync(Rn.m[2] + o, D2 + o, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
        LEM_CUDA_TRY(cudaMemcpyAsync(Rn.m[3] + o, D3 + o, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
        LEM_CUDA_TRY(dgemm_sq(n, 1, R.m[0] + o, H1 + o, Rn.m[1] + o, 1.0, 1.0, st));
        LEM_CUDA_TRY(dgemm_sq(n, 1, R.m[0] + o, H2 + o, Rn.m[2] + o, 1.0, 1.0, st));
        LEM_CUDA_TRY(dgemm_sq(n, 1, R.m[0] + o, H3 + o, Rn.m[3] + o, 1.0, 1.0, st));
        LEM_CUDA_TRY(dgemm_sq(n, 1, R.m[0] + o, R.m[0] + o, Rn.m[0] + o, 1.0, 0.0, st));
      }
      std::swap(R, Rn);
    }
  }
  const size_t pc = size_t(ctx->n_int) * ctx->n_loc;
  extract_rows_kernel<<<grid1(ctx->n_int * ctx->n_loc, nb), 256, 0, st>>>(ctx->d_P + size_t(c0) * pc, ctx->n_int,
                                                                         ctx->n_loc, R.m[1], n, n, 0, d_bc);
  extract_rows_kernel<<<grid1(ctx->n_int * ctx->n_loc, nb), 256, 0, st>>>(ctx->d_P3 + size_t(c0) * pc, ctx->n_int,
                                                                         ctx->n_loc, R.m[3], n, n, 0, d_bc);
  LEM_CUDA_TRY(cudaGetLastError());
  int status = 0;
  LEM_CUDA_TRY(cudaMemcpyAsync(&status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  LEM_CUDA_TRY(cudaStreamSynchronize(st));
  if (status != 0) return fail(LEM_ENUMERIC, "singular Pade denominator (V - U) in the propagator build");
  if (tc.g) LEM_TRY(tc_gemm_check(tc.g, st));
  return LEM_OK;
}

lem_status build_propagators_impl(lem_ctx* ctx, const double* d_state);

lem_status build_propagators(lem_ctx* ctx, const double* d_state) {
  nvtxRangePushA("lem_build_propagators");
  const lem_status st = build_propagators_impl(ctx, d_state);
  nvtxRangePop();
  return st;
}

lem_status build_propagators_impl(lem_ctx* ctx, const double* d_state) {
  if (ctx->desc.reaction && !d_state) return fail(LEM_EINVAL, "the reaction Jacobian needs the state");
  const int64_t nc = int64_t(ctx->classes.size());
  const int64_t n = ctx->n_loc;
  const bool rb3 = ctx->desc.scheme == LEM_SCHEME_RB3;
  const int nmat = rb3 ? 45 : ctx->desc.mode == LEM_MODE_PHI ? 19 : 11;
  // batch size from a scratch budget of 8 GiB
  const int gjc = rb3 ? 5 * int(n) : ctx->desc.mode == LEM_MODE_PHI ? 3 * int(n) : 2 * int(n);
  const double per = double(nmat) * n * n * sizeof(double) +
                     (ctx->build_tc ? double(tc_gemm_bytes(int(n), 1, gjc)) + sizeof(double) * n * GJ_KB : 0.0);
  int64_t bmax = std::max<int64_t>(1, int64_t((8.0 * (1ull << 30)) / per));
  bmax = std::min<int64_t>(bmax, 65535);
  for (int64_t c0 = 0; c0 < nc; c0 += bmax) {
    int nb = int(std::min<int64_t>(bmax, nc - c0));
    LEM_TRY(rb3 ? build_batch_phi3(ctx, int(c0), nb, d_state) : build_batch(ctx, int(c0), nb, d_state));
  }
  // the third-order Rosenbrock step evaluates its defect with the Jacobian's state
  if (rb3 && ctx->desc.reaction)
    LEM_CUDA_TRY(cudaMemcpyAsync(ctx->d_um, d_state, sizeof(double) * ctx->npts, cudaMemcpyDeviceToDevice,
                                 ctx->stream));
  ctx->built = true;
  ctx->build_gen++;
  ctx->steps_since_build = 0;
  return LEM_OK;
}

}  // namespace lem
