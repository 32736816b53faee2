// Internal declarations shared by the liblem translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lem.h"

namespace lem {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
lem_status fail(lem_status s, const std::string& msg);
lem_status cuda_fail(cudaError_t e, const char* what);
// makes `dev` current for a scope and restores the caller's device
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

#define LEM_CUDA_TRY(call)                                 \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return ::lem::cuda_fail(e_, #call); \
  } while (0)

#define LEM_TRY(call)                   \
  do {                                  \
    lem_status s_ = (call);             \
    if (s_ != LEM_OK) return s_;        \
  } while (0)

// ---------------------------------------------------------------- plan
// One owner tile D_i and its window M_i (Sec. 3). Window node (a, b) is mesh node
// ((org[0] + a) mod ny, (org[1] + b) mod nx); 1D problems use axis 1 only (ny = 1).
struct TileDesc {
  int32_t org[2];   // window origin (may be negative on a periodic axis)
  int32_t wext[2];  // window extent per axis
  int32_t iofs[2];  // owner-tile offset inside the window
  int32_t iext[2];  // owner-tile extent per axis
  int32_t t0[2];    // first owner node per axis (mesh coordinates)
  int32_t cls;      // propagator class
  int32_t pad;
};

// One distinct local operator: windows with identical local matrices share it.
struct ClassDesc {
  int32_t rep_tile;  // a tile of this class (its window defines the local matrix)
  int32_t ntiles;
  int32_t wext[2];
  int32_t iext[2];
  int32_t iofs[2];
  int32_t whole[2];  // window covers a whole periodic axis (wrap couplings inside)
};

// Device-side stencil: per node (stride 1) or constant (stride 0), dt-scaled.
struct Stencil {
  const double* c[5];  // C, W, E, S, N
  int64_t stride;
};

struct SplitPlan;  // tcgen05 split-precision state (step_split.cu)
struct BandPlan;   // truncated propagators (step_band.cu)

}  // namespace lem

struct lem_ctx {
  lem_problem_desc desc;
  int device = 0;
  cudaStream_t stream = nullptr;
  int64_t ny = 1, nx = 1, npts = 0;
  int bcy = LEM_BC_DIRICHLET0, bcx = LEM_BC_DIRICHLET0;
  // plan
  std::vector<lem::TileDesc> tiles;
  std::vector<lem::ClassDesc> classes;
  std::vector<int32_t> class_order;    // tiles sorted by class
  std::vector<int32_t> class_offset;   // start of each class in class_order (nclasses+1)
  std::vector<double> h_coef;          // dt-scaled constant stencil (C, W, E, S, N); empty if per node
  std::vector<int> squarings;          // per class, after the build
  int64_t n_loc = 0, n_int = 0;        // padded window / tile sizes
  bool built = false;
  bool build_tc = false;               // propagator products on the tensor cores (split tiers)
  int cplx = 0;                        // complex problem: interleaved states, n_loc / n_int are the
                                       // real-embedding sizes (2 x window / tile nodes)
  int build_gen = 0;                   // incremented by every propagator build
  int steps_since_build = 0;
  // device buffers (owned)
  double* d_coef = nullptr;            // 5 * (stride ? npts : 1), dt-scaled
  lem::TileDesc* d_tiles = nullptr;
  int32_t* d_class_order = nullptr;
  double* d_P = nullptr;               // nclasses * n_int * n_loc
  double* d_P3 = nullptr;              // third-order Rosenbrock: the phi_3 propagators, same layout
  float* d_P3_32 = nullptr;            // FP32 copy of d_P3 for the reduced-precision GEMV
  double* d_um = nullptr;              // third-order Rosenbrock: the state of the last Jacobian
  double* d_u0 = nullptr;              // third-order Rosenbrock: u^n kept across the two stages
  float* d_P32 = nullptr;              // FP32 copy for the reduced-precision GEMV
  int p32_gen = -1;                    // build_gen the FP32 copy was made from
  int apply_path = 0;                  // lem_apply_path: how lem_step applies the propagators
  double* d_r = nullptr;               // npts (residual)
  double* d_U = nullptr;               // ntiles * n_loc (gathered windows)
  double* d_Y = nullptr;               // ntiles * n_int (local results)
  double* d_state_tmp = nullptr;       // npts (host-state path)
  int* d_status = nullptr;             // device error word
  int64_t device_bytes = 0;
  lem::SplitPlan* split = nullptr;
  // truncated propagators (lem_set_truncation): off while band_tol < 0
  double band_tol = -1.0;
  int band_gen = -1;                   // build_gen the packed boxes were made from
  int apply_path_dense = 0;            // the apply path lem_create chose, restored when off
  lem::BandPlan* band = nullptr;
  // optional event timing of the apply kernel
  bool timing = false;
  int timing_period = 1;               // bracket every timing_period-th apply launch
  int64_t timing_count = 0;
  std::vector<cudaEvent_t> ev_pool;    // pairs (start, stop)
  size_t ev_used = 0;
  cudaError_t timing_begin(cudaEvent_t* stop);
  void timing_end(cudaEvent_t stop);
  lem::Stencil stencil() const;
};

namespace lem {
// plan.cpp
lem_status validate(const lem_problem_desc* d);
lem_status make_plan(lem_ctx* ctx);
// builder.cu
lem_status build_propagators(lem_ctx* ctx, const double* d_state);
// step_fp64.cu
lem_status step_fp64(lem_ctx* ctx, double* d_u);
// step_fp64.cu: dt F(u) (or its complex / porous variants) into r on the context stream
cudaError_t launch_residual_fp64(const lem_ctx* ctx, double* r, const double* u);
// step_gemv.cu
lem_status step_gemv(lem_ctx* ctx, double* d_u, bool f32);
// blocks per tile of a batched GEMV launch with `threads` threads per block
int gemv_row_split(const lem_ctx* ctx, int threads);
// step_band.cu: truncated propagators (extents from ctx->band_tol, packed boxes, apply)
lem_status band_prepare(lem_ctx* ctx);
lem_status band_step(lem_ctx* ctx, double* d_u);
lem_status band_get(lem_ctx* ctx, int64_t cls, int32_t* ext, int64_t* row_values);
int64_t band_values(const lem_ctx* ctx);
void band_destroy(lem_ctx* ctx);
// nsteps of a small linear problem in one cooperative launch; *done false: not eligible
lem_status step_gemv_multi(lem_ctx* ctx, double* d_u, int nsteps, bool f32, bool* done);
lem_status gemv_set_smem(lem_ctx* ctx);
// step_split.cu
lem_status split_prepare(lem_ctx* ctx);
// nsteps split steps of the FP64 state d_u. fuse_io: the first kernel of the run (the measuring
// residual pass) reads d_u itself (a state in device memory); otherwise a separate streaming
// conversion does (a state in mapped host memory, read once over the link). A streaming
// conversion writes the result back either way.
lem_status split_step(lem_ctx* ctx, double* d_u, int nsteps, bool fuse_io);
// the steps of split_step on a resident float-float state, with the residual scale carried
// across calls through d_carry (one unsigned on the device; carry_in: it holds the previous
// step's max|r|), and the conversions split_step does around them. in64 (with carry_in false):
// the measuring pass reads the FP64 state there and writes (uh, ul) from it.
lem_status split_run(lem_ctx* ctx, float* uh, float* ul, int nsteps, unsigned* d_carry, bool carry_in,
                     const double* in64 = nullptr);
lem_status split_to_ff(lem_ctx* ctx, const double* d_u, float* uh, float* ul);
lem_status split_from_ff(lem_ctx* ctx, const float* uh, const float* ul, double* d_u);
void split_destroy(lem_ctx* ctx);
lem_status split_check_error(lem_ctx* ctx);
bool split_eligible(const lem_ctx* ctx);
lem_status encode_f16_map(CUtensorMap* m, void* base, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
                          const cuuint32_t* box, const char* what, int swizzle_bytes = 128);
// multi-problem split steps (one residual and one GEMM launch per step for a whole batch)
struct SplitBatch;
bool split_batch_eligible(lem_ctx* const* ctxs, int n);
// cap: widest window block per problem (0: each context's own width; else the cheapest power of
// two in [16, cap] per problem)
lem_status split_batch_prepare(lem_ctx* const* ctxs, double* const* d_states, int n, int cap, SplitBatch** out);
double split_batch_executed_flops(const SplitBatch* b);
lem_status split_batch_step(SplitBatch* b, int nsteps, cudaStream_t st, cudaEvent_t* ev = nullptr);
double split_batch_gemm_flops(const SplitBatch* b, lem_ctx* const* ctxs);
lem_status split_batch_check_error(SplitBatch* b);
void split_batch_destroy(SplitBatch* b);
// builder_tc.cu: FP64 products of the propagator build as exact sums of FP16 slice products
// on the tensor cores (split-precision tiers)
struct TcGemm;
// workspace for products of nb matrices of n x n and rank-64 updates of n x gjcols ones
size_t tc_gemm_bytes(int n, int nb, int gjcols);
lem_status tc_gemm_create(int n, int nb, int gjcols, cudaStream_t st, TcGemm** out);
void tc_gemm_destroy(TcGemm* g, cudaStream_t st);
// C = A B + D (D optional) on strided batches of row-major FP64 matrices (A M x K, B K x N)
lem_status tc_gemm_ex(TcGemm* g, int nbatch, const int* map, int M, int N, int K, const double* A, int64_t lda,
                      int64_t sA, const double* B, int64_t ldb, int64_t sB, const double* D, int64_t ldd,
                      int64_t sD, int zr0, int zr1, double* C, int64_t ldc, int64_t sC, cudaStream_t st);
// the same for square n x n matrices stored back to back
lem_status tc_gemm(TcGemm* g, int n, int nbatch, const int* map, const double* A, const double* B, const double* D,
                   double* C, cudaStream_t st);
lem_status tc_gemm_check(TcGemm* g, cudaStream_t st);
// builder.cu: whether propagators of a precision tier are built with the tensor-core products
bool builder_uses_tc(int prec);
// abi.cpp: take a built single-class propagator from a context with the same local operator
lem_status adopt_propagators(lem_ctx* dst, lem_ctx* src, cudaEvent_t built);
// allocation helper that tracks bytes
lem_status dev_alloc(lem_ctx* ctx, void** p, size_t bytes);
}  // namespace lem
