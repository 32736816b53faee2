/*
 * lem.h -- C ABI of the GB300 (sm_103a) Local Exponential Method library (liblem.so).
 *
 * The Local Exponential Method (L. Bonaventura, "Local Exponential Methods: a domain
 * decomposition approach to exponential time integration of PDEs", arXiv 1505.02248)
 * replaces the global exponential step of a semi-discrete linear (or linearised) PDE
 *     du/dt = A u + g                                  (Sec. 2, Eq. spacedisc)
 * by independent local problems on overlapping windows M_i = D_i U B_i (Sec. 3):
 *     v^{n+1}_{M_i} = v^n_{M_i} + dt phi_1(dt A_{M_i}) (A_{M_i} v^n_{M_i} + g_{M_i}(t^n))
 *                                                      (Sec. 3, Eq. lem)
 * after which only the owner rows D_i are written back (Sec. 3, step 3).
 *
 * Conventions used by every entry point
 * -------------------------------------
 * - Meshes are 1D (n[0] = N) or 2D (n[0] = ny rows, n[1] = nx columns); states are
 *   contiguous row-major [y][x] arrays of double, one value per interior mesh node
 *   (complex problems: one interleaved (re, im) pair of doubles per node).
 * - The operator A is a 3-point (1D) or 5-point (2D) stencil given by its entries in
 *   the order C (diagonal), W (x-1), E (x+1), S (y-1), N (y+1); NOT multiplied by dt.
 *   Homogeneous Dirichlet walls drop the outside neighbour (g = 0); periodic axes wrap.
 * - Tiles D_i are tile[a] nodes per axis (the last tile of an axis may be ragged);
 *   windows add overlap[a] nodes per side, clipped at Dirichlet walls, wrapped on
 *   periodic axes (a periodic window that would reach around the axis is the whole axis).
 * - LEM_MODE_PHI uses the neighbour values frozen at t^n as the artificial-boundary data
 *   (the literal Eq. lem); LEM_MODE_EXP uses zero data: u_D <- R_D exp(dt A_M) u_M.
 * - All windows read u^n (Jacobi update); every node is written by its owner tile only.
 * - Device pointers are CUDA device addresses on the context's device; host pointers are
 *   ordinary CPU memory. The caller owns every buffer it passes; the library copies what
 *   it keeps (coefficients) and owns its propagators and workspaces.
 * - Errors: every call returns a lem_status; nothing is thrown across the ABI.
 *   lem_last_error() returns a thread-local message for the last failure.
 *   A context is not re-entrant: calls on one context must not overlap.
 * - Entry points that implement a passage of the paper cite it. The rest have no counterpart
 *   there and say what they serve: status and error strings, plan queries, propagator
 *   checkpoints, timing, synchronisation, batching and serving.
 */
#ifndef LEM_H
#define LEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LEM_OK = 0,
  LEM_EINVAL = 1,     /* invalid argument or descriptor */
  LEM_ENOMEM = 2,     /* device or host allocation failed (or was refused by a budget) */
  LEM_ECUDA = 3,      /* a CUDA runtime/driver call failed; see lem_last_error() */
  LEM_EBUSY = 4,      /* resource in use (server queue full) */
  LEM_ENOTREADY = 5,  /* propagators not built / result not ready */
  LEM_ETIMEOUT = 6,   /* a bounded wait expired */
  LEM_ENUMERIC = 7    /* singular Pade denominator or non-finite values */
} lem_status;

typedef enum { LEM_BC_DIRICHLET0 = 0, LEM_BC_PERIODIC = 1 } lem_bc;
typedef enum { LEM_MODE_PHI = 0, LEM_MODE_EXP = 1 } lem_mode;
/* LEM_PREC_FP64: propagators, residual and apply in IEEE binary64.
 * Propagators of the split tiers are built with tensor-core products (every Pade product,
 * squaring and elimination update an exact sum of FP16 slice products, about 2^-45 of the
 * operands' scale; the environment variable LEM_BUILD_PRODUCTS=fp64 forces FP64 products).
 * LEM_PREC_SPLIT: propagators applied in reduced precision within
 * 1e-6 relative L2 of the FP64 result after 100 steps, also for fields that decay by orders
 * of magnitude over the run. When every window shares one propagator (2D periodic, constant
 * coefficients, no reaction, tiles dividing the mesh, tile_x a multiple of 8, window width
 * tile_x + 2 overlap_x <= 64) it runs on the tcgen05 tensor cores: P = P_int + P2 + P3 with
 * one scale per row, r = r_int + r2 + r3 with one scale per step (FP16 pieces), the
 * P_int r_int product exact in FP32, five correction products, float-float state and
 * residual. Otherwise it runs the FP64 path.
 * LEM_PREC_SPLIT_FAST: two pieces of each operand (four products) on the tensor path, FP32
 * propagators with float-float accumulation in a batched GEMV otherwise (PHI mode). Each
 * step's increment carries a relative error near 2^-21 of sum_k |P_ik| |r_k|: within 1e-6
 * after 100 steps on fields that stay smooth (measured 1e-7 on 2048^2 advection-diffusion),
 * not on rough fields that decay fast. EXP mode with a split tier on a problem without a
 * shared propagator runs the FP64 path. lem_get_info reports the path taken. */
typedef enum { LEM_PREC_FP64 = 0, LEM_PREC_SPLIT = 1, LEM_PREC_SPLIT_FAST = 2 } lem_prec;

/* LEM_SCHEME_EULER: one window-local phi_1 stage per step (Eq. lem; with the reaction the
 * exponential Euler-Rosenbrock step of Sec. 4).
 * LEM_SCHEME_RB3: the third-order exponential Rosenbrock step exprb32 (Sec. 4.2 uses a
 * third-order exponential Rosenbrock method; Hochbruck, Ostermann and Schweitzer 2009):
 *   U = u + phi_1(dt J_m) dt F(u),  u' = U + 2 phi_3(dt J_m) dt (G(U) - G(u)),  G = F - J_m,
 * both stages window by window with per-class phi_1 and phi_3 propagators built together
 * (J_m: the Jacobian at the last refresh). PHI mode only; runs on the batched GEMV (FP64
 * propagators, or FP32 with LEM_PREC_SPLIT_FAST). */
typedef enum { LEM_SCHEME_EULER = 0, LEM_SCHEME_RB3 = 1 } lem_scheme;

/* How lem_step applies the propagators (lem_info.apply_path). */
typedef enum {
  LEM_APPLY_FP64_GEMM = 0,   /* FP64, one gathered GEMM per class of tiles */
  LEM_APPLY_FP64_GEMV = 1,   /* FP64, one batched GEMV over all tiles (many classes) */
  LEM_APPLY_F32_GEMV = 2,    /* FP32 propagators, float-float accumulation (complex: of FP32
                                FMA sums over 16-byte chunks of a row) */
  LEM_APPLY_TC_SPLIT = 3,    /* shared propagator on the tcgen05 tensor cores */
  LEM_APPLY_FP64_BAND = 4,   /* truncated FP64 propagators (lem_set_truncation), batched GEMV */
  LEM_APPLY_F32_BAND = 5     /* truncated FP32 propagators, float-float accumulation */
} lem_apply_path;

typedef struct {
  int ndim;               /* 1 or 2 */
  int64_t n[2];           /* mesh nodes per axis: {N, unused} or {ny, nx} */
  int bc[2];              /* lem_bc per axis, same order as n */
  const double* coef[5];  /* host pointers to C, W, E, S, N (S, N unused in 1D) */
  int64_t coef_stride;    /* 0: each coef[k] points at one value (constant coefficients);
                             1: each points at n[0]*n[1] values, row-major */
  int reaction;           /* 0: linear; 1: adds u - u^3 to A u (exponential Euler-
                             Rosenbrock, Jacobian A + diag(1 - 3u^2), Sec. 4); 2: the
                             porous-medium equation of Sec. 4.2 (Eq. porous), F(u) = A phi(u)
                             with phi(u) = |u|^(m-1) u and m = porous_m, Jacobian
                             A diag(phi'(u)); real problems, LEM_SCHEME_EULER, stepped by
                             lem_step (batches, the server and the allocation-free step refuse
                             it) */
  double dt;              /* time step (> 0) */
  int tile[2];            /* owner-tile size per axis (>= 1) */
  int overlap[2];         /* buffer width H per side and axis (>= 0) */
  int mode;               /* lem_mode */
  int prec;               /* lem_prec */
  int refresh;            /* reaction 1 or 2: rebuild the Jacobian propagators every
                             `refresh` steps (0: build once at the first step) */
  int scheme;             /* lem_scheme (0: the exponential Euler step of Eq. lem) */
  int complex_values;     /* 1: complex coefficients and states (e.g. the Schroedinger test of
                             Sec. 4.1). coef[k] then holds the real parts and coef_im[k] the
                             imaginary parts (NULL: zero); states are interleaved (re, im)
                             FP64 pairs, 2 * n[0] * n[1] doubles. Linear problems only, scheme
                             0; the apply runs on the batched GEMV with each class's propagator
                             stored as its real embedding [[Re P, -Im P], [Im P, Re P]]. */
  const double* coef_im[5];
  double porous_m;        /* reaction 2: the exponent m (finite, > 1); ignored otherwise */
} lem_problem_desc;

typedef struct lem_ctx lem_ctx;

/* Plan facts of a context (filled by lem_get_info). */
typedef struct {
  int64_t ntiles;         /* number of owner tiles D_i */
  int64_t nclasses;       /* distinct local operators (propagators) */
  int64_t n_loc;          /* padded window size (max |M_i|; complex: twice that, the real
                             embedding of the propagator) */
  int64_t n_int;          /* padded tile size (max |D_i|; complex: twice that) */
  int squarings_max;      /* largest scaling-and-squaring count s over the classes */
  int built;              /* 1 once propagators exist */
  int split_path;         /* 1 if lem_step runs the tcgen05 split-precision kernel */
  int64_t device_bytes;   /* device memory held by the context */
  int apply_path;         /* lem_apply_path */
} lem_info;

/* Create a context on CUDA device `device`, enqueueing its work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream). Validates the descriptor, copies the
 * coefficients, plans tiles/windows (Sec. 3, Fig. 3) and groups windows with identical
 * local operators into classes. Allocates device memory. Does not build propagators.
 * Errors: LEM_EINVAL (descriptor), LEM_ENOMEM, LEM_ECUDA. On error *out is NULL. */
lem_status lem_create(const lem_problem_desc* desc, int device, void* cuda_stream, lem_ctx** out);

/* Build every class's local propagator on the device (Sec. 3 step 2 with Pade
 * approximation and scaling-and-squaring, Sec. 1 / Sec. 4): P = R_D phi_1(dt A_M)
 * (PHI) or R_D exp(dt A_M) (EXP), degree-13 Pade, s from the exact 1-norm, Gauss-Jordan
 * elimination with partial pivoting for the denominator. FP64 tier: FP64 products; split
 * tiers: tensor-core slice products and a blocked elimination (see lem_prec).
 * LEM_SCHEME_RB3 builds phi_1 and phi_3 together; complex problems build the real embedding.
 * d_state (device, FP64, may be NULL for linear problems) is the state at which the
 * Jacobian of a nonlinear problem (reaction 1 or 2) is taken. Synchronises the context stream
 * before returning.
 * Errors: LEM_EINVAL (nonlinear problem without state), LEM_ENUMERIC (singular denominator),
 * LEM_ECUDA. */
lem_status lem_build_propagators(lem_ctx* ctx, const double* d_state);

/* Advance the device state d_state (FP64, row-major, in/out; complex: interleaved pairs) by
 * nsteps LEM steps (Sec. 3 steps 1-3). Builds the propagators first if they do not exist;
 * for a nonlinear problem (reaction 1 or 2) it rebuilds them every `refresh` steps. Small linear real problems on
 * the GEMV paths run all nsteps in one cooperative launch (identical results). On the
 * tensor-core split path the call's first kernel (the first step's measuring residual pass)
 * reads d_state, converting it to the float-float state the steps run on. Work is
 * enqueued on the context stream; the call returns after enqueueing (no synchronisation)
 * unless a rebuild is due.
 * Errors: LEM_EINVAL (nsteps < 0, NULL state), LEM_ECUDA. */
lem_status lem_step(lem_ctx* ctx, double* d_state, int nsteps);

/* Same as lem_step on a HOST state (pinned or pageable): copies it to the device,
 * advances nsteps, copies it back and synchronises. The first call allocates a device copy
 * of the state, kept by the context. On the tensor-core split path (apply path
 * LEM_APPLY_TC_SPLIT, propagators built) with pinned host memory that is mapped into the
 * device's address space, the state is read and written in place by the kernels that convert
 * it to and from the float-float state instead (same results, no device copy).
 * Errors: those of lem_step, LEM_ENOMEM, LEM_ETIMEOUT (a bounded wait in a tensor-core kernel
 * expired), LEM_ECUDA. */
lem_status lem_step_host(lem_ctx* ctx, double* h_state, int nsteps);

/* Copy class `cls`'s propagator (n_int x n_loc, row-major, FP64, zero padded) into host
 * memory h_out. Rows follow the tile's owner nodes in row-major order, columns the window
 * nodes in row-major order. Complex problems: the real embedding [[Re P, -Im P],
 * [Im P, Re P]] (owner rows real parts then imaginary parts; window columns likewise).
 * Errors: LEM_ENOTREADY (not built), LEM_EINVAL. */
lem_status lem_get_propagator(lem_ctx* ctx, int64_t cls, double* h_out);

/* The same for the phi_3 propagator of class `cls` (LEM_SCHEME_RB3 contexts only; LEM_EINVAL
 * otherwise): R_D phi_3(dt J_M), the correction stage of the third-order Rosenbrock step. */
lem_status lem_get_propagator_phi3(lem_ctx* ctx, int64_t cls, double* h_out);

/* Load every class's propagator from host memory (FP64, nclasses x n_int x n_loc, the layout
 * lem_get_propagator returns per class) instead of building them: with lem_get_propagator this
 * checkpoints and restores a context's propagators bit for bit. h_squarings (nclasses values,
 * or NULL) is only recorded. Marks the context built. Errors: LEM_EINVAL, LEM_ECUDA. */
lem_status lem_set_propagators(lem_ctx* ctx, const double* h_P, const int* h_squarings);

/* Class of tile `tile` (row-major over the tile grid) or -1 on a bad index. */
int64_t lem_tile_class(const lem_ctx* ctx, int64_t tile);

/* Squaring count s used for class `cls` (-1 before the build or on a bad index). */
int lem_class_squarings(const lem_ctx* ctx, int64_t cls);

/* Fill *out with the context's plan facts (lem_info). Errors: LEM_EINVAL (NULL argument). */
lem_status lem_get_info(const lem_ctx* ctx, lem_info* out);

/* Host-only planning query (no device is touched): validates `desc` and reports the
 * decomposition of Sec. 3 -- number of tiles and classes, padded window and tile sizes.
 * If tile_info is not NULL it receives 11 int32 per tile (row-major over the tile grid):
 * window origin (y, x), window extent (y, x), owner offset in the window (y, x),
 * owner extent (y, x), first owner node (y, x), class. 1D meshes use the x entries
 * (y entries are 0, 1, 0, 1, 0). Errors: LEM_EINVAL. */
lem_status lem_plan_query(const lem_problem_desc* desc, int64_t* ntiles, int64_t* nclasses,
                          int64_t* n_loc, int64_t* n_int, int32_t* tile_info);

/* Per-kernel timing of the dominant propagator-apply kernel (for benchmarks).
 * lem_set_timing(ctx, k) with k >= 1 makes later lem_step calls bracket every k-th launch
 * (k = 1: every launch; an event between two launches keeps the second from starting its
 * set-up while the first finishes, so a period larger than 1 disturbs less) of the apply
 * kernel (the tcgen05 split GEMM, the FP64 apply GEMMs, the GEMV -- with LEM_SCHEME_RB3 both
 * stages of a step together -- or the persistent multi-step GEMV) with CUDA events on the
 * context stream; lem_get_timing synchronises, adds the elapsed times of all recorded
 * launches since the last call to *total_ms and their count to *launches, and resets them.
 * Errors: LEM_EINVAL, LEM_ECUDA. */
lem_status lem_set_timing(lem_ctx* ctx, int enable);
lem_status lem_get_timing(lem_ctx* ctx, double* total_ms, int64_t* launches);

/* Allocation-free FP64 step (the paper has no counterpart; this is a service to callers).
 * Same result as lem_step on an LEM_PREC_FP64 context, for callers that must not allocate
 * device memory while they step: runtimes that own all device memory through their own
 * pool and forbid later driver allocations, and loops that cannot take cudaMalloc's
 * implicit synchronisation. Its per-step scratch comes from one static 8 MiB device array
 * that every GPU loading liblem.so holds until the process exits; no call allocates or frees
 * memory. The scratch is the residual, plus the gathered windows and local results on the
 * GEMM apply path (apply_path LEM_APPLY_FP64_GEMM); contexts on the batched GEMV
 * (LEM_APPLY_FP64_GEMV, many propagator classes) need the residual alone and run the same
 * GEMV kernel as lem_step.
 * - Needs built propagators (lem_build_propagators first: LEM_ENOTREADY otherwise) and
 *   no Jacobian refresh (reaction with refresh > 0: LEM_EINVAL), since building allocates.
 * - Real problems with the exponential Euler scheme only; the porous-medium problem
 *   (reaction 2) and truncated propagators (lem_set_truncation with tol >= 0) are refused
 *   (LEM_EINVAL).
 * - Problems whose scratch, npts (+ ntiles*(n_loc + n_int) on the GEMM path) doubles (each
 *   part rounded up to 32), exceeds 8 MiB are rejected with LEM_EINVAL and a message giving
 *   both sizes.
 * - The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 *   which may load the library's device code on that device) and keeps it for the life of
 *   the process; make that first call before any stream capture. A device reset
 *   (cudaDeviceReset) invalidates the kept address: do not call this entry point after one.
 * - Every call on a device shares the one array, which keeps the last call's contents
 *   (each step rewrites every element it reads, so nothing needs clearing). Calls whose
 *   work overlaps on the GPU (other streams, other contexts, other threads) race on it.
 * Errors: LEM_EINVAL, LEM_ENOTREADY, LEM_ECUDA. */
lem_status lem_step_fp64_noalloc(lem_ctx* ctx, double* d_state, int nsteps);

/* Truncated propagators (Sec. 2, Theorem 1: the entries of the exponential of a banded
 * matrix decay faster than exponentially away from the band, which is what makes the local
 * problems accurate at all). With tol >= 0, each owner row of every class's propagator keeps
 * only the window nodes inside a box around its owner node, offsets -ly..hy along y and
 * -lx..hx along x in window coordinates, and later lem_step calls apply the kept entries only
 * (apply_path LEM_APPLY_F32_BAND for LEM_PREC_SPLIT_FAST in PHI mode, LEM_APPLY_FP64_BAND
 * otherwise, whatever path lem_create chose). Each side's extent, per class, is the smallest
 * e >= 0 with
 *     max_d sum_{m beyond e on that side} |P_dm| <= (tol / 4) * max_d sum_m |P_dm|,
 * so one step's increment at any owner node moves by at most tol * max_d sum_m |P_dm| *
 * max|r| (r the residual in PHI mode, the state in EXP mode). tol = 0 keeps every nonzero
 * entry; tol < 0 turns truncation off and restores the path lem_create chose. Extents are
 * recomputed from the propagators after every build (refreshes included); the first step
 * after a build synchronises the context stream once to read them. A stored box row holds
 * min(ly + hy + 1, wy) x min(lx + hx + 1, wx) values (columns padded to a multiple of 4).
 * Real problems with LEM_SCHEME_EULER only (complex or third-order contexts: LEM_EINVAL);
 * windows of at most 1024 nodes per axis. The batch's fused schedule, the server and the
 * allocation-free step do not take truncated contexts (a batch runs them in lanes).
 * Errors: LEM_EINVAL. */
lem_status lem_set_truncation(lem_ctx* ctx, double tol);

/* The box kept for class cls: ext = {ly, hy, lx, hx}; *row_values (may be NULL) = values
 * stored per owner row. cls = -1: ext is zeroed and *row_values is the number of values stored
 * for all classes together (what one step streams). Computes the extents if the propagators
 * changed since the last step.
 * Errors: LEM_EINVAL (no truncation set, class out of range), LEM_ENOTREADY (not built),
 * LEM_ECUDA. */
lem_status lem_get_band(lem_ctx* ctx, int64_t cls, int32_t* ext, int64_t* row_values);

/* Synchronise the context stream and return any deferred device error. */
lem_status lem_sync(lem_ctx* ctx);

/* Synchronise the context stream and free everything the context holds (device memory,
 * events, the split path's packed operands). NULL is a no-op. The caller's state buffers
 * and stream are not touched. */
void lem_destroy(lem_ctx* ctx);

/* ------------------------------------------------------------------ batching
 * Advance many independent problems (contexts) together with one CUDA graph launch per
 * `steps_per_launch` LEM steps. At creation every context is built and warmed up on a copy
 * of its state and its step time is measured; an autotuner then captures and times candidate
 * schedules (lem_batch_candidates) and keeps the fastest (lem_batch_info): lanes with
 * lanes/2, lanes and 2 lanes (within 1..n), and, when every context is on the same
 * tensor-core split tier, the fused schedule with window-block width caps 0 (each context's
 * own block), 128, 64 and 32 (each problem takes the power of two in [16, cap] whose blocks
 * load the fewest operand bytes). The states d_states[i] (device, FP64) are captured: each launch
 * advances them in place. Contexts with a Jacobian refresh (reaction with refresh > 0) are
 * rejected, because rebuilding propagators cannot be captured; so are complex contexts and the
 * porous-medium problem (step those with lem_step). The contexts' streams are used only outside the
 * graph; the graph runs on `stream`. The paper has no batching layer (its local problems are
 * independent, Sec. 3). Errors: LEM_EINVAL, LEM_ENOMEM, LEM_ECUDA. */
typedef struct lem_batch lem_batch;

lem_status lem_batch_create(lem_ctx* const* ctxs, double* const* d_states, int n, int steps_per_launch,
                            int lanes, void* cuda_stream, lem_batch** out);

/* Replay the graph `launches` times on the batch stream (asynchronous). */
lem_status lem_batch_run(lem_batch* b, int launches);

/* Measured single-launch time of each problem (ms, host array of n) and its lane. */
lem_status lem_batch_schedule(const lem_batch* b, double* est_ms, int* lane);

/* Which schedule the graph runs. The candidates are captured and timed on scratch copies of
 * the states at creation, and the fastest is kept: lanes (every context's own launches on
 * concurrent graph branches, problems assigned longest-first) or fused (all contexts on the
 * same tensor-core split tier: one residual and one persistent GEMM launch per LEM step for
 * the whole batch). lanes_ms and fused_ms are the best timed candidate of each kind;
 * fused_ms = -1 when the contexts cannot be fused. The environment variable
 * LEM_BATCH_SCHEDULE=lanes|fused|fused:<cap>, read at creation, restricts the choice to one
 * kind (or one fused width cap). */
lem_status lem_batch_info(const lem_batch* b, int* fused, double* lanes_ms, double* fused_ms);

/* Wait for the batch stream; LEM_ETIMEOUT if a tensor-core kernel gave up waiting. */
lem_status lem_batch_sync(lem_batch* b);

/* One autotuner candidate: fused (1) or lanes (0), its lane count (lanes) or window-block
 * width cap (fused), the best of three timed graph launches (ms), and whether it was chosen. */
typedef struct {
  int fused;
  int lanes;
  int n_cap;
  double ms;
  int chosen;
} lem_batch_candidate;

/* The autotuner's candidates in the order they were timed: *count = how many; up to `max`
 * are copied to out. Errors: LEM_EINVAL. */
lem_status lem_batch_candidates(const lem_batch* b, int max, lem_batch_candidate* out, int* count);

/* Work of one fused GEMM launch (one LEM step of every problem): the algorithmic FLOPs
 * (products x 2 x owner rows x window nodes over all windows) and the FLOPs the MMAs execute
 * (128-row M blocks, whole window blocks, window rows padded to 16-node K steps). Errors:
 * LEM_EINVAL (NULL arguments, or the batch runs the lanes schedule). */
lem_status lem_batch_gemm_work(const lem_batch* b, double* algorithmic_flops, double* executed_flops);

/* Fused schedule only: run `nsteps` LEM steps of every problem outside the graph (advancing the
 * captured states like a launch does) with CUDA events around each kernel, and report the
 * time spent in the GEMM launches, in the residual launches and in the rest (state
 * conversions), plus the GEMM launches' algorithmic FLOPs (products x 2 x owner rows x window
 * nodes x windows). LEM_EINVAL on a lanes schedule. */
lem_status lem_batch_profile(lem_batch* b, int nsteps, double* gemm_ms, double* residual_ms, double* other_ms,
                             double* gemm_flops);

void lem_batch_destroy(lem_batch* b);

/* ------------------------------------------------------------------ serving
 * A server advances many independent LEM problems on one device with continuous batching:
 * requests are admitted while their device memory fits the budget (otherwise they wait in
 * the queue; they are not failed), every admitted request advances a few LEM steps at a time
 * on the stream of its context, and requests that arrive while others run join between those
 * chunks, so their work overlaps on the device. Problems with identical descriptors and
 * precision share one context (one set of propagators), kept cached while the budget allows.
 * The precision follows the tolerance tier: tol >= 1e-6 selects LEM_PREC_SPLIT when the
 * problem is eligible for it, anything tighter (or an ineligible problem) LEM_PREC_FP64.
 * The paper has no serving layer; Sec. 3's independent local problems are what makes the
 * requests independent. A server is thread-safe. */
typedef struct lem_server lem_server;

typedef struct {
  int64_t submitted, admitted, completed, failed;
  int64_t queued, active;       /* at the time of the call */
  int64_t dof_steps;            /* owner nodes x LEM steps of completed requests */
  double p50_ms, p99_ms;        /* submit-to-result latency of completed requests */
  double first_admit_to_last_done_s;
  int64_t device_bytes;         /* states, scratch and cached contexts held now */
  int64_t ctx_hits, ctx_misses; /* context cache */
  int64_t ctx_adopted;          /* new contexts that took a cached propagator of the same local
                                   operator (another mesh size) instead of building one */
  double worker_admit_s;        /* worker-thread time spent admitting (context creation) */
  double worker_issue_s;        /* worker-thread time spent issuing steps (incl. first builds) */
  double worker_build_s;        /* of worker_admit_s: building the first propagator of each operator */
  int64_t ctx_built;            /* contexts that built at admission (first of their operator) */
  int64_t adopt_failed;         /* contexts whose operator had a donor that did not match */
  /* per tier: [0] tol >= 1e-6 (the split tier where the problem allows it), [1] tol < 1e-6 */
  int64_t tier_completed[2], tier_dof_steps[2];
  double tier_p50_ms[2], tier_p99_ms[2];
} lem_server_stats;

/* Create a server on `device` with a device-memory budget in bytes (states, scratch and cached
 * propagators; 0 = 80 GiB). Starts one worker thread. Requests with tol >= 1e-6 run on the
 * tensor-core split tier where their problem allows it (2D periodic, one shared propagator)
 * and keep their state in float-float on the device until they complete, so each result is
 * the same bit for bit as one lem_step call of all its steps; the others run the FP64 path.
 * The tiers queue separately, each in arrival order: the split tier is admitted first, the
 * FP64 tier while fewer than 8 of its requests run and within three quarters of the budget.
 * Split-tier contexts get the device's highest stream priority, FP64-tier ones its lowest, and
 * FP64-tier steps are issued only while no split-tier request has work on the GPU or waits
 * for admission (else one FP64-tier chunk every 50 ms). Errors: LEM_EINVAL, LEM_ECUDA. */
lem_status lem_server_create(size_t hbm_budget_bytes, int device, lem_server** out);

/* Queue a request to advance the host state h_state (FP64, row-major, in/out; it must stay
 * valid and untouched until the request is done) by nsteps LEM steps of the problem `desc`
 * (copied) within relative tolerance tier `tol`. Returns at once with a ticket. Real problems
 * only, without the porous-medium nonlinearity (reaction 2).
 * Errors: LEM_EINVAL (descriptor, complex or porous-medium problem, nsteps < 0, NULL pointers),
 * LEM_EBUSY (server stopping). */
lem_status lem_submit(lem_server* srv, const lem_problem_desc* desc, double tol, double* h_state,
                      int nsteps, uint64_t* ticket);

/* Non-blocking: *done = 1 once the result is back in h_state. Returns the request's error
 * status if it failed (then *done = 1), LEM_EINVAL for an unknown ticket, else LEM_OK. */
lem_status lem_poll(lem_server* srv, uint64_t ticket, int* done);

/* Block until the request is done or `timeout_s` seconds pass (LEM_ETIMEOUT; the request
 * keeps running). Returns the request's own status when done. */
lem_status lem_wait(lem_server* srv, uint64_t ticket, double timeout_s);

lem_status lem_server_get_stats(lem_server* srv, lem_server_stats* out);

/* Zero the counters, timers and latency record (after a warm-up, say); requests in flight
 * are still counted when they complete. Cached contexts and propagators stay. */
lem_status lem_server_reset_stats(lem_server* srv);

/* Stop the worker after the admitted requests finish (queued ones are failed with LEM_EBUSY),
 * free everything. */
void lem_server_destroy(lem_server* srv);

const char* lem_status_str(lem_status s);
const char* lem_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LEM_H */
