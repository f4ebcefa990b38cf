/*
 * mg.h - C ABI of the GB300 delayed-assembly multigrid library (libmg.so).
 *
 * Solves -div(eps grad u) = f on the unit square / cube with u = 0 on the
 * boundary, using d-linear Ritz-Galerkin finite elements on a regular grid of
 * N^d cells, N = 3^L (Murray & Weinzierl, "Delayed approximate matrix
 * assembly in multigrid with dynamic precisions", Section "A matrix-free
 * additive multigrid solver on spacetrees": nodal d-linear elements giving
 * 9-/27-point stencils; 3:1 refinement of the spacetree).
 *
 * Conventions shared by every entry point:
 *   - Every call returns an mg_status; no exception crosses the ABI.  On an
 *     error, mg_last_error() returns a thread-local message.
 *   - Descriptors passed in are caller-owned and copied; the library owns all
 *     device memory it allocates.  Host buffers passed to mg_get_* are
 *     caller-owned and written synchronously.
 *   - Vertex arrays are the full (N+1)^d grid, lexicographic with x fastest,
 *     boundary entries included (they are zero).  Cells are numbered the same
 *     way on the N^d grid.  The 2^d local vertices of a cell are numbered by
 *     the bits (b_x, b_y[, b_z]) of the local index.
 *   - Work is issued on the problem's CUDA stream (given at creation or owned
 *     by the problem); calls that return host data synchronise that stream.
 *   - One problem must not be used from two threads at once; distinct
 *     problems may be used concurrently.
 */
#ifndef MG_H
#define MG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MG_OK = 0,
  MG_ERR_INVALID = 1,        /* bad argument: size not 3^L, bad dim, null pointer, ... */
  MG_ERR_OOM = 2,            /* device or host allocation failed, or above the HBM budget */
  MG_ERR_CUDA = 3,           /* a CUDA call failed (message in mg_last_error) */
  MG_ERR_TIMEOUT = 4,        /* a bounded wait ran out */
  MG_ERR_DIVERGED = 5,       /* ||r|| grew above 1e2 ||r_0|| */
  MG_ERR_NOT_CONVERGED = 6,  /* max_cycles reached before rtol */
  MG_ERR_PENDING = 7,        /* request not finished yet (mg_poll) */
  MG_ERR_CANCELLED = 8,      /* request cancelled or server shut down */
  MG_ERR_INJECTED = 9        /* failure injected on the host for tests */
} mg_status;

/* Material field families (eps > 0).  The field is evaluated at sub-box
 * centres x = (2(i s + j) + 1) / (2 N s) per axis, i the cell and j the
 * sub-box index (Section "Numerical computation of stencils": eps is taken
 * constant on each of the s^d sub-boxes of a cell). */
typedef enum {
  MG_EPS_CONST = 0,    /* eps = v_out */
  MG_EPS_DISC = 1,     /* eps = v_in if |x - center|^2 < radius^2 else v_out */
  MG_EPS_FOURIER = 2,  /* eps = v_out exp(sigma sqrt(2/M) sum_m cos(2 pi k_m.x + phase_m)) */
  MG_EPS_BOXES = 3,    /* eps = v_in inside the union of [lo, hi) boxes, else v_out */
  MG_EPS_THETA = 4     /* eps = 1 + (0.3/d) prod_i exp(-theta x_i) cos(pi theta x_i)
                          (the paper's Eq. "theta-setup") */
} mg_eps_kind;

#define MG_MAX_MODES 32
#define MG_MAX_BOXES 64

typedef struct {
  int32_t kind;          /* mg_eps_kind */
  int32_t n_modes;       /* FOURIER: M, 1..MG_MAX_MODES */
  int32_t n_boxes;       /* BOXES: 1..MG_MAX_BOXES */
  int32_t pad0;
  double v_out;          /* constant value / background / Fourier base factor */
  double v_in;           /* DISC and BOXES inside value */
  double center[3];      /* DISC */
  double radius;         /* DISC */
  double sigma;          /* FOURIER amplitude */
  double theta;          /* THETA */
  double jump_x;         /* all kinds: eps *= jump_factor where x_0 >= jump_x */
  double jump_factor;    /* 1 = no jump */
  int32_t k[MG_MAX_MODES][3];  /* FOURIER integer wavenumbers */
  double phase[MG_MAX_MODES];  /* FOURIER phases */
  double box_lo[MG_MAX_BOXES][3];
  double box_hi[MG_MAX_BOXES][3];
} mg_eps_desc;

/* Operator storage and arithmetic of a solve. */
typedef enum {
  /* element matrices at s_schedule[n_s-1] in FP64, assembled before the first
   * cycle (the paper's a priori assembly, p = (T, _, 8)); FP64 everywhere */
  MG_PATH_FP64_PLAIN = 0,
  /* FP64 storage and arithmetic; cycling starts on the geometric stencils
   * (s = 1) while s_schedule[1..] are assembled on a side stream and
   * published at cycle boundaries (Section "Asynchronous and anarchic
   * stencil integration"); finished chunks are held until the schedule is
   * done, the solver waits for them, or 16 cycles have passed since the first
   * of them finished, so that one publication restarts the iteration once */
  MG_PATH_FP64_DELAYED = 1,
  /* as FP64_DELAYED, but the fine element matrices are stored as FP32 cell
   * centre eps plus a lossy hierarchical surplus (FP8-e4m3 / FP16 / FP32 with
   * an FP32 per-cell scale; Section "Precision toggling and information
   * density"), V-cycles run in FP32 and the outer residual, norms and the
   * coarsest solve in FP64 */
  MG_PATH_MIXED_DELAYED = 2,
  /* mixed storage/arithmetic, final accuracy assembled before cycling */
  MG_PATH_MIXED_PLAIN = 3
} mg_path;

typedef enum {
  MG_OUTER_FCG = 0,        /* flexible CG (Notay FCG(1)) preconditioned by the V-cycle */
  MG_OUTER_RICHARDSON = 1  /* residual correction u += V(f - A u) */
} mg_outer;

/* Multigrid cycle of one outer iteration (applied to the outer residual). */
typedef enum {
  MG_CYCLE_V = 0,           /* multiplicative V(nu_pre, nu_post), damped Jacobi, exact coarsest solve */
  MG_CYCLE_ADDITIVE = 1,    /* additive: every level smooths (one damped Jacobi step from zero) its
                               restriction of the fine residual at once, the coarsest is solved
                               exactly, all corrections are prolongated and summed (Section
                               "adaFAC-x", the "standard additive scheme" term of Eq. "adaFAC-x") */
  MG_CYCLE_ADAFAC_PI = 2,   /* additive plus, on every level above the coarsest, minus P of one
                               damped Jacobi step on the next coarser level of the injected level
                               residual (adaFAC-PI: P and injection in the auxiliary equation) */
  MG_CYCLE_ADAFAC_JAC = 3   /* the same with the auxiliary right-hand side R (r_l - A_l c_l): the
                               level residual left by the level's own Jacobi step, restricted
                               (adaFAC-Jac: Jacobi-smoothed restriction) */
} mg_cycle;

typedef struct {
  int32_t dim;             /* 2 or 3 */
  int32_t n_cells;         /* cells per axis, 3^L with L >= 2 (N >= 9: at least one level above the 3^d coarse solve) */
  mg_eps_desc eps;
  double f_const;          /* right-hand side f (constant) */
  int32_t path;            /* mg_path */
  int32_t outer;           /* mg_outer */
  int32_t s_schedule[8];   /* accuracies (sub-boxes per axis), increasing; the
                              last one is final.  Delayed paths start at s = 1. */
  int32_t n_s;             /* 1..8 */
  double compress_tau;     /* mixed paths: per-cell entry error bound relative
                              to max|A_c| (0 => 1e-6) */
  double omega;            /* Jacobi damping (0 => 0.6) */
  int32_t nu_pre, nu_post; /* smoothing steps (0,0 => 2,2) */
  double rtol;             /* stop at ||f - A u||_2 <= rtol ||f||_2 (0 => 1e-8) */
  int32_t max_cycles;      /* (0 => 500) */
  int32_t chunks;          /* delayed assembly chunks along the last axis (0 => auto) */
  const double* u0;        /* optional host initial guess, (N+1)^d values; NULL => 0.
                              Read during mg_create_problem only. */
  double adapt_C;          /* > 0: adaptive per-cell accuracy (Section "Adaptive stencil
                              integration", Eq. "termination-criterion"): each cell walks
                              s_schedule and stops refining at the first level whose
                              element matrix differs from the stored previous one by less
                              than adapt_C in the relative element-wise maximum norm (the
                              paper uses 1%); the plain paths then assemble the whole
                              schedule before solving.  0 => every cell reaches the last
                              accuracy of the schedule. */
  int32_t cycle;           /* mg_cycle: the multigrid cycle each outer iteration applies */
  int32_t adapt_keep;      /* adapt_C > 0: which matrix a cell keeps when its change falls below
                              adapt_C.  0 => the newer one (the rule as stated in Section
                              "Adaptive stencil integration"); 1 => the older one it was
                              tested against, with that older accuracy (the account of Table
                              "memory-footprint" in the Results: the lowest accuracy that
                              passes is used all the way through).  Other values: MG_ERR_INVALID. */
  double coarse_tau;       /* mixed paths, > 0: every coarse level stores its Galerkin operator
                              as the hierarchical surplus over its one-sample rediscretisation
                              eps(x_C) K_ref h_C^(d-2) (eps at the coarse cell centre), with the
                              finest level's storage classes under this relative bound (Section
                              "Precision toggling and information density"); the level's
                              stencils, the next Galerkin product and the coarsest factor use
                              the stored operator.  0 => coarse operators in full FP32. */
} mg_problem_desc;

typedef struct {
  int32_t status;          /* mg_status of the solve */
  int32_t cycles;          /* V-cycles (outer iterations) run */
  int32_t publishes;       /* chunk publications applied during the solve */
  int32_t final_s;         /* accuracy of the operator at the end */
  double rel_residual;     /* ||f - A u||_2 / ||f||_2, FP64, stored operator */
  double time_ms;          /* wall time of mg_solve */
  double assembly_ms;      /* wall time spent blocked on assembly (plain paths) */
  int64_t cells_by_class[4];   /* mixed paths: cells per storage class 0..3 */
  int64_t payload_bytes;   /* fine-level operator bytes (payload + per-cell data) */
} mg_solve_info;

typedef struct mg_problem mg_problem;

/* Creates a problem: allocates the level hierarchy, computes the geometric
 * (s = 1, cell-centre eps) stencils and their Galerkin coarse operators.
 * cuda_stream: a cudaStream_t to issue work on, or NULL for an own stream.
 * Errors: MG_ERR_INVALID (dim, n_cells, eps, schedule), MG_ERR_OOM, MG_ERR_CUDA. */
mg_status mg_create_problem(const mg_problem_desc* desc, void* cuda_stream, mg_problem** out);

/* Frees every device and host resource of the problem (waits for its work). */
mg_status mg_destroy_problem(mg_problem* p);

/* Assembles the finest-level element matrices at accuracy s (s^d sub-boxes
 * per cell; Section "Numerical computation of stencils", A^(geo)(n)), stores
 * them in the problem's format and recomputes the coarse Galerkin operators.
 * async = 0: in stream order, published at once.  async = 1: on the side
 * stream chunk by chunk; completed chunks are published at a later cycle
 * boundary, under the holding rule of MG_PATH_FP64_DELAYED (Section
 * "Asynchronous and anarchic stencil integration").
 * Errors: MG_ERR_INVALID (s < 1 or s > 64), MG_ERR_OOM, MG_ERR_CUDA. */
mg_status mg_assemble_level(mg_problem* p, int s, int async);

/* Runs n outer iterations (each one multigrid cycle of desc->cycle) from the
 * current solution (n = 0: only the residual),
 * publishing completed asynchronous chunks at cycle boundaries, and returns
 * the FP64 relative residual ||f - A u||_2 / ||f||_2 of the stored operator.
 * rel_residual may be NULL.  Errors: MG_ERR_INVALID, MG_ERR_CUDA. */
mg_status mg_vcycle(mg_problem* p, int n, double* rel_residual);

/* Full solve according to desc->path: for plain paths assembles
 * s_schedule[n_s-1] first; for delayed paths starts the schedule on the side
 * stream and cycles meanwhile.  Stops when rel_residual <= rtol AND every
 * chunk holds its final accuracy (never earlier: Section "Consistency with
 * dynamic termination criteria and starvation effects").  info may be NULL.
 * Errors: MG_ERR_NOT_CONVERGED, MG_ERR_DIVERGED, MG_ERR_CUDA. */
mg_status mg_solve(mg_problem* p, mg_solve_info* info);

/* Copies u ((N+1)^d FP64 values) to host_dst; n must be (N+1)^d. */
mg_status mg_get_solution(const mg_problem* p, double* host_dst, size_t n);

/* Copies the stored (decoded) element matrices of level `level` (0 = finest,
 * 1 = the next coarser, ...) as FP64, 2^d x 2^d row-major per cell, cells in
 * index order; n must be n_cells(level)^d * 4^d. */
mg_status mg_get_element_matrices(const mg_problem* p, int level, double* host_dst, size_t n);

/* Decoded element matrices of selected cells of `level` (flat cell indices,
 * host array of ncells entries); host_dst receives ncells * 4^d FP64 values,
 * 2^d x 2^d row-major per cell, in the order of `cells`.  Used for sampled
 * checks of large grids.  Errors: MG_ERR_INVALID (index out of range). */
mg_status mg_get_cell_matrices(const mg_problem* p, int level, const int64_t* cells, size_t ncells,
                               double* host_dst);

/* One record per outer iteration of the last mg_solve (Section "Consistency
 * with dynamic termination criteria and starvation effects": the residual
 * and the number of pending background integration tasks per iteration).
 * rel_residual_est: FP64 paths the recurrence residual ||r||/||f||; mixed
 * paths the outer residual at the last restart times the inner FP32
 * residual (an estimate of ||f - A(u + e)|| / ||f||).  pending_jobs: chunk
 * assembly jobs enqueued, running, finished or held and not yet published. */
typedef struct {
  int32_t cycle;           /* 1-based outer iteration */
  int32_t pending_jobs;
  int32_t publishes;       /* chunk publications so far */
  int32_t restarted;       /* 1 if an outer restart preceded this iteration */
  double rel_residual_est;
  double time_ms;          /* since the start of mg_solve, when the iteration's scalars were read */
} mg_trace_entry;

/* Copies up to cap records of the last solve to host_out (may be NULL with
 * cap = 0) and the total count to *n.  Errors: MG_ERR_INVALID (null p or n). */
mg_status mg_get_trace(const mg_problem* p, mg_trace_entry* host_out, size_t cap, size_t* n);

/* The paper's own storage format (Section "Precision toggling and
 * information density") applied to the finest level's stored operator A:
 * per cell the hierarchical surplus A - eps_c K_ref h^(d-2) (eps_c the
 * cell-centre value the path stores), held with p3 bytes per entry: a sign
 * bit, a truncated mantissa of 8 (p3 - 1) - 1 bits and a signed-char exponent
 * without bias (p3 = 8: plain FP64).  p3 = 0 (nothing stored) when the
 * surplus' Frobenius norm is below delta, else the smallest p3 with every
 * entry's truncation error at most delta.  The values the format cannot
 * normalise (below 2^-127) are held as multiples of 2^-(127 + m); values at or
 * above 2^128 saturate.  Outputs (each may be NULL): p3 per cell (host,
 * n_cells^d bytes), the decoded stored matrices eps_c K + trunc(surplus)
 * (host, n_cells^d * 4^d FP64, 2^d x 2^d row-major per cell), and the
 * statistics below; n must be n_cells^d.  The problem is not modified.
 * Errors: MG_ERR_INVALID (n, delta < 0 or not finite), MG_ERR_OOM, MG_ERR_CUDA. */
typedef struct {
  int64_t cells_by_p3[9];   /* cells per p3 = 0 .. 8 (1 never occurs) */
  double bytes_full;        /* 4^d doubles per cell */
  double bytes_paper;       /* one marker byte plus 4^d p3 bytes per cell */
  double compression;       /* bytes_full / bytes_paper */
  double max_abs_error;     /* max over all entries |stored - A| */
} mg_paper_format_stats;

mg_status mg_paper_format(const mg_problem* p, double delta, uint8_t* p3_host, double* decoded_host, size_t n,
                          mg_paper_format_stats* stats);

/* Storage classes (0..3) of the cells of coarse level `level` (1 = the first
 * coarse level) after the last Galerkin rebuild, when desc->coarse_tau > 0
 * (host array of n_cells(level)^d bytes).  Errors: MG_ERR_INVALID (level out
 * of range, n, or coarse compression off). */
mg_status mg_get_coarse_classes(const mg_problem* p, int level, uint8_t* cls, size_t n);

/* Checkpoint of a problem's state (not in the paper; for resuming a solve in
 * another process or after a restart).  The state holds the solution u, the
 * finest level's stored operator chunk by chunk with each chunk's accuracy s
 * (FP64 matrices, or the class bytes, segment bases and class pools of the
 * mixed paths, byte for byte) and, with adaptive accuracy, every cell's final
 * flag and accuracy; coarse operators are rebuilt on import.  A pending FP32
 * correction of the mixed paths is folded into u first.
 * mg_export_state: host_buf NULL => *size receives the bytes needed; else
 *   cap must be at least that and the state is written to host_buf.
 * mg_import_state: p must come from a descriptor with the same dim, n_cells,
 *   path and chunking; replaces its stored operator and u (the problem then
 *   restarts its outer iteration from the imported u).
 * Both wait for the problem's stream and fail with MG_ERR_PENDING while
 * delayed assembly jobs are in flight.  Errors: MG_ERR_INVALID (arguments,
 * cap, a buffer that is not a state of a compatible problem or is truncated),
 * MG_ERR_PENDING, MG_ERR_OOM, MG_ERR_CUDA. */
mg_status mg_export_state(mg_problem* p, void* host_buf, size_t cap, size_t* size);
mg_status mg_import_state(mg_problem* p, const void* host_buf, size_t size);

/* Per-cell storage class (0..3) and cell-centre eps of the finest level; the
 * arrays hold n_cells^d entries; either pointer may be NULL. */
mg_status mg_get_cell_data(const mg_problem* p, uint8_t* cls, double* eps_c, size_t n);

/* Accuracy s of the stored element matrix of every finest-level cell
 * (n_cells^d entries, cell index order): with adapt_C > 0 the level at which
 * the cell became final (or the last one integrated); otherwise the published
 * accuracy of the cell's chunk.  Call after mg_solve or a synchronous
 * mg_assemble_level (integrations still in flight are not reflected).
 * Errors: MG_ERR_INVALID (n). */
mg_status mg_get_cell_accuracy(const mg_problem* p, int32_t* s_out, size_t n);

/* Test hooks on the stored operator of `level` (0 = finest), vectors on the
 * host, (N_level+1)^d FP64 values each, boundary entries ignored/zero:
 *   op = 0: y = A x (Dirichlet rows zero)
 *   op = 1: y = x + omega diag(A)^-1 (b - A x)   (one damped Jacobi sweep)
 *   op = 2: y = b - A x
 * The arithmetic is the level's own (FP32 V-cycle arithmetic for mixed paths
 * on level 0 when `inner` = 1; the FP64 outer arithmetic when inner = 0). */
mg_status mg_apply_level(mg_problem* p, int level, int op, int inner, const double* x,
                         const double* b, double* y);

/* Test hooks on the grid transfers of the V-cycle between `level` and
 * level + 1 (Section "Stencil assembly variants": a sweep fused with the
 * transfer that follows or precedes it), in the level's V-cycle arithmetic
 * (inner as in mg_apply_level).  x, b: host (N_level+1)^d FP64 vectors;
 * c: host (N_level+1+1)^d FP64 vector of level + 1:
 *   op = 0: out (level + 1 size) = R (b - A x), R = P^T the transpose of the
 *           d-linear 3:1 prolongation (c is not read)
 *   op = 1: out (level size) = S(x + P c), S one damped Jacobi sweep with b
 * The level's fused kernels run where it has them (op = 0 on a split
 * compressed 3D finest level), the separate passes elsewhere.  Errors:
 * MG_ERR_INVALID (no level below `level`, null vectors), MG_ERR_CUDA. */
mg_status mg_apply_transfer(mg_problem* p, int level, int op, int inner, const double* x, const double* b,
                            const double* c, double* out);

/* Runs one V-cycle e = V(b) on the finest level from e = 0 with the
 * problem's operators; b and e are host (N+1)^d FP64 vectors. */
mg_status mg_vcycle_apply(mg_problem* p, const double* b, double* e);

/* Times `reps` back-to-back launches of one kernel of the solve on the
 * problem's stream with CUDA events (3 untimed launches first) and returns
 * the mean milliseconds per launch:
 *   which = 0: finest-level damped Jacobi sweep in the V-cycle arithmetic
 *   which = 1: finest-level FP64 matvec of the outer loop (with dot products)
 *   which = 2: finest-level FP64 residual f - A u
 *   which = 3: Galerkin product finest -> next coarser level
 *   which = 4: the element-matrix integration kernel alone (Section
 *              "Numerical computation of stencils") on the first chunk of
 *              the finest level at the last accuracy of the schedule: its
 *              interface cells on piecewise-constant fields, else every cell
 *              of the chunk; outputs go to scratch buffers (the stored
 *              operator is not changed)
 *   which = 5: finest-level residual and restriction b_c = R (b - A u) in the
 *              V-cycle arithmetic (the fused kernels where the level has them)
 *   which = 6: the restriction alone of a finest-level vector
 *   which = 7: one V-cycle of the solve from the finest level (right-hand side
 *              and iterate buffers as they stand)
 *   which = 8: the same from the next coarser level
 *   which = 9: the same from the level below that
 *   which = 10: one inner iteration of the mixed paths (V-cycle and flexible-CG
 *              step, replayed as the solve replays it), back to back
 *   which = 11: the same, each followed by the host's read of the iteration's
 *              scalars as in mg_solve (the difference is the host round trip)
 * The problem's iteration vectors are used as scratch (the next cycle
 * restarts the outer iteration).  Errors: MG_ERR_INVALID, MG_ERR_PENDING
 * (which = 4 while delayed assembly jobs are in flight), MG_ERR_CUDA. */
mg_status mg_profile_kernel(mg_problem* p, int which, int reps, double* ms_per_launch);

/* Measures the throughput of one arithmetic pipe of the current device with
 * kernels of independent dependency chains (a calibration for the pipe
 * fractions this library reports; the paper has no counterpart):
 *   kind = 0: FP32 fused multiply-add, kind = 1: FP64 fused multiply-add,
 *   kind = 2: FP32 exponential (__expf, the special-function unit).
 * *ops_per_s receives the operations per second (one FMA counts as one
 * operation).  Allocates a small device buffer.  Errors: MG_ERR_INVALID,
 * MG_ERR_CUDA. */
mg_status mg_measure_peak(int kind, double* ops_per_s);

/* Test hook for host-side failure injection (the paper has none; Section
 * "Asynchronous and anarchic stencil integration" runs assembly as
 * independent background tasks, and this checks that a failed one is
 * reported): from now on, every side-stream assembly job of accuracy s of
 * this problem's delayed solves ends with MG_ERR_INJECTED on the host, before
 * any device work for that chunk; s = 0 turns it off.  mg_solve then returns
 * MG_ERR_INJECTED at the next cycle boundary and the problem stays valid for
 * mg_destroy_problem.  Errors: MG_ERR_INVALID (null p or s < 0). */
mg_status mg_inject_assembly_failure(mg_problem* p, int s);

/* Number of kernels of this library launched so far in this process
 * (graph replays count every kernel they contain). */
uint64_t mg_launch_count(void);

/* Allocation-free variant of the mixed-precision assembly (the paper has no
 * counterpart: it is an interface for callers that cannot allocate device
 * memory while they run, e.g. a process that plans its whole device
 * footprint up front or an application whose own allocator owns the device,
 * and for which a cudaMalloc would break that plan or synchronise the device).
 * For the cells [cell0, cell0 + ncell) of an n_cells^dim grid (whole x-rows:
 * cell0 and ncell multiples of n_cells) it computes, at accuracy s with the
 * storage rule of tolerance tau (0 => 1e-6), exactly what the mixed paths
 * store: the FP32 cell-centre eps, the storage class (0..3) and the decoded
 * surplus entries (FP32, NP = 6 (2D) / 28 (3D) per cell, pair order a < b;
 * zeros for class 0).  All pointers are caller-owned DEVICE buffers:
 * eps_c_out holds n_cells^dim floats (the whole grid is written), cls_out
 * ncell bytes, surplus_out ncell * NP floats.  Work is issued on cuda_stream
 * (NULL = legacy default stream); the call returns without synchronising.
 * Scratch: a fixed 64 MiB (67,108,864-byte) device array inside the library.
 * One call needs ncell * REC_MAX record bytes (REC_MAX = 112 in 3D, 32 in
 * 2D) rounded up to a multiple of 256, plus rows * ceil(n_cells/32) * 32
 * padded class bytes (rows = ncell / n_cells), and the sum must not exceed
 * 64 MiB: at n_cells = 243 that is at most 2,442 x-rows (593,406 cells) in
 * 3D.  The eps descriptor is checked as at problem creation.  Larger ranges
 * and bad descriptors return MG_ERR_INVALID with the reason in
 * mg_last_error().  The array is shared by every call on a device and keeps
 * the last call's contents, so calls that overlap on the GPU (different
 * streams, or host threads) race and must be serialised by the caller.  The
 * first call on a device looks up the array's device address (once per
 * device, with that device current): make that first call before any stream
 * capture.  Allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine).  Errors: MG_ERR_INVALID, MG_ERR_CUDA. */
mg_status mg_assemble_surplus_noalloc(const mg_eps_desc* eps, int dim, int n_cells, int s, double tau,
                                      int64_t cell0, int64_t ncell, float* eps_c_out, uint8_t* cls_out,
                                      float* surplus_out, void* cuda_stream);

/* ---------------- serving ---------------- */

typedef struct {
  int32_t max_active;       /* concurrent solves on the GPU (0 => 8) */
  int32_t use_graphs;       /* nonzero: each request replays its outer iteration as a
                               captured CUDA graph (one graph per request and iteration
                               kind); 0: kernel by kernel */
  double hbm_budget_bytes;  /* admission budget (0 => free HBM at creation minus 4 GiB) */
  int32_t inject_fail_every;/* tests: fail every k-th admission on the host (0 = off) */
  int32_t pad0;
} mg_server_desc;

typedef struct {
  int32_t status;           /* MG_OK when solved; error status otherwise */
  int32_t cycles;
  int32_t publishes;
  int32_t pad0;
  double rel_residual;
  double queue_ms;          /* submit -> admission */
  double solve_ms;          /* admission -> done */
  double total_ms;          /* submit -> done (time to solution) */
} mg_result;

typedef struct mg_server mg_server;

/* Starts a server thread that admits submitted problems while the HBM
 * budget and max_active allow, runs their delayed-assembly solves
 * concurrently on separate streams and records per-request results. */
mg_status mg_server_create(const mg_server_desc* desc, mg_server** out);

/* Queues a problem.  solution_dst (optional, (N+1)^d doubles, caller-owned)
 * receives u when the request finishes; it must stay valid until mg_poll
 * returns a final status.  ticket receives the request id. */
mg_status mg_submit(mg_server* s, const mg_problem_desc* desc, double* solution_dst,
                    uint64_t* ticket);

/* MG_ERR_PENDING until the request finishes, then its final status; result
 * (optional) is filled once finished. */
mg_status mg_poll(mg_server* s, uint64_t ticket, mg_result* result);

/* Blocks until every submitted request has finished or timeout_ms elapsed
 * (MG_ERR_TIMEOUT). */
mg_status mg_server_drain(mg_server* s, double timeout_ms);

/* Cancels queued requests, waits for running ones, frees everything. */
mg_status mg_server_destroy(mg_server* s);

/* Thread-local message of the last error on this thread ("" if none). */
const char* mg_last_error(void);

/* Library version string. */
const char* mg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MG_H */
