/*
 * taps.h -- C ABI of the GB300 (sm_103a) TAPS hot path.
 *
 * TAPS (Tensor-decomposition-based A Priori Surrogate) solves a space-parameter-time
 * PDE in CP form u(x) = sum_m prod_d sum_I N~_I(x_d) U_d[I, m] (Eq. 13) by Galerkin
 * projection (Eq. 25) onto 1D C-HiDeNN shape functions (Eq. 1) and the subspace
 * iteration of Algorithm 1 (Eq. 43).  This library runs every step on one GPU:
 * 1D assembly, the per-dimension Gram contractions, the coefficient (Hadamard)
 * combine, the n_d*M block-banded reduced solve, normalisation, residuals and
 * reconstruction.
 *
 * Conventions used by every entry point
 *   - All functions return an int status: TAPS_OK (0) or a negative TAPS_ERR_*.
 *     No entry point aborts or traps; device-side failures (zero pivot, non-finite
 *     value, a bounded wait that ran out) are reported through the status.
 *   - Host pointers are read during the call only; the caller keeps ownership.
 *   - Objects (taps_dim, taps_problem, taps_factors) are opaque, library-owned and
 *     device-resident until their *_destroy call.  They are bound to the CUDA device
 *     that was current at creation and to the stream given at creation; every
 *     kernel of an object is launched on that stream.  Calls are synchronous with
 *     respect to the host unless stated otherwise.
 *   - Factor matrices U_d are n_free(d) x M, column-major (mode m is contiguous),
 *     FP64, free nodes only (Dirichlet / zero-initial-condition nodes are dropped:
 *     the Kronecker delta of Eq. 3 makes their value the boundary value, here 0).
 *   - Band storage of a 1D matrix over the free nodes: row-major n_free x (2*hb+1),
 *     entry (i, k) holds Op[i, i + k - hb], zero where the column is not a free node;
 *     hb = 2*s + 1 (shape functions of nodes more than 2s+1 apart share no element).
 */
#ifndef TAPS_H
#define TAPS_H

#ifdef __cplusplus
extern "C" {
#endif

#define TAPS_MAX_DIMS 8
#define TAPS_MAX_S 4       /* patch size s <= 4 */
#define TAPS_MAX_P 3       /* reproducing order p <= 3 */
#define TAPS_MAX_QUAD 12   /* Gauss points per element */
#define TAPS_MAX_M 128     /* modes per factor */
#define TAPS_MAX_TERMS 128    /* operator terms R */
#define TAPS_MAX_SOURCES 4096 /* source terms R_f (slab chaining adds M per term and slab) */

/* ---- status codes ---------------------------------------------------------- */
#define TAPS_OK 0
#define TAPS_ERR_INVALID_ARG (-1)   /* bad size, kind, pointer, or a patch with < p+1 nodes */
#define TAPS_ERR_SINGULAR (-2)      /* zero / non-finite pivot in a reduced or patch solve */
#define TAPS_ERR_NONFINITE (-3)     /* NaN or Inf in a result */
#define TAPS_ERR_NOT_CONVERGED (-4) /* tolerance not met in the allowed sweeps (result kept) */
#define TAPS_ERR_TIMEOUT (-5)       /* a bounded device-side wait ran out */
#define TAPS_ERR_CUDA (-6)          /* a CUDA runtime call failed */
#define TAPS_ERR_OOM (-7)           /* device allocation failed */
#define TAPS_ERR_SCRATCH_LIMIT (-8) /* request larger than the fixed scratch of taps_eval_grid_noalloc */

/* ---- dimension kinds (Eq. 11: spatial, parametric, temporal variables) ------ */
#define TAPS_SPACE 0
#define TAPS_PARAM 1
#define TAPS_TIME 2

/* ---- 1D operator kinds (Sec. 2.5, Eqs. 31-35) -------------------------------- */
#define TAPS_OP_K 0    /* stiffness      K_ij = int B~_i B~_j                          */
#define TAPS_OP_M 1    /* mass           M_ij = int N~_i N~_j                          */
#define TAPS_OP_G 2    /* time deriv.    G_ij = int N~_i B~_j   (test i, trial j)      */
#define TAPS_OP_W 3    /* weighted mass  W_ij = int N~_i w(x) N~_j, w = weight_poly    */
#define TAPS_OP_BLO 4  /* point mass at the low end  (convection face, Eqs. 21/25)     */
#define TAPS_OP_BHI 5  /* point mass at the high end                                   */
#define TAPS_NUM_OPS 6
/* Weighted operators (App. A: coefficients that depend on the solution, kept in the
 * separated form, weight every 1D integral by one mode's C-HiDeNN field
 * w(x) = sum_k N~_k(x) w_k): op code TAPS_OP_WEIGHTED + j in a term names weighted
 * operator j of that dim, defined by taps_problem_set_weighted_ops.  Bases:
 *   TAPS_OP_K:  int w B~_i B~_j      TAPS_OP_M:  int w N~_i N~_j
 *   TAPS_OP_G:  int N~_i d/dt (w N~_j) = int N~_i (w' N~_j + w B~_j)
 * A dim with weighted operators is solved by block elimination. */
#define TAPS_OP_WEIGHTED 16
#define TAPS_MAX_WEIGHTED 64   /* weighted operators per dim */
#define TAPS_MAX_SLOTS 72      /* distinct operators (plain and weighted) per dim */

/* ---- source factor kinds g(x) of a separable source term -------------------- */
#define TAPS_SRC_CONST 0  /* par[0]                                       */
#define TAPS_SRC_SIN 1    /* sin(par[0] * x + par[1])                     */
#define TAPS_SRC_GAUSS 2  /* exp(-(x - par[0])^2 / (2 par[1]^2))          */
#define TAPS_SRC_POLY 3   /* par[0] + par[1] x + par[2] x^2 + par[3] x^3  */
#define TAPS_SRC_NODAL 4  /* C-HiDeNN interpolant of nodal values (all nodes) */
#define TAPS_SRC_OPVEC 5  /* q = Op v over the free nodes: par[0] = operator kind, nodal = v
                             (n_free values); the projection of a field already in the
                             C-HiDeNN space, e.g. the end state of a previous time slab */
#define TAPS_SRC_OPVEC_FULL 6 /* q = (Op v)[free nodes] with v given at ALL nodes (constrained
                                 ones included): the lifting of non-homogeneous Dirichlet
                                 data; par[0] = operator kind, nodal = v (n values) */

/* ---- precisions of the Gram / SpMM contractions (reduced solves stay FP64) --- */
#define TAPS_FP64 0
#define TAPS_FP32 1   /* FP32 Gram / SpMM contractions; FP64 solves and residuals */
#define TAPS_MIXED 2  /* FP64 Grams; the n small M x M systems of the fast-diagonalisation
                         solve factorised in FP32 and refined in FP64 to FP64 backward
                         accuracy (FP64 LU fallback per system) */
#define TAPS_BF16 3   /* Gram / SpMM contractions on BF16-rounded operands (factors, bands,
                         source vectors) with FP32 accumulation; FP64 solves and residuals;
                         handled by taps_solve like TAPS_FP32 (guard, FP64 polish) */

/* ---- residual kinds ----------------------------------------------------------- */
#define TAPS_RES_ALS 0   /* max_d ||K^[d] U_d - Q^[d]|| / ||Q^[d]|| of Eq. 42           */
#define TAPS_RES_FULL 1  /* ||F - A u||_2 / ||F||_2 over the free tensor-grid unknowns   */

/* ---- initialisation of factor columns ---------------------------------------- */
#define TAPS_INIT_GIVEN 0   /* start from the factors as they are (taps_factors_set) */
#define TAPS_INIT_RANDOM 1  /* U(-1,1), SplitMix64 counter-based draws (seed, d, i, m) */
#define TAPS_INIT_ZERO 2    /* new column: 0 in the first dim, 1 elsewhere            */

/* ---- reduced solvers ---------------------------------------------------------- */
#define TAPS_SOLVER_BLOCK_LU 0   /* block-banded Gaussian elimination, FP64 */
#define TAPS_SOLVER_FASTDIAG 1   /* fast diagonalisation (Sec. 2.6) for every dimension whose
                                    operators form a symmetric pencil with a mass-like partner
                                    (K/M, W, ...: n_d x n_d pencil, n_d small M x M solves);
                                    else, for a dimension with two operators whose coefficient
                                    matrices are symmetric (every other dimension's operators
                                    symmetric, e.g. the time dimension of a transient problem)
                                    and M <= 32, diagonalisation on the mode side (M x M
                                    pencil, M banded n_d x n_d solves); block LU otherwise */
#define TAPS_SOLVER_MODEDIAG 2   /* diagonalisation on the mode side wherever it applies (one or
                                    two operators, symmetric coefficients, M <= 32, band
                                    half-width <= 5): no n_d x n_d decomposition, cost
                                    O(M^3 + M^2 n_d + banded solves) per dimension; else as
                                    TAPS_SOLVER_FASTDIAG */
#define TAPS_SOLVER_AUTO 3       /* batches only: the first graph sweep times one sweep of the
                                    batch with FASTDIAG and with MODEDIAG (factors restored)
                                    and keeps the faster */

typedef struct taps_dim taps_dim;
typedef struct taps_problem taps_problem;
typedef struct taps_factors taps_factors;

/* One independent dimension (Eq. 11) on n uniform nodes over [lo, hi] with
 * C-HiDeNN hyperparameters s (patch size), a (dilation), p (reproducing order)
 * of Eq. 1, n_quad Gauss points per element (Table 1: Gaussian integration).
 * dirichlet_lo/hi = 1 drops that end node (homogeneous Dirichlet, or the zero
 * initial condition of a time dimension).  weight_poly gives w(x) of TAPS_OP_W. */
typedef struct {
  int kind;
  int n;
  double lo, hi;
  int s;
  double a;
  int p;
  int n_quad;
  int dirichlet_lo, dirichlet_hi;
  double weight_poly[4];
} taps_dim_desc;

/* One operator term alpha * (x)_d Op_d of A (the separated integrals of Eq. 33). */
typedef struct {
  double alpha;
  int op[TAPS_MAX_DIMS];
} taps_term;

/* One separable source term beta * (x)_d g_d; q_{r,d} = int N~ g_d (Eq. 30 forcing). */
typedef struct {
  double beta;
  int kind[TAPS_MAX_DIMS];
  double par[TAPS_MAX_DIMS][4];
  const double* nodal[TAPS_MAX_DIMS]; /* TAPS_SRC_NODAL: host array of n values;
                                         TAPS_SRC_OPVEC: host array of n_free values;
                                         TAPS_SRC_OPVEC_FULL: host array of n values */
} taps_source;

typedef struct {
  int precision;     /* TAPS_FP64 | TAPS_FP32 (Gram and SpMM contractions) */
  int solver;        /* TAPS_SOLVER_* */
  int normalize;     /* 1: unit-norm columns for d < D after each solve (default 1) */
} taps_sweep_opts;

typedef struct {
  int sweeps;          /* sweeps performed */
  double change;       /* max_d ||U_d^new - U_d^old||_F / ||U_d^new||_F of the last sweep */
  double seconds;      /* wall time of the call */
} taps_sweep_report;

typedef struct {
  int M0, M_max;       /* first and last mode count of the greedy schedule */
  double als_tol;      /* per-M stop on the factor change (Sec. 2.6 convergence check) */
  double res_tol;      /* stop once the residual of kind res_kind is <= res_tol */
  int res_kind;        /* TAPS_RES_* */
  int max_sweeps;      /* per mode count */
  int precision;       /* TAPS_FP64 | TAPS_FP32 for the sweeps */
  int polish_sweeps;   /* FP64 sweeps allowed after an FP32 phase stalls (refinement) */
  int solver;          /* TAPS_SOLVER_* */
  int init;            /* TAPS_INIT_* for the columns added by the schedule */
  unsigned seed;       /* seed of TAPS_INIT_RANDOM */
  int history_cap;     /* capacity of the report's history arrays (0: none) */
  int graphs;          /* 0: direct launches.  1: replay each sweep + residual as a
                          captured CUDA graph (captured on first use per factors / M /
                          precision / solver; falls back to direct launches if capture
                          is unavailable).  2: run the whole sweep loop of each M on the
                          device, one graph whose conditional WHILE node repeats sweep,
                          residual and the stopping test (FP64 / MIXED with the Eq. 42
                          residual and profiling events off; otherwise as 1); the same
                          sweeps and factors as 1, without a host round trip per sweep */
  double res_stall;    /* greedy stop on stagnation: growth ends once the residual (kind
                          res_kind) at the end of a mode count exceeds (1 - res_stall) times
                          its value at the end of the previous mode count, two mode counts
                          in a row (0: off) */
  int M_step;          /* modes appended per growth step of the greedy schedule (0 or 1: one) */
} taps_solve_opts;

typedef struct {
  int M;               /* final mode count */
  int sweeps;          /* total sweeps */
  int fp64_sweeps;     /* of which FP64 */
  double rho;          /* final residual of kind res_kind */
  double rho_full;     /* final ||F - A u|| / ||F|| */
  double change;       /* last factor change */
  double seconds;      /* wall time of the solve */
  int converged;       /* 1 if rho <= res_tol */
  /* optional per-sweep history, caller-owned host arrays of history_cap entries */
  int* hist_M;
  double* hist_change;
  double* hist_rho;
  int hist_len;
} taps_solve_report;

/* ---- status ------------------------------------------------------------------- */
const char* taps_status_string(int status);
int taps_version(void);

/* ---- 1D assembly (Eq. 1 shape functions; Eqs. 31-35 matrices; Table 1 quadrature)
 * Builds, on the device, the C-HiDeNN patch inverses of every node, the shape
 * function tables at the Gauss points of every element and the banded matrices of
 * all TAPS_NUM_OPS kinds over the free nodes.  `stream` is a cudaStream_t (NULL:
 * legacy default stream).  Errors: TAPS_ERR_INVALID_ARG for n < 2, s > TAPS_MAX_S,
 * p > TAPS_MAX_P, n_quad outside [1, TAPS_MAX_QUAD], hi <= lo, or an end patch with
 * fewer than p+1 nodes; TAPS_ERR_SINGULAR if a patch moment matrix is singular. */
int taps_assemble_1d(const taps_dim_desc* desc, void* stream, taps_dim** out);
/* Sizes of an assembled dimension: all nodes, free nodes, band half-width hb. */
int taps_dim_info(const taps_dim* dim, int* n_all, int* n_free, int* half_band);
/* Copy the band of operator `op` (n_free x (2hb+1), row-major, FP64) to host memory. */
int taps_dim_copy_band(const taps_dim* dim, int op, double* host_out);
/* Copy the shape tables (Eq. 1) to host memory: N and dN/dx at every Gauss point of
 * every element, layout [n-1][n_quad][2s+2] with local node k <-> global e - s + k
 * (entries of nodes outside [0, n) are 0), plus the Gauss abscissae x [n-1][n_quad]. */
int taps_dim_copy_shape(const taps_dim* dim, double* N_out, double* B_out, double* x_out);
void taps_dim_destroy(taps_dim* dim);

/* ---- problem: A = sum_t alpha_t (x)_d Op[t][d], F = sum_r beta_r (x)_d q_{r,d}
 * (the separated Galerkin operator and force of Eqs. 33-41).  `dims` are assembled
 * dimensions (the problem keeps pointers: they must outlive it).  Source projections
 * q_{r,d} are computed on the device.  Errors: TAPS_ERR_INVALID_ARG for D outside
 * [1, TAPS_MAX_DIMS], R outside [1, TAPS_MAX_TERMS], Rf outside [1, TAPS_MAX_SOURCES], an operator or source kind
 * out of range (operators: the plain kinds and TAPS_OP_WEIGHTED + j, j < TAPS_MAX_WEIGHTED;
 * at most TAPS_MAX_SLOTS distinct ones per dim), or a NULL nodal array. */
int taps_problem_create(taps_dim* const* dims, int D, const taps_term* terms, int R,
                        const taps_source* sources, int Rf, void* stream,
                        taps_problem** out);
/* Define or update weighted operators 0..count-1 of dim `dim` (op codes
 * TAPS_OP_WEIGHTED + j): base[j] is TAPS_OP_K, TAPS_OP_M or TAPS_OP_G and
 * weights + j * n_d holds the nodal values of its weight at ALL n_d nodes of the dim
 * (host memory, FP64, row j per operator).  The bands of those operators that the
 * problem's terms use are assembled on the device (restricted to the free nodes);
 * the next sweep or solve refreshes the Gram matrices.  Every weighted operator a
 * term uses must be defined before the first sweep (else TAPS_ERR_INVALID_ARG).
 * Errors: TAPS_ERR_INVALID_ARG for a bad dim, count outside [1, TAPS_MAX_WEIGHTED],
 * a NULL array or a base other than K, M, G. */
int taps_problem_set_weighted_ops(taps_problem* prob, int dim, int count, const int* base,
                                  const double* weights);
/* Copy the band of operator `op` (a plain kind or TAPS_OP_WEIGHTED + j) of dim `dim`
 * as the problem's terms use it: [n_free][2 hb + 1] FP64 values, row i holding
 * entries (i, i + k - hb) over the free nodes, to host memory.  TAPS_ERR_INVALID_ARG if
 * no term uses `op` in that dim. */
int taps_problem_copy_op(const taps_problem* prob, int dim, int op, double* host_out);
/* Copy q_{r,d} (n_free(d) FP64 values) to host memory. */
int taps_problem_copy_source(const taps_problem* prob, int r, int d, double* host_out);
/* Recompute every dim's Gram matrices (Eq. 34) from the factors U at `precision`
 * (TAPS_FP64, TAPS_FP32: CUDA cores; TAPS_BF16: tensor cores where the dim allows, see
 * taps_batch_refresh_grams).  Synchronous. */
int taps_problem_refresh_grams(taps_problem* prob, const taps_factors* U, int precision);
/* Copy the current Grams of dim d for mode count M: gram_out [nops][M][M] row-major,
 * Gamma_o[m][n] = U[:, m]^T Op_o U[:, n], one per distinct operator of the dim in slot
 * order (ops_out receives their op codes, nops_out their count); h_out [R_f][M].  Any
 * output pointer may be NULL.  M must not exceed the problem's workspace (the largest M
 * swept or refreshed). */
int taps_problem_copy_grams(const taps_problem* prob, int d, int M, double* gram_out, double* h_out, int* ops_out,
                            int* nops_out);
void taps_problem_destroy(taps_problem* prob);

/* ---- factors: D device matrices U_d (n_free(d) x M, column-major, FP64; Eq. 7) --- */
int taps_factors_create(const taps_problem* prob, int M_cap, taps_factors** out);
/* Set M (<= M_cap) and copy host_U[d] (n_free(d) x M column-major) to the device. */
int taps_factors_set(taps_factors* U, int M, const double* const* host_U);
/* Copy the current factors to host_U[d] (n_free(d) x M column-major each). */
int taps_factors_get(const taps_factors* U, double* const* host_U);
/* Copy the factors of src into dst (same problem, on the device); dst takes src's mode
 * count.  TAPS_ERR_INVALID_ARG if the problems differ or src's modes exceed dst's
 * capacity. */
int taps_factors_copy(taps_factors* dst, const taps_factors* src);
/* |u_A - u_B| / |u_A| for the CP tensors of two factor sets of the same problem (the
 * Euclidean norm of the nodal values on the free nodes), on the device: the
 * convergence check of the global-local iteration (App. A).  The difference is
 * evaluated as a CP tensor of D * max(M_A, M_B) telescoped terms (per mode,
 * prod a_d - prod b_d = sum_k prod_{d<k} b_d (a_k - b_k) prod_{d>k} a_d, the shorter set
 * padded with zero columns) through 1D Gram products, so small changes keep their
 * relative accuracy (no |a|^2 + |b|^2 - 2<a, b> cancellation).  0 when u_A = 0 and for
 * identical factor sets. */
int taps_factors_rel_change(const taps_factors* A, const taps_factors* B, double* out);
int taps_factors_M(const taps_factors* U);
/* Device pointer of U_d (n_free(d) x M_cap storage, leading dimension n_free(d)). */
const double* taps_factors_device_ptr(const taps_factors* U, int d);
void taps_factors_destroy(taps_factors* U);

/* ---- sweeps (Algorithm 1 inner loop, Eq. 43) ------------------------------------
 * Runs n_sweeps sweeps over d = 1..D: coefficient matrices C_op = Hadamard products
 * of the other dimensions' Grams U_e^T Op U_e (Eq. 34/35), force F_d, block-banded
 * reduced solve sum_op Op_d U_d C_op^T = F_d, normalisation of U_d (d < D), Gram
 * refresh of dim d.  opts may be NULL (FP64, block LU, normalise).  Errors:
 * TAPS_ERR_SINGULAR (zero or non-finite pivot; factors then undefined),
 * TAPS_ERR_TIMEOUT, TAPS_ERR_CUDA. */
int taps_sweep(taps_problem* prob, taps_factors* U, int n_sweeps, const taps_sweep_opts* opts,
               taps_sweep_report* rep);

/* ---- residuals (FP64) ---------------------------------------------------------
 * kind TAPS_RES_ALS: max over d of ||sum_op Op_d U_d C_op^T - F_d||_F / ||F_d||_F
 * with all factors at their current values (the residual of the coupled system
 * Eq. 42).  kind TAPS_RES_FULL: ||F - A u||_2 / ||F||_2 by the Gram identity
 * ||F||^2 - 2 F^T A u + ||A u||^2, each a sum of products of 1D inner products
 * (cancellation limits it to about 1e-8 relative). */
int taps_residual(taps_problem* prob, const taps_factors* U, int kind, double* rho_out);

/* ---- solve: greedy mode schedule M0..M_max with sweeps to tolerance ----------------
 * For each M: sweep until rho (kind res_kind) <= res_tol or the factor change <=
 * als_tol or max_sweeps; then stop if rho <= res_tol (or, with res_stall > 0, once rho
 * has stagnated over two mode counts), else append M_step columns per factor (init
 * rule, at most up to M_max) and continue.  With precision TAPS_FP32 the sweeps use FP32
 * Grams; once the FP32 sweeps stop improving, up to polish_sweeps FP64 sweeps
 * refine the result to FP64 accuracy.  U must have M_cap >= M_max; with init
 * TAPS_INIT_GIVEN its current M columns are the start (M0 is then ignored), else it
 * is reset to M0 columns drawn by the init rule.  Returns TAPS_ERR_NOT_CONVERGED if
 * the tolerance is not met (factors and report are still valid). */
int taps_solve(taps_problem* prob, taps_factors* U, const taps_solve_opts* opts,
               taps_solve_report* rep);

/* ---- evaluation (Eq. 13) -------------------------------------------------------
 * Grid: u on the tensor grid of node slices idx_d = start[d] + step[d] * j,
 * j < count[d] (all-node numbering; constrained nodes are 0).  out_dev is caller-
 * owned device memory of prod count[d] values, C order (last dim fastest), dtype
 * out_dtype (TAPS_FP64: double, TAPS_FP32: float).  Asynchronous on the problem's
 * stream.  Errors: TAPS_ERR_INVALID_ARG for an index outside [0, n). */
int taps_eval_grid(const taps_problem* prob, const taps_factors* U, const int* start,
                   const int* count, const int* step, void* out_dev, int out_dtype);
/* Allocation-free variant of taps_eval_grid (the paper has no counterpart: this is a
 * service for callers of this library).  Same arguments, same values (up to the
 * order of the FP sums) and the same C-order output, but it allocates nothing: no
 * cudaMalloc, no cudaFree, no allocating library routine.  It is meant for callers
 * that cannot allocate device memory when they need a field -- code that runs
 * under a fixed, fully reserved memory budget, or inside a host framework whose hot
 * path forbids allocation and the synchronisation an allocation may imply.  Its
 * working memory (the gathered factor rows, sum_d count[d] * M values of the
 * output type) lives in one fixed array of TAPS_NOALLOC_SCRATCH_BYTES in device
 * global memory, which every GPU that loads this library holds until the process
 * exits.  Requests that need more return TAPS_ERR_SCRATCH_LIMIT and touch nothing.
 * Every call looks up that array's device address with the calling device current
 * (no allocation; nothing cached, so a reset primary context is safe); the first
 * lookup on a device may load the library's device code, so make the first call on
 * each device before any stream capture.  Every call on a device shares the one array and it keeps the last
 * call's contents (each call overwrites all it reads, so nothing needs clearing);
 * calls whose kernels overlap on the GPU -- on different streams, or different
 * problems launched concurrently -- race on it and must be serialised by the
 * caller.  Asynchronous on the problem's stream. */
#define TAPS_NOALLOC_SCRATCH_BYTES (4u << 20)
int taps_eval_grid_noalloc(const taps_problem* prob, const taps_factors* U, const int* start,
                           const int* count, const int* step, void* out_dev, int out_dtype);
/* Points: u^TD(x) = sum_m prod_d sum_I N~_I(x_d) U_d[I, m] at n_pts points; pts_dev is
 * device memory [n_pts][D] row-major (coordinates clamped to [lo, hi]); out_dev
 * receives n_pts FP64 values.  Asynchronous on the problem's stream. */
int taps_eval_points(const taps_problem* prob, const taps_factors* U, int n_pts,
                     const double* pts_dev, double* out_dev);

/* ---- batched independent instances ------------------------------------------------
 * A batch holds `count` (problem, factors) pairs -- distinct problems, each created on
 * its own stream -- and sweeps them together (Algorithm 1 inner loop per instance).
 * With graphs = 1, one sweep of every instance is captured once as one CUDA graph
 * (instances on their own streams, forked from and joined to the batch's stream)
 * and replayed n_sweeps times; otherwise each instance runs its own launch sequence
 * in turn.  Every instance's Grams are first recomputed from its current factors.
 * changes_out (count values, optional) receives each instance's factor change of its
 * last sweep.  status_out (count values, optional) receives each instance's status
 * (the first numerical error of its sweeps, e.g. TAPS_ERR_SINGULAR when fixed-M sweeps
 * have made its factors numerically rank deficient); every instance runs all
 * n_sweeps regardless, and with status_out given the call returns TAPS_OK unless a
 * launch fails.  Without status_out the first instance error is returned.  The
 * pointers must outlive the batch.  Errors as taps_sweep, TAPS_ERR_INVALID_ARG for a
 * shared problem or empty factors.  Pencil decompositions are made at creation, in
 * waves of instances whose kernels run concurrently on the instances' streams. */
typedef struct taps_batch taps_batch;
int taps_batch_create(taps_problem* const* probs, taps_factors* const* Us, int count, int precision,
                      int solver, taps_batch** out);
int taps_batch_sweep(taps_batch* batch, int n_sweeps, int graphs, double* changes_out, int* status_out);
/* The solver a batch's sweeps use (for TAPS_SOLVER_AUTO the tuner's choice, made by the
 * first graph sweep) and the tuner's two trial times in ms (FASTDIAG, MODEDIAG; -1
 * before tuning or without AUTO).  Either pointer may be NULL. */
int taps_batch_info(const taps_batch* batch, int* solver_out, float* trial_ms_out);
/* Recompute the Gram matrices Gamma_{o,d} = U_d^T Op_{o,d} U_d and h_{r,d} = U_d^T q_{r,d}
 * (Eq. 34) of every dim of every instance from the current factors, all instances at
 * once (the SpMM + Gram refresh of Algorithm 1, batched).  precision TAPS_BF16: one
 * persistent launch on the tensor cores (tcgen05, factors, bands and source vectors
 * rounded to bfloat16, the banded product kept to ~16 bits as two bfloat16 parts, FP32
 * accumulation in tensor memory); CTAs pull (instance, dim) items from a device queue,
 * largest first.  The first such call times the chunk height (64 or 128 nodes) and the
 * CTAs per SM (1 to 4) on the batch and keeps the fastest (taps_batch_gram_info).
 * Every item needs M <= 64, R_f <= 64 and at most 4 distinct operators, else
 * TAPS_ERR_INVALID_ARG.  precision TAPS_FP64: each instance's FP64 refresh on its own
 * stream.  The batch's sweeps keep their own precision; this call replaces the
 * instances' Grams until the next sweep recomputes them.  ms_out (optional): device time
 * of the refresh (CUDA events on the batch's stream, the queue set-up excluded);
 * bytes_out (optional): its algorithmic bytes (FP64 factors, bands and source vectors
 * read once, Grams written).  Synchronous. */
int taps_batch_refresh_grams(taps_batch* batch, int precision, float* ms_out, double* bytes_out);
/* The tuner's choice of taps_batch_refresh_grams (chunk rows, CTAs per SM; 0 before the
 * first BF16 call) and its 6 trial times in ms for (rows, CTAs per SM) = (64, 1), (64, 2),
 * (64, 3), (64, 4), (128, 1), (128, 2) (-1 where the shared memory or TMEM does not allow
 * the occupancy).  Pointers may be NULL. */
int taps_batch_gram_info(const taps_batch* batch, int* rows_out, int* ctas_per_sm_out, float* table_ms_out);
void taps_batch_destroy(taps_batch* batch);

/* ---- learned warm start (the paper's Algorithm 1 starts from random values) ------
 * A fully connected FP32 network n_in -> H (x hidden_layers, tanh) -> n_out (linear)
 * with hand-written forward, backward (mean squared error) and Adam kernels.  It maps
 * an instance's parameter vector and a mode index to that mode's factor profiles;
 * taps_factors_from_profiles turns predictions into initial factors.  Parameters are
 * one flat FP32 array: per layer W [out][in] row-major, then b [out].  Weights start
 * Xavier-uniform from SplitMix64 draws of `seed`.  All device pointers are
 * caller-owned; calls run on `stream` (taps_mlp_train and the _get/_set calls
 * synchronise it). */
#define TAPS_MLP_MAX_LAYERS 8
typedef struct taps_mlp taps_mlp;
int taps_mlp_create(int n_in, int n_hidden, int hidden_layers, int n_out, unsigned seed, void* stream,
                    taps_mlp** out);
long long taps_mlp_num_params(const taps_mlp* net);
int taps_mlp_get_params(const taps_mlp* net, float* host, long long n);
int taps_mlp_set_params(taps_mlp* net, const float* host, long long n);  /* also resets Adam */
/* y_dev[batch][n_out] = net(x_dev[batch][n_in]) */
int taps_mlp_forward(taps_mlp* net, const float* x_dev, int batch, float* y_dev);
/* loss = mean (net(x) - t)^2 over batch x n_out; parameter gradients kept on the device
 * (and copied to grad_host, nparams floats, when it is not NULL). */
int taps_mlp_grad(taps_mlp* net, const float* x_dev, const float* t_dev, int batch, float* loss_out,
                  float* grad_host);
/* one Adam step with the last gradients (bias-corrected moments) */
int taps_mlp_adam(taps_mlp* net, float lr, float beta1, float beta2, float eps);
/* `steps` full-batch gradient + Adam(0.9, 0.999, 1e-8) steps; loss of the last step */
int taps_mlp_train(taps_mlp* net, const float* x_dev, const float* t_dev, int batch, int steps, float lr,
                   float* loss_out);
void taps_mlp_destroy(taps_mlp* net);
/* Initial factors from predicted profiles: prof_dev [M][D * n_ref + 1] (FP32), per
 * dim d a profile at n_ref uniform points of [lo_d, hi_d] (all-node coordinates),
 * then the mode weight.  U_d[:, m] = the profile interpolated linearly at the free
 * nodes; the last dim is multiplied by weight_scale * weight.  Sets the factors' M. */
int taps_factors_from_profiles(const taps_problem* prob, taps_factors* U, int M, const float* prof_dev,
                               int n_ref, double weight_scale);

/* ---- profiling: per kernel class, CUDA events on the problem's stream ----------
 * taps_profile_reset clears the counters; with enable_events = 1 every launch of a
 * class is bracketed by CUDA events (read back at the library's own stream
 * synchronisation points).  Launch counts are kept whether or not events are on.
 * taps_profile_get returns, for one class, the launches, the summed device time in
 * milliseconds (events only) and the algorithmic FP64/FP32 flops and DRAM bytes the
 * launches were charged with (the roofline numerators). */
#define TAPS_PROF_GRAM 0          /* fused banded SpMM + Gram (partial + reduce)   */
#define TAPS_PROF_COEFF 1         /* Hadamard coefficient combine                   */
#define TAPS_PROF_BLOCK_ASSEMBLE 2 /* reduced block band + right-hand side          */
#define TAPS_PROF_BLOCK_LU 3      /* cooperative block-banded elimination           */
#define TAPS_PROF_BACKSUB 4       /* block back substitution                        */
#define TAPS_PROF_NORMALIZE 5     /* column normalisation + factor change           */
#define TAPS_PROF_RESIDUAL 6      /* residual kernels                               */
#define TAPS_PROF_EVAL 7          /* grid reconstruction                            */
#define TAPS_PROF_OTHER 8         /* initialisation, pencil set-up, copies           */
#define TAPS_PROF_FASTDIAG 9      /* fast diagonalisation: the n small M x M solves  */
#define TAPS_PROF_FD_TRANSFORM 10 /* fast diagonalisation: back to the nodal basis   */
#define TAPS_PROF_MODEDIAG 11     /* mode-side diagonalisation: M x M eigenproblem,
                                     banded solves, transform                       */
#define TAPS_PROF_NUM 12
int taps_profile_reset(taps_problem* prob, int enable_events);
int taps_profile_get(taps_problem* prob, int kernel_class, long long* launches, double* ms,
                     double* flops, double* bytes);

/* The library's bounded device-side grid barrier, for testing failure detection
 * without a GPU fault: `ctas` CTAs (1..64) meet twice at a barrier that expects
 * ctas + missing arrivals (missing 0..64), each wait bounded by poll_limit polls
 * (1..2^26).  Returns TAPS_OK when missing = 0; with missing > 0 every wait runs out,
 * the kernel records the timeout and returns, and the call returns TAPS_ERR_TIMEOUT
 * with the CUDA context intact.  `stream` is a cudaStream_t (NULL: legacy stream). */
int taps_util_barrier_test(int ctas, int missing, long long poll_limit, void* stream);

/* ---- the FP64 reciprocal of the small reduced solves (no counterpart in the method;
 * exposed so that its accuracy can be checked against IEEE division) ---------------
 * y[i] = 1 / x[i] for n device doubles, from the hardware's approximate reciprocal
 * refined by one step of the series 1/x = y0 (1 + e + e^2), e = 1 - x y0; within one
 * unit in the last place of 1.0 / x for normal x whose reciprocal is normal.  x_dev and
 * y_dev are device pointers (they may alias); stream is a cudaStream_t or NULL.
 * Asynchronous; TAPS_ERR_INVALID_ARG for n < 0 or null pointers with n > 0. */
int taps_util_rcp(const double* x_dev, double* y_dev, long long n, void* stream);

/* ---- the eigen-solve of the mode-side diagonalisation (Sec. 2.6) on its own -------
 * For the M x M pencil of a mode-side solve, C_X symmetric positive definite and C_Y
 * symmetric (both row-major device arrays; only their symmetric parts are used; CY_dev
 * may be NULL for a single operator, lam = 0 then): W (row-major device M x M, column j
 * the generalised eigenvector of C_Y w = lam_j C_X w, W^T C_X W = I) and lam (device
 * [M]), computed as the mode-side solve computes them for 32 < M from a cold start:
 * FP32 Jacobi rotations, then FP64 first-order corrections of the basis by matrix
 * products, and FP64 rotations when a correction is rejected.  *refined (host int,
 * may be NULL) receives 1 when the corrections were accepted, 0 when the rotation pass
 * ran.  Synchronous on `stream` (a cudaStream_t or NULL); allocates its workspace.
 * TAPS_ERR_INVALID_ARG for M outside (32, TAPS_MAX_M], M > 116 (S and V must fit in
 * shared memory) or null pointers; TAPS_ERR_SINGULAR when C_X is not positive definite
 * (a Cholesky pivot below -1e-8 times the largest diagonal entry). */
int taps_util_md_pencil(const double* CX_dev, const double* CY_dev, int M, double* W_dev, double* lam_dev,
                        int* refined, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TAPS_H */
