/*
 * sait.h: C ABI of the GB300 SAIT library (libsait.so).
 *
 * SAIT (Z. Lu, "A sparse approximate inverse for triangular matrices based
 * on Jacobi iteration", arXiv 2106.12836) replaces the two triangular
 * substitutions of an ILU preconditioner, U (L x) = y, by two sparse
 * matrix-vector products x = M_U (M_L y), where each M approximates T^-1 by
 * the truncated Jacobi series
 *
 *     M = sum_{i < m_terms} T~^i D^-1,   D = diag(T),   T~ = I - D^-1 T
 *
 * (Section 2, equations M_poly and T_inverse), built by the Horner recursion
 * M_k D = T~ (M_{k-1} D) + I (equation Recursive) with a dropping rule applied
 * after every product (Algorithms 1-3).
 *
 * Conventions for every entry point:
 *  - Matrices are square CSR with int32 row pointers and column indices,
 *    columns ascending within each row, FP64 values.  A sait_csr holds
 *    DEVICE pointers owned by the caller; the library reads them during the
 *    call only.
 *  - Vectors (double*) are DEVICE pointers of length n owned by the caller.
 *  - Every call is ordered on the CUDA stream given to sait_ctx_create.  Calls
 *    documented as "synchronizes" wait for that stream before returning;
 *    sait_spmv, sait_apply and sait_prec_apply only enqueue work.
 *  - Errors are returned as sait_status, never thrown and never fatal; the
 *    arguments are validated before any kernel is launched.
 *    sait_ctx_last_error gives a one-line description of the last failure.
 *  - A context and everything created with it belong to one host thread at a
 *    time.  sait_mat and sait_prec objects must be destroyed before their
 *    context; a sait_prec does not own the matrices it refers to.
 */
#ifndef SAIT_H
#define SAIT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SAIT_OK = 0,
    SAIT_ERR_INVALID_ARG = 1,    /* bad pointer, size, option, or unsorted/out-of-range column */
    SAIT_ERR_NOT_TRIANGULAR = 2, /* an entry lies on the wrong side of the diagonal */
    SAIT_ERR_ZERO_PIVOT = 3,     /* missing, zero or non-finite diagonal entry */
    SAIT_ERR_OOM = 4,            /* device allocation failed */
    SAIT_ERR_CUDA = 5,           /* any other CUDA runtime error */
    SAIT_ERR_NOT_CONVERGED = 6,  /* solver reached maxit; x holds the last iterate */
    SAIT_ERR_BREAKDOWN = 7,      /* Krylov breakdown (zero inner product) */
    SAIT_ERR_TIMEOUT = 8,        /* a bounded device-side wait ran out */
    SAIT_ERR_NONFINITE = 9,      /* NaN or Inf met in a solver */
    SAIT_ERR_UNSUPPORTED = 10    /* size beyond a documented limit (e.g. nnz >= 2^31) */
} sait_status;

/* Dropping rules applied to the unit-diagonal iterate M D after each product
 * T~ (M D) + I.  The diagonal entry is never dropped (Section 3). */
typedef enum {
    SAIT_DROP_NONE = 0,    /* keep every structural entry (exact series) */
    SAIT_DROP_ABS = 1,     /* Algorithm 2, SAIT_Thr: drop |v| < tau */
    SAIT_DROP_ROWREL = 2,  /* drop |v| < tau * max_j |(M D)_ij| of the current row */
    SAIT_DROP_PATTERN = 3, /* Algorithm 3, SAIT_Pat: the first p products are not dropped
                              and fix the pattern S; later products drop entries outside S */
    SAIT_DROP_HYBRID = 4   /* the hybrid strategy the paper's source leaves commented out
                              after Algorithm 3: the first p products are not dropped, later
                              ones drop |v| < tau */
} sait_drop_kind;

typedef struct {
    int32_t kind;   /* sait_drop_kind */
    int32_t p;      /* SAIT_DROP_PATTERN: pattern-building products; SAIT_DROP_HYBRID:
                       undropped products; 0 <= p */
    double tau;     /* SAIT_DROP_ABS / ROWREL / HYBRID: threshold, 0 <= tau < 1 */
} sait_drop;

/* Storage precision of a matrix's values for products (the FP64 values are
 * always kept as well) and the arithmetic of the products:
 *   SAIT_F64       FP64 values, FP64 arithmetic;
 *   SAIT_F32/BF16  FP32 / BF16 values, FP32 accumulation, and an FP32
 *                  intermediate vector in the SAIT apply (fewest bytes; the
 *                  rounding depends on the input, so the apply is not exactly
 *                  linear -- restarted GMRES absorbs that, BiCGSTAB can stall);
 *   SAIT_F32_X64/BF16_X64  FP32 / BF16 values and an FP64 intermediate;
 *                  single-vector products are summed in double-float (~47
 *                  significant bits, error-free two-sums on the FP32 pipe),
 *                  block products in FP64: the rounded matrix applied to
 *                  ~1e-14 relative, a fixed linear preconditioner with the
 *                  byte savings of the storage. */
typedef enum {
    SAIT_F64 = 0,
    SAIT_F32 = 1,
    SAIT_BF16 = 2,
    SAIT_F32_X64 = 3,
    SAIT_BF16_X64 = 4
} sait_dtype;

typedef enum { SAIT_LOWER = 0, SAIT_UPPER = 1 } sait_uplo;

typedef struct {
    int64_t n;               /* rows = columns */
    int64_t nnz;             /* row_ptr[n] */
    const int32_t *row_ptr;  /* device, n + 1 entries, row_ptr[0] = 0 */
    const int32_t *col;      /* device, nnz entries */
    const double *val;       /* device, nnz entries */
} sait_csr;

typedef struct {
    int32_t iters;      /* Arnoldi steps (GMRES) or iterations, two products with A each (BiCGSTAB) */
    int32_t cycles;     /* GMRES restart cycles / BiCGSTAB recurrence restarts */
    int32_t reorth_steps; /* GMRES: Arnoldi steps that needed a second Gram-Schmidt pass */
    int32_t pad;
    double rel_resid;   /* true ||b - A x||_2 / ||b||_2 at exit, computed in FP64 */
} sait_info;

/* Groups of launches timed with CUDA events when timing is enabled. */
typedef enum {
    SAIT_TIMER_APPLY = 0,     /* SAIT preconditioner applies z = M_U (M_L r) (two products) */
    SAIT_TIMER_SPMV = 1,      /* products with A inside the solvers and sait_spmv */
    SAIT_TIMER_ORTHO = 2,     /* GMRES Gram-Schmidt + Givens step (per Arnoldi step) */
    SAIT_TIMER_BUILD = 3,     /* whole sait_build calls */
    SAIT_TIMER_ILU = 4,       /* whole sait_ilu0 calls */
    SAIT_TIMER_TRISOLVE = 5,  /* exact-ILU preconditioner applies (two substitutions) */
    SAIT_TIMER_COUNT = 6
} sait_timer;

typedef struct {
    int64_t launches;                 /* kernel launches (graph kernel nodes included) */
    double ms[SAIT_TIMER_COUNT];      /* event-timed milliseconds per group */
    int64_t calls[SAIT_TIMER_COUNT];  /* calls that did work (counted on the device for
                                         launches a solver may skip after convergence) */
} sait_stats;

typedef struct sait_ctx_s *sait_ctx;
typedef struct sait_mat_s *sait_mat;
typedef struct sait_prec_s *sait_prec;

/* ---- context ----------------------------------------------------------- */

/* Create a context on the current CUDA device.  stream: a cudaStream_t, or
 * NULL for the legacy default stream.  The context owns pinned host staging
 * and the stream-ordered pool its temporaries come from. */
sait_status sait_ctx_create(sait_ctx *ctx, void *stream);
sait_status sait_ctx_destroy(sait_ctx ctx);
/* Static description of a status code. */
const char *sait_status_string(sait_status st);
/* Description of the last failure on this context ("" if none).  The pointer
 * stays valid until the next call on the context. */
const char *sait_ctx_last_error(sait_ctx ctx);

/* Turn event timing of the launch groups of sait_timer on (1) or off (0).
 * Timing adds two event records per timed call; it is off by default. */
sait_status sait_ctx_set_timing(sait_ctx ctx, int enable);
/* Restrict event timing to the groups whose bit (1 << sait_timer) is set in
 * groups (all groups by default), and within each of them to one call in
 * every (every >= 1, else SAIT_ERR_INVALID_ARG): the events around a timed
 * call cost the launch overlap of the kernels they separate, so a caller that
 * needs one group's average can leave the other calls untouched.  Timer totals
 * and call counts then cover the timed calls only. */
sait_status sait_ctx_set_timing_groups(sait_ctx ctx, uint32_t groups, int32_t every);
/* Polls a device-side dependency wait makes before it gives up with
 * SAIT_ERR_TIMEOUT (the waits of sait_ilut's rows on the rows they depend on).
 * polls <= 0 restores the default (2^22 polls with a growing sleep between them,
 * about a second).  A small limit makes a factorisation whose rows have to wait
 * at all return SAIT_ERR_TIMEOUT; the context stays usable.  Affects later
 * calls on this context only. */
sait_status sait_ctx_set_wait_limit(sait_ctx ctx, int64_t polls);
/* on != 0 (the default): sait_bicgstab_batched and sait_bicgstab_multi run
 * their iterations inside a WHILE conditional graph node, one graph launch per
 * restart round.  on = 0: the same 8-iteration graph is replayed from the host,
 * with a status read after each replay -- the path taken anyway where
 * conditional nodes are unavailable, and the one a kernel profiler can look
 * into (profilers skip the kernels of graphs with conditional nodes).  Both
 * run the same kernels in the same order, so the results are identical.
 * Affects later calls on this context only. */
sait_status sait_ctx_set_device_loop(sait_ctx ctx, int32_t on);
/* Read the launch count and timer totals accumulated since the last reset
 * (launches made by this host thread).  reset = 1 clears them afterwards.
 * Synchronizes. */
sait_status sait_ctx_stats(sait_ctx ctx, sait_stats *out, int reset);

/* ---- matrices ---------------------------------------------------------- */

/* Copy a caller CSR matrix into a library-owned matrix (FP64 storage).
 * Validates row pointers and column order.  Synchronizes. */
sait_status sait_mat_create_csr(sait_ctx ctx, const sait_csr *A, sait_mat *out);
sait_status sait_mat_destroy(sait_mat M);
/* Rows and stored entries of M. */
sait_status sait_mat_info(sait_mat M, int64_t *n, int64_t *nnz);
/* Copy M's CSR arrays (FP64 values) into caller device buffers of n + 1,
 * nnz and nnz entries.  Any pointer may be NULL to skip it.  Enqueues only. */
sait_status sait_mat_export_csr(sait_ctx ctx, sait_mat M, int32_t *row_ptr, int32_t *col,
                                double *val);
/* Select the storage precision and arithmetic of M's products (sait_dtype);
 * creates the reduced copy of the values on first use.  Synchronizes. */
sait_status sait_mat_set_store(sait_ctx ctx, sait_mat M, sait_dtype store);

/* ---- ILU factors (Section 4: level-0 and level-1 ILU factors are SAIT's input) */

/* Level-0 incomplete LU of A on A's pattern (Saad, Algorithm 10.4, IKJ order):
 * sait_iluk with level 0. */
sait_status sait_ilu0(sait_ctx ctx, const sait_csr *A, sait_mat *L, sait_mat *U);

/* Level-of-fill incomplete LU, ILU(level) for level 0 or 1 (Saad, Algorithm
 * 10.5): the entries of A's pattern have level 0, an update a_ij -= l_ik u_kj
 * gives (i,j) the level lev_ik + lev_kj + 1, and entries above `level` are
 * dropped; the elimination runs in IKJ order on the kept pattern, so the
 * factors are bit-identical to a row-by-row evaluation of the algorithm.  The
 * paper feeds level-0 and level-1 factors to SAIT (Section 4, Tables
 * runtime_SAIT and runtime_Jacobi).  Computed on the GPU: the level-1 pattern
 * row by row, then the numeric rows by warps that wait for the rows they
 * depend on (bounded waits).
 * A: device CSR, sorted columns, every diagonal entry stored.  *L: unit lower
 * triangular with its unit diagonal stored; *U: upper triangular with the
 * pivots; both new matrices owned by the caller.  Errors: level < 0 gives
 * SAIT_ERR_INVALID_ARG, level > 1 or a row with more than 512 level-1
 * candidate columns SAIT_ERR_UNSUPPORTED, a missing diagonal or a zero or
 * non-finite pivot SAIT_ERR_ZERO_PIVOT, a dependency wait that runs out
 * SAIT_ERR_TIMEOUT.  Synchronizes. */
sait_status sait_iluk(sait_ctx ctx, const sait_csr *A, int32_t level, sait_mat *L, sait_mat *U);

/* ILUT(tau, lfil) factors of A (Saad, Iterative Methods for Sparse Linear
 * Systems, Algorithm 10.6); threshold ILU factors are among the triangular
 * inputs the paper gives SAIT (Section 4).  Row i starts from a_i*, eliminates
 * its columns k < i in increasing order (fill included) with w_k /= u_kk,
 * drops w_k when |w_k| < tau ||a_i*||_2, then keeps the lfil largest entries
 * of the L part and of the U part above the same threshold; the pivot is
 * always kept.  Output as sait_ilu0: *L unit lower with the diagonal stored,
 * *U upper with the pivots, both owned by the caller.  The factors are
 * bit-identical to a row-by-row evaluation of the algorithm.
 * Requirements: tau >= 0, 0 <= lfil <= 32 (else SAIT_ERR_INVALID_ARG /
 * SAIT_ERR_UNSUPPORTED); every working row holds at most 256 entries, else
 * SAIT_ERR_UNSUPPORTED.  A zero or non-finite pivot gives
 * SAIT_ERR_ZERO_PIVOT.  Rows wait on earlier rows with bounded waits; a wait
 * that runs out gives SAIT_ERR_TIMEOUT.  Synchronizes. */
sait_status sait_ilut(sait_ctx ctx, const sait_csr *A, double tau, int32_t lfil, sait_mat *L, sait_mat *U);

/* ---- SAIT build (Algorithms 1-3) ---------------------------------------- */

/* Build M ~ T^-1 with m_terms series terms (m_terms >= 1; the loop of
 * Algorithm 1 runs m_terms - 1 times, so the paper's SAIT_Thr(tau, m) is
 * m_terms = m + 1 and SAIT_Pat(p, m) is m_terms = p + m + 1).  T must be
 * triangular on side uplo with every diagonal entry stored, nonzero and
 * finite.  Each product row is accumulated in ascending order of T~'s
 * columns with FP64 fused multiply-adds; the dropping rule acts on M D before
 * the final column scaling M = (M D) D^-1.  store selects the product
 * precision (sait_mat_set_store).  Output limit: nnz(M) < 2^31.
 * Synchronizes (the output size is data-dependent). */
sait_status sait_build(sait_ctx ctx, sait_mat T, sait_uplo uplo, int32_t m_terms, sait_drop drop,
                       sait_dtype store, sait_mat *M);

/* ---- products ----------------------------------------------------------- */

/* y = A x with A's selected storage precision and arithmetic (sait_dtype).
 * x and y must not overlap.  Enqueues only. */
sait_status sait_spmv(sait_ctx ctx, sait_mat A, const double *x, double *y);

/* SAIT preconditioner apply z = M_U (M_L r) (Section 3.1).  The intermediate
 * vector is FP64 when both matrices use FP64-accurate arithmetic (SAIT_F64,
 * *_X64), otherwise FP32.  r and z must not overlap.  Enqueues only. */
sait_status sait_apply(sait_ctx ctx, sait_mat ML, sait_mat MU, const double *r, double *z);

/* Block products for many right-hand sides / block eigenvectors.  X, Y, R, Z
 * are row-major n x k device blocks with leading dimensions ld >= k (entry
 * (i, t) at X[i * ldx + t]).  Each entry of the matrix is read once per block
 * whatever k is (Section 4.4 applies SAIT to a block of vectors this way).
 * Enqueue only. */
sait_status sait_spmm(sait_ctx ctx, sait_mat A, int32_t k, const double *X, int64_t ldx, double *Y,
                      int64_t ldy);
/* Z = M_U (M_L R) for a block of k vectors (intermediate block FP64 when both
 * matrices are stored in FP64, else FP32).  Enqueue only. */
sait_status sait_apply_multi(sait_ctx ctx, sait_mat ML, sait_mat MU, int32_t k, const double *R,
                             int64_t ldr, double *Z, int64_t ldz);

/* ---- autotuning ---------------------------------------------------------------- */

typedef struct {
    int32_t ncand;       /* candidates timed */
    int32_t chosen;      /* index of the fastest */
    int32_t format[6];   /* 0 CSR, 1 SELL-32 */
    int32_t lanes[6];    /* lanes per row (32 for SELL-32) */
    float us[6];         /* mean time of one product y = M x, microseconds */
} sait_tune_report;

/* Times every product kernel that can serve M in its current storage
 * precision (SELL-32 when its padding stays under 20%, CSR with 2..32 lanes
 * per row) on this context's stream and makes the fastest the one every later
 * product with M uses (sait_spmv, the SAIT apply, solver products).  A
 * project extension: the paper has no product kernels to choose between.
 * Synchronizes. */
sait_status sait_mat_autotune(sait_ctx ctx, sait_mat M, sait_tune_report *report);

typedef struct {
    int32_t ncand;
    int32_t chosen;
    int32_t tile_rows[6];  /* candidate tile sizes (rows) */
    float us[6];           /* one tiled dot + per-system reduction, microseconds */
} sait_batch_tune_report;

/* Chooses the tile size of the batched solver's schedule (tiles never cross a
 * system; one block reduces one tile) for the batch described by n and
 * sys_ptr (device, as in sait_bicgstab_batched) by timing the tiled dot and
 * the per-system reduction for 512..8192-row tiles, and keeps the fastest in
 * ctx for later sait_bicgstab_batched calls.  Synchronizes. */
sait_status sait_batch_autotune(sait_ctx ctx, int64_t n, int32_t nsys, const int64_t *sys_ptr,
                                sait_batch_tune_report *report);
/* Sets the tile size directly (32 .. 2^20 rows; default 2048). */
sait_status sait_ctx_set_batch_tile(sait_ctx ctx, int64_t rows);

/* ---- optimal parameters (Section 3, "Optimal parameters") -------------------------
 * The solver's runtime is iter(M_L, M_U) x (comp(M_L, M_U) + othercomp): a
 * more accurate SAIT pair (smaller tau, larger p or m) lowers the iteration
 * count but raises the cost of every apply, so some parameters minimise the
 * runtime, and they depend on the problem, the solver and the machine.
 * sait_tune_params measures them instead of guessing. */

typedef enum { SAIT_SOLVER_GMRES = 0, SAIT_SOLVER_BICGSTAB = 1, SAIT_SOLVER_PCG = 2 } sait_solver;

typedef struct {
    int32_t m_terms; /* series terms, as in sait_build */
    int32_t pad;
    sait_drop drop;  /* dropping rule, as in sait_build */
} sait_param;

#define SAIT_PARAM_MAX 16

typedef struct {
    int32_t ncand;
    int32_t chosen;                  /* index of the shortest runtime among the converged
                                        candidates; -1 when none converged */
    int32_t status[SAIT_PARAM_MAX];  /* sait_status of the candidate's build, or else of its solve */
    int32_t iters[SAIT_PARAM_MAX];   /* solver iterations (GMRES: Arnoldi steps) */
    int64_t nnz[SAIT_PARAM_MAX];     /* nnz(M_L) + nnz(M_U) */
    float build_ms[SAIT_PARAM_MAX];  /* both sait_build calls, CUDA events on the ctx stream */
    float solve_ms[SAIT_PARAM_MAX];  /* the solve from x = 0, CUDA events on the ctx stream */
    double rel_resid[SAIT_PARAM_MAX];
} sait_param_report;

/* For each of the ncand (1..SAIT_PARAM_MAX) candidates in cand (host array):
 * builds M_L = SAIT(L) and M_U = SAIT(U) in storage precision store, solves
 * A x = b from x = 0 with the given solver (restart is used by GMRES only)
 * preconditioned by z = M_U (M_L r), times both with CUDA events, and frees
 * the pair.  A candidate's runtime is build_ms + solve_ms when count_build is
 * nonzero (one solve per preconditioner), else solve_ms (the preconditioner
 * is reused).  L (unit lower, diagonal stored) and U come from sait_ilu0 or
 * sait_ilut; A, L, U stay untouched.  b, x: device, n doubles; on return x
 * holds the chosen candidate's solution.  A candidate whose build runs out
 * of memory, or whose solve does not converge, breaks down or meets a
 * non-finite value, is recorded and skipped; any other failure ends the call.  Returns SAIT_OK when at
 * least one candidate converged, else SAIT_ERR_NOT_CONVERGED (report filled
 * either way).  Synchronizes. */
sait_status sait_tune_params(sait_ctx ctx, sait_mat A, sait_mat L, sait_mat U, const double *b, double *x,
                             sait_solver solver, int32_t restart, double tol, int32_t maxit, int32_t ncand,
                             const sait_param *cand, sait_dtype store, int32_t count_build,
                             sait_param_report *report);

/* ---- batched solves ---------------------------------------------------------- */

typedef struct {
    int32_t nsys;           /* systems (or right-hand sides) */
    int32_t converged;      /* with true relative residual <= tol */
    int32_t max_iters;      /* largest per-system iteration count */
    int32_t graph_replays;  /* iterations run from the captured graph (a multiple of 8) */
    double max_rel_resid;   /* largest true ||b_s - A_s x_s|| / ||b_s|| */
    int32_t device_loop;    /* 1: the iterations looped on the device inside a WHILE
                               conditional graph node; 0: the 8-iteration graph was
                               replayed from the host (conditional nodes unavailable) */
    int32_t graph_launches; /* launches of an executable graph by the host */
} sait_batch_info;

/* BiCGSTAB on many independent systems at once.  A is block diagonal: system
 * s owns rows and columns sys_ptr[s] .. sys_ptr[s+1] (device int64 array of
 * nsys + 1 entries, sys_ptr[0] = 0, sys_ptr[nsys] = n) and has no entry
 * outside its block.  P: a SAIT pair built from A's ILU(0) factors (block
 * diagonal as well) or NULL.  Every system has its own scalars, stopping test
 * (true relative residual <= tol) and iteration count (<= maxit); converged
 * systems stop changing.  Eight iterations and the count of the systems still
 * active are captured once as the body of a WHILE conditional graph node, so
 * one graph launch runs the iterations on the device until every system has
 * stopped or maxit iterations (rounded up to a multiple of 8) have run; a
 * restart from the true residual (a system whose recurrence residual met tol
 * but whose true residual did not) starts another launch.  rel_resid (device,
 * nsys doubles) and iters (device, nsys ints) receive per-system results when
 * not NULL.  Synchronizes. */
sait_status sait_bicgstab_batched(sait_ctx ctx, sait_mat A, sait_prec P, int32_t nsys, const int64_t *sys_ptr,
                                  const double *b, double *x, double tol, int32_t maxit, sait_batch_info *info,
                                  double *rel_resid, int32_t *iters);
/* BiCGSTAB for k right-hand sides of one matrix at once: B, X row-major n x k
 * (contiguous), one set of scalars per column; the products are block
 * products (sait_spmm / sait_apply_multi), so each matrix entry is read once
 * per iteration for all k columns.  k in 1..32 or a divisor of 256.
 * Same conventions as sait_bicgstab_batched. */
sait_status sait_bicgstab_multi(sait_ctx ctx, sait_mat A, sait_prec P, int32_t k, const double *B, double *X,
                                double tol, int32_t maxit, sait_batch_info *info, double *rel_resid,
                                int32_t *iters);

/* ---- adjoint support ------------------------------------------------------ */

/* *out = M^T as a new matrix with the same storage precision (rows sorted).
 * The transposed SAIT apply of the adjoint, (M_U M_L)^T = M_L^T M_U^T, is
 * sait_prec_create_sait(ctx, MU^T, ML^T).  Synchronizes. */
sait_status sait_mat_transpose(sait_ctx ctx, sait_mat M, sait_mat *out);
/* out[e] = alpha * u[row(e)] * v[col(e)] for every stored entry e of A, in
 * A's CSR order (nnz entries).  With alpha = -1, u = lambda (adjoint
 * solution) and v = x this is dl/dA on A's pattern.  Enqueue only. */
sait_status sait_outer_on_pattern(sait_ctx ctx, sait_mat A, double alpha, const double *u, const double *v,
                                  double *out);

/* Largest n accepted by sait_apply_static. */
#define SAIT_APPLY_STATIC_MAX_N 2097152

/* z = M_U (M_L r) like sait_apply, but allocating nothing.  The paper has no
 * counterpart: this is for callers that cannot let the library allocate
 * device memory when the preconditioner is applied -- loops whose latency
 * budget forbids allocator calls, and frameworks or embedded runtimes that
 * hand out all device memory from their own pools, sized once at start-up.
 * The caller still owns r and z (device, n doubles, not overlapping); the
 * intermediate vector lives in a fixed 16 MiB array compiled into the
 * library, present on every device that loads the library until the process
 * exits.  Requirements and behaviour:
 *  - n <= SAIT_APPLY_STATIC_MAX_N, else SAIT_ERR_UNSUPPORTED; ML and MU must
 *    live on the current device (else SAIT_ERR_INVALID_ARG).
 *  - Enqueues two products on `stream` (a cudaStream_t, NULL = legacy default
 *    stream) and returns; no context is needed, and sait_ctx_last_error does
 *    not see its failures.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress); make that first call before any stream capture.
 *    A device reset (cudaDeviceReset) frees the array together with every
 *    matrix on the device; the context that has to be created again to
 *    rebuild the matrices makes the next call look the address up again.
 *  - Every call on a device shares the one array: calls whose work overlaps
 *    on the GPU (different streams, no ordering between them) race and give
 *    wrong results.  Calls ordered on one stream are safe. */
sait_status sait_apply_static(sait_mat ML, sait_mat MU, const double *r, double *z, void *stream);

/* ---- preconditioner objects for the solvers ----------------------------- */

/* SAIT pair: applies z = M_U (M_L r). */
sait_status sait_prec_create_sait(sait_ctx ctx, sait_mat ML, sait_mat MU, sait_prec *P);
/* Exact ILU: z = U^-1 (L^-1 r) by level-scheduled substitution (the exact
 * triangular solves SAIT replaces; the paper's comparison in Section 4).
 * Computes the level sets on the GPU.  Synchronizes. */
sait_status sait_prec_create_ilu(sait_ctx ctx, sait_mat L, sait_mat U, sait_prec *P);
/* Jacobi sweeps (Section 4, comparison with Jacobi iteration): `sweeps`
 * iterations of x^j = T~ x^{j-1} + D^-1 b (Section 2, equation Jacobi_iter)
 * from x^0 = 0, first on L y = r, then on U z = y.  This applies the undropped
 * series M_k of both factors without forming it; it is the comparator the
 * paper uses to show why the stored SAIT matrices are cheaper.  L and U are
 * any square matrices with a nonzero diagonal (triangular in practice) and
 * must outlive P.  sweeps >= 1, else SAIT_ERR_INVALID_ARG; a zero, missing or
 * non-finite diagonal entry gives SAIT_ERR_ZERO_PIVOT.  Synchronizes. */
sait_status sait_prec_create_jacobi(sait_ctx ctx, sait_mat L, sait_mat U, int32_t sweeps, sait_prec *P);
/* Number of level sets of the lower and upper factor (ILU preconditioner). */
sait_status sait_prec_levels(sait_prec P, int32_t *levels_lower, int32_t *levels_upper);
/* z = P r; enqueues only. */
sait_status sait_prec_apply(sait_ctx ctx, sait_prec P, const double *r, double *z);
sait_status sait_prec_destroy(sait_prec P);

/* ---- solvers (Section 4 uses PCG/LOBPCG; GMRES and BiCGSTAB extend it to
 * the nonsymmetric case) ------------------------------------------------ */

/* Restarted GMRES(restart) with right preconditioning (Saad, Algorithm 9.5):
 * Arnoldi with classical Gram-Schmidt and one reorthogonalisation, the second
 * pass of each vector delayed into the next step's sweep (DCGS2: two sweeps
 * over the basis per step), Givens rotations on the device applied once a
 * column is final, x <- x + P (V y) at the end of each cycle.  Dots run in
 * FP32 and updates in double-float on an FP32 (hi, lo) copy of the basis; the
 * Arnoldi relation holds to ~1e-14 and the basis is orthogonal to ~1e-7.
 * P may be NULL (no preconditioner).  x: in, the initial guess; out, the
 * solution.  Stops when the true relative residual ||b - A x|| / ||b|| <= tol
 * (checked at the end of every cycle; the rotated residual estimate ends a
 * cycle early).  maxit bounds the Arnoldi steps.  1 <= restart <= 512.
 * The host reads a device status word every few steps.  Synchronizes;
 * fills *info if info is not NULL. */
sait_status sait_gmres(sait_ctx ctx, sait_mat A, sait_prec P, const double *b, double *x,
                       int32_t restart, double tol, int32_t maxit, sait_info *info);

/* Preconditioned conjugate gradients (Saad, Algorithm 9.1), the solver of the
 * paper's experiments (Section 4).  The preconditioner is applied as given --
 * the SAIT pair M_U M_L is not symmetric, as in the paper.  Stops when the
 * recursive residual satisfies ||r|| <= tol ||b||; info->rel_resid is the true
 * residual at exit, info->iters the iterations.  Same conventions as
 * sait_gmres. */
sait_status sait_pcg(sait_ctx ctx, sait_mat A, sait_prec P, const double *b, double *x, double tol, int32_t maxit,
                     sait_info *info);

/* The k smallest eigenpairs of symmetric positive definite A by LOBPCG
 * (Knyazev 2001; the paper's block eigensolver, Section 4.4) with the SAIT
 * preconditioner P applied to the residual block as two block products (or
 * none when P is NULL).  X: device, n x k row-major; in: initial block (full
 * rank), out: eigenvectors (orthonormal).  lambda: device, k doubles,
 * ascending.  Converged columns (||A x_j - lambda_j x_j|| <= tol lambda_j
 * ||x_j||) are locked softly; the Rayleigh-Ritz step on [X, W, P] is FP64
 * (Cholesky, one-block Jacobi eigensolver).  1 <= k <= 20, 3k <= n.
 * info->iters: iterations; info->rel_resid: largest column residual.
 * Synchronizes every iteration (active count). */
sait_status sait_lobpcg(sait_ctx ctx, sait_mat A, sait_prec P, int32_t k, double *X, double *lambda, double tol,
                        int32_t maxit, sait_info *info);

/* BiCGSTAB with right preconditioning (van der Vorst 1992; Saad,
 * Algorithm 7.7 on A P u = b).  Same conventions as sait_gmres; maxit bounds
 * the iterations (two products with A each). */
sait_status sait_bicgstab(sait_ctx ctx, sait_mat A, sait_prec P, const double *b, double *x,
                          double tol, int32_t maxit, sait_info *info);

#ifdef __cplusplus
}
#endif

#endif /* SAIT_H */
