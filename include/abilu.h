/*
 * abilu.h — C ABI of the GB300 (sm_103a) asynchronous block ILU(0) library.
 *
 * The method: Kashi & Nadarajah, "An asynchronous incomplete block LU
 * preconditioner for computational fluid dynamics on unstructured grids".
 * A 4x4 block-sparse system A x = b (Sec. 2: the d+2 = 4 unknowns of a cell are
 * contiguous) is solved by right-preconditioned flexible GMRES (Sec. 2, Sec. 6)
 * with M = L U, where L and U are computed by fixed-point sweeps of Eq. (bilu)
 * (Sec. 4.2) and applied by block triangular sweeps (Algorithm 5, Sec. 4.1).
 *
 * Conventions that hold for every entry point
 * -------------------------------------------
 * Storage. Block CSR with 4x4 blocks: rowptr int32[n+1], colind int32[nnzb],
 *   column indices strictly increasing inside each row, the diagonal block
 *   present in every row; values double[nnzb][4][4], each block row-major.
 *   Vectors are double[n][4] (all 4 unknowns of a cell contiguous).
 * Memory. Unless a parameter says "host", every pointer is a DEVICE pointer on
 *   the current CUDA device, owned by the caller, and must stay valid until the
 *   work enqueued on `stream` has finished.  Value and vector pointers must be
 *   16-byte aligned.  Handles (abilu_pattern, abilu_factors) are owned by the
 *   library and hold their own device memory, released by *_destroy.
 * Streams. `stream` is a cudaStream_t (NULL = the legacy default stream).  All
 *   calls enqueue work on it and return without waiting, except the ones whose
 *   description says they synchronise (they return a result that lives on the
 *   device: pattern validation, fgmres_solve, abilu_factors_status).
 * Errors. Every call returns an abilu_status; nothing aborts or throws across
 *   the ABI and no kernel traps.  abilu_last_error() gives a message for the
 *   last non-OK status of the calling thread.  ABILU_WARN_SINGULAR means the
 *   call succeeded but a singular (or non-finite) diagonal block was replaced
 *   by the identity for its inversion: the "modified iteration" of Sec. 4.2.
 * Threads. Handles are not thread-safe: one host thread (or external locking)
 *   per handle.  Different handles may be used concurrently on different streams.
 */
#ifndef ABILU_H
#define ABILU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void *abilu_stream; /* a cudaStream_t */

typedef enum {
    ABILU_OK = 0,
    ABILU_EINVAL = 1,          /* bad argument or malformed pattern */
    ABILU_ENOMEM = 2,          /* device allocation failed */
    ABILU_ECUDA = 3,           /* a CUDA runtime call failed */
    ABILU_ENOCONV = 4,         /* FGMRES stopped at max_iters above rtol */
    ABILU_ETIMEOUT = 5,        /* a bounded device-side wait ran out */
    ABILU_WARN_SINGULAR = 6    /* success, but singular diagonal blocks were replaced */
} abilu_status;

typedef enum {
    ABILU_F64 = 0,             /* factors stored in FP64, sweeps in FP64 */
    ABILU_F32 = 1,             /* factors stored in FP32, apply sweeps in FP32 */
    ABILU_BF16 = 2             /* factors stored in BF16, apply sweeps in FP32 */
} abilu_dtype;

typedef enum {
    ABILU_SYNC = 0,            /* Jacobi-type sweeps: every update reads the previous iterate */
    ABILU_ASYNC = 1            /* in-place sweeps reading the latest values, no barrier between sweeps */
} abilu_mode;

typedef enum {
    ABILU_INIT_FROM_A = 0,          /* X^0 = A (L^0 = strictly lower part of A, unscaled) */
    ABILU_INIT_FROM_PREVIOUS = 1    /* X^0 = the factors currently in the handle (warm start) */
} abilu_init;

typedef struct abilu_pattern_s *abilu_pattern;
typedef struct abilu_factors_s *abilu_factors;

/* Library version string, e.g. "abilu-gb300 0.1". Host memory, static. */
const char *abilu_version(void);

/* Message for the last non-OK status returned to the calling thread (static). */
const char *abilu_last_error(void);

/* Number of CUDA kernels this library has launched in this process so far
 * (all threads, all devices).  Instrumentation: the difference across a region
 * is how many of the library's kernels ran in it. */
uint64_t abilu_kernel_launches(void);

/*
 * Pattern analysis (the block sparsity pattern S_B of Sec. 4.2, which must
 * contain every diagonal block).  Copies rowptr/colind (device pointers) into
 * the handle, checks them, finds the diagonal of each row, splits every row
 * into its strictly lower (L) and strictly upper (U) blocks, and lists for
 * every block (i,j) the product pairs (L_ik, U_kj), k < min(i,j), of Eq. (bilu)
 * whose two blocks are both in S_B.  Synchronises `stream` (it reads back the
 * validation result).  ABILU_EINVAL for n < 1, nnzb < n, unsorted or
 * out-of-range columns or a missing diagonal block.  *out is set on success.
 */
abilu_status abilu_pattern_create(int32_t n, int32_t nnzb, const int32_t *rowptr,
                                  const int32_t *colind, abilu_stream stream,
                                  abilu_pattern *out);
void abilu_pattern_destroy(abilu_pattern p);

/* Host-side counts of a pattern: n, nnzb, strictly-lower blocks, strictly-upper
 * blocks, product pairs, largest row length, blocks a build sweep updates (all
 * but the strictly-upper blocks without product pairs, which stay equal to A).
 * `out` is host int64_t[7]. */
abilu_status abilu_pattern_counts(abilu_pattern p, int64_t *out);

/* Copies the pattern's rowptr (int32[n+1]) and colind (int32[nnzb]) into
 * caller-owned device arrays (either may be NULL).  Asynchronous on `stream`. */
abilu_status abilu_pattern_arrays(abilu_pattern p, int32_t *rowptr, int32_t *colind,
                                  abilu_stream stream);

/*
 * Factor storage for one pattern: L (strictly lower blocks), U (strictly upper
 * blocks), inv(U_ii) and U_ii, in `dtype`, plus the work vectors of the
 * triangular sweeps.  F64: build arithmetic and 4x4 inversions in FP64.
 * F32/BF16: the build sweeps compute in FP32 from an FP32 copy of A, and each
 * inversion is an FP32 adjugate refined by one error-free Newton step (the
 * FP32 rounding of the exact inverse for cond(U_ii) << 4000); the apply
 * sweeps run in FP32.  F32 also keeps inv(U_ii) U_ij for the upper sweeps.
 */
abilu_status abilu_factors_create(abilu_pattern p, abilu_dtype dtype, abilu_factors *out);
void abilu_factors_destroy(abilu_factors f);

/*
 * Factors of the scalar variant the paper compares against: Chow and Patel's
 * asynchronous ILU(0) taken entry by entry on the scalar pattern (every entry
 * of every block), Sec. 3.2, Eq. (scalarilu_fp_detail), Algorithm 3, applied
 * by scalar triangular sweeps (Algorithm 2).  abilu_build, abilu_apply,
 * fgmres_solve and abilu_factors_export take such a handle like a block one
 * (sync/async sweeps, zero guesses, X^0 = A); a zero pivot is replaced by 1 and
 * counted.  Export writes X in A's layout with each diagonal block holding its
 * strictly lower L entries (unit diagonal implied) and the rest of U; Dinv is
 * not written.  Diagnostics and batches are block-only.  dtype: ABILU_F64 only
 * (ABILU_EINVAL otherwise).
 */
abilu_status abilu_factors_create_scalar(abilu_pattern p, abilu_dtype dtype, abilu_factors *out);

/*
 * Build the preconditioner: `nsweeps` fixed-point sweeps of Eq. (bilu),
 *   U_ij = A_ij - sum_{k<i} L_ik U_kj            (i <= j),
 *   L_ij = (A_ij - sum_{k<j} L_ik U_kj) U_jj^-1  (i > j),
 * over every block of S_B at once.  ABILU_SYNC: x^{n+1} = h(x^n) (Eq.
 * seq_blockilu_fp), deterministic and bit-reproducible; ABILU_ASYNC: in-place
 * updates reading whatever values are current, work items (single blocks for
 * FP32/BF16 factors, block rows for FP64) taken in chunks from a queue, no
 * barrier between sweeps (Algorithm 4 with blocks, Eq. async_blockilu_fp).
 * `A_vals` double[nnzb][4][4] on the device.
 * nsweeps >= 0 (0 leaves X^0).  Singular diagonal blocks met during the build
 * are counted on the device; read them with abilu_factors_status.
 */
abilu_status abilu_build(abilu_factors f, const double *A_vals, int nsweeps, abilu_mode mode,
                         abilu_init init, abilu_stream stream);

/*
 * Apply the preconditioner, z ~= (L U)^{-1} r: `nsweeps_lower` sweeps on
 * L y = r from y = 0, then `nsweeps_upper` sweeps on U z = y from z = 0
 * (Algorithm 5 and its backward analogue, zero initial guesses, Sec. 6 setup).
 * ABILU_SYNC: Jacobi sweeps; ABILU_ASYNC: in-place sweeps (backward row order
 * for U) with no barrier between sweeps.  r and z are double[n][4], distinct.
 * Sweep counts >= 0; 0 lower sweeps gives y = 0.
 */
abilu_status abilu_apply(abilu_factors f, const double *r, double *z, int nsweeps_lower,
                         int nsweeps_upper, abilu_mode mode, abilu_stream stream);

/*
 * abilu_apply_noalloc — the synchronous FP64 preconditioner application for
 * callers that cannot allocate device memory.  The paper has no counterpart:
 * this is an interface for callers that cannot call cudaMalloc (code inside
 * another library's allocator hooks or memory pool, frameworks that reserve
 * all device memory up front, code that must not allocate while a CUDA graph
 * is being built).  It allocates nothing: the factors come in as plain arrays
 * and the sweep vectors live in a fixed __device__ array inside the library.
 *
 * Computes the same z as abilu_apply(..., ABILU_SYNC) on FP64 factors:
 * nsweeps_lower Jacobi sweeps on L y = r from y = 0, then nsweeps_upper on
 * U z = y from z = 0.  rowptr/colind: the pattern (device int32[n+1],
 * int32[nnzb], 4-byte aligned), which must be one that abilu_pattern_create
 * accepts: nothing here validates it (a column outside [0, n) is skipped, so
 * it reads nothing out of bounds, but the result is then meaningless);
 * X: double[nnzb][4][4] factors in A's pattern layout (L_ij at column < row,
 * U_ij at column > row, the diagonal entry ignored), as abilu_factors_export
 * writes them; Dinv: double[n][4][4] = inv(U_ii); r, z: double[n][4],
 * distinct.  All device pointers, caller-owned; X, Dinv, r and z must be
 * 16-byte aligned (ABILU_EINVAL otherwise, checked before any device work).
 *
 * Limit: n <= 65,536 cells (the fixed scratch is 3 vectors of that size,
 * 6 MiB, held by every GPU that loads the library until the process exits);
 * larger n returns ABILU_EINVAL without touching the device.  The first call
 * on each device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current).  With lazy module loading that first call is
 * also where the library's module is loaded on the device and the 6 MiB array
 * is reserved, so a caller that may not allocate at all should make one call
 * during its set-up (any small valid call), and before any stream capture.
 * The looked-up address is kept for the life of the process: after
 * cudaDeviceReset on a device this entry point must not be used there again.
 * All calls share the one array: calls whose work overlaps on the GPU
 * (different streams or host threads) race on it; serialise them.  Asynchronous
 * on `stream`; returns ABILU_EINVAL for bad arguments.
 */
abilu_status abilu_apply_noalloc(int32_t n, const int32_t *rowptr, const int32_t *colind,
                                 const double *X, const double *Dinv, const double *r, double *z,
                                 int nsweeps_lower, int nsweeps_upper, abilu_stream stream);

/*
 * Block sparse matrix-vector product y = alpha * A x + beta * y (FP64), the
 * product FGMRES needs once per iteration (Sec. 6 setup).  x and y distinct.
 * beta == 0 does not read y.
 */
abilu_status bsr_spmv(abilu_pattern p, const double *A_vals, double alpha, const double *x,
                      double beta, double *y, abilu_stream stream);

/*
 * Copy the factors out in A's pattern layout, FP64: X[nnzb][4][4] holds L_ij at
 * positions with column < row and U_ij at column >= row; Dinv[n][4][4] holds
 * inv(U_ii).  Either pointer may be NULL.
 */
abilu_status abilu_factors_export(abilu_factors f, double *X, double *Dinv, abilu_stream stream);

/*
 * Diagnostics of the current factors against A (Sec. 6.2, the quantities the
 * paper tracks over pseudo-time steps), evaluated in FP64 from the stored
 * factors; `out` is host double[4]:
 *   out[0] = ||x - h(x)||_1, the ILU fixed-point residual over all entries of
 *            L and U, h being the map of Eq. (blockH) with inv(U_jj) recomputed
 *            from the stored U_jj (the paper plots its ratio to the value at
 *            the initial guess: call this after a 0-sweep build for that);
 *   out[1] = max |(LU)_ij - A_ij| over the blocks of S_B (0 at the fixed point);
 *   out[2] = ||L - I||_inf, the max-norm of the Jacobi iteration matrix of the
 *            lower block triangular solve (unit diagonal blocks);
 *   out[3] = ||D_U^{-1}(U - D_U)||_inf for the upper solve, D_U = block diagonal.
 * Synchronises `stream`.
 */
abilu_status abilu_factors_diagnostics(abilu_factors f, const double *A_vals, double *out,
                                       abilu_stream stream);

/* Synchronises `stream`, then returns in *singular_blocks (host) how many
 * singular diagonal blocks the builds since the last call replaced, and resets
 * the count.  Returns ABILU_ETIMEOUT (and resets it) if a bounded wait inside
 * an asynchronous application's staged pipeline ran out since the last call
 * (the results of that application are then invalid; never expected). */
abilu_status abilu_factors_status(abilu_factors f, int64_t *singular_blocks, abilu_stream stream);

/* Spin limit of the bounded device-side waits of this handle's builds and
 * applications called directly (abilu_build, abilu_apply): polls before a wait
 * gives up and counts a timeout (read with abilu_factors_status).  0 restores
 * the library default, 2^24.  fgmres_solve uses its options' spin_limit for
 * its own duration and leaves the handle's value as it was.  limit >= 0. */
abilu_status abilu_factors_set_spin_limit(abilu_factors f, int64_t limit);

/* Launch shape of the asynchronous block build (FP32/BF16 factors): the work
 * blocks a warp takes per ticket from the build's queue (a multiple of 32 in
 * 32..512; 0 restores the default, 128).  A ticket is made of sub-chunks of
 * 64 consecutive blocks (32 for sizes that are not multiples of 64) spread
 * evenly over the work list, so the blocks in flight cover one short span in
 * each part of the list.  Any value gives a legal asynchronous iteration
 * (Algorithm 4 with blocks); it trades the contention on the one ticket
 * counter against load balance and against how many of the rows a block
 * reads were already updated in the current sweep (a shorter span in flight
 * per part of the list leaves a lower ILU fixed-point residual after the same
 * sweeps).  An autotuner's knob
 * (abilu_batch_set_build_chunk sets it on a batch's factors). */
abilu_status abilu_factors_set_build_chunk(abilu_factors f, int32_t blocks);

/* Failure injection for tests of the bounded waits (no counterpart in the
 * paper).  With `enable` nonzero, the next asynchronous build of block factors
 * on `f` that uses the ordered variant (the work list has fewer than four
 * tickets per resident warp: every small system) starts its
 * per-chunk sweep flags one sweep behind, a value no warp ever publishes: the
 * first wait of every chunk polls `spin_limit` times, gives up, counts a
 * timeout and the warp stops.  That build leaves the factors partly swept,
 * and the call that reports its status (fgmres_solve, abilu_factors_status)
 * returns ABILU_ETIMEOUT.  The flag is cleared by that build; no GPU fault,
 * trap or hang is involved. */
abilu_status abilu_factors_inject_stall(abilu_factors f, int enable);

/* Instrumentation of the build sweeps (Eq. bilu; the paper times its sweeps
 * the same way, Sec. 6).  With `enable` nonzero, every later build of block
 * factors on this handle (abilu_build, or the build inside fgmres_solve)
 * records two CUDA events on its stream, right before its first and right
 * after its last sweep kernel (the preparation pass over A and the scaled
 * upper blocks are outside them); `enable` 0 stops it.  The events are the
 * handle's, created by the first enabling call (ABILU_ECUDA if that fails).
 * abilu_factors_sweep_time waits for the second event of the last timed build
 * and returns the device time between the two in *ms (host, milliseconds);
 * ABILU_EINVAL if no build was timed since timing was enabled (scalar factors
 * are never timed). */
abilu_status abilu_factors_timing(abilu_factors f, int enable);
abilu_status abilu_factors_sweep_time(abilu_factors f, float *ms);

typedef struct {
    int32_t restart;            /* m of FGMRES(m); 1..64 */
    int32_t max_iters;          /* total Arnoldi steps over all restarts */
    double rtol;                /* stop at ||b - A x|| <= rtol ||b|| */
    int32_t build_sweeps;       /* sweeps of abilu_build done inside the solve */
    int32_t apply_sweeps_lower; /* sweeps on L per preconditioner application */
    int32_t apply_sweeps_upper; /* sweeps on U per preconditioner application */
    int32_t mode;               /* abilu_mode for build and apply */
    int32_t build;              /* 1: build the factors from A inside the solve; 0: use them as they are */
    int32_t init;               /* abilu_init for that build */
    int32_t reorth;             /* 0: one classical Gram-Schmidt pass; 1: two passes (CGS2).
                                   With 0 and rtol >= 1e-7 the pass is one reduction:
                                   h_{j+1,j} = sqrt(||w||^2 - sum_k h_k^2), formed with the
                                   dot products; below 1e-7 h_{j+1,j} is the explicit norm of
                                   the updated w (that formula assumes an orthonormal basis,
                                   which a classical basis loses as the residual falls) */
    int32_t zero_guess;         /* 1: start from x0 = 0 (x is overwritten; r0 = b, no SpMV) */
    int64_t spin_limit;         /* polls of a bounded device-side wait before it gives up and
                                   the solve returns ABILU_ETIMEOUT (the ordered asynchronous
                                   build's per-chunk wait, the staged sweeps' barrier waits);
                                   0: the library default, 2^24; >= 0 */
} fgmres_opts;

typedef struct {
    int32_t iters;              /* Arnoldi steps over all restarts */
    int32_t restarts;           /* restart cycles completed */
    double rel_resid_est;       /* last Givens estimate / ||b|| */
    double rel_resid_true;      /* ||b - A x|| / ||b|| computed in FP64 at exit */
    int64_t singular_blocks;    /* singular diagonal blocks replaced in the build */
    int32_t status;             /* abilu_status of the solve */
} fgmres_result;

/* Defaults: restart 30, max_iters 2500, rtol 1e-6, 1 build / 3+3 apply sweeps
 * (the paper's choice, Sec. 6.1), ABILU_ASYNC, build from A, reorth 0,
 * zero_guess 0 (x holds x0), spin_limit 0 (the library default). */
void fgmres_default_opts(fgmres_opts *opts);

/*
 * Solve A x = b by FGMRES(m) right-preconditioned with block ILU(0) (Sec. 2,
 * Sec. 6 setup): x holds x0 on entry (double[n][4], device) and the solution
 * on return.  `f` is a factors handle of pattern `p` (built inside the solve
 * when opts->build is 1), or, with opts->build = 0, of another pattern with
 * the same n (the filled pattern of abilu_parilut).  Arnoldi, Givens rotations, the SpMV and the true
 * residual are FP64 whatever the factor dtype.  `res` (host) is filled.
 * Synchronises `stream`.  Returns ABILU_ENOCONV (with res filled) when
 * max_iters is reached above rtol; ABILU_WARN_SINGULAR on a converged solve
 * whose build replaced singular blocks.
 */
abilu_status fgmres_solve(abilu_pattern p, const double *A_vals, abilu_factors f,
                          const double *b, double *x, const fgmres_opts *opts,
                          fgmres_result *res, abilu_stream stream);

/*
 * Multigrid with block ILU smoothing.  The paper's closing section names
 * asynchronous block ILU iterations as fine-grain parallel multigrid smoothers
 * as future work (with the study of their smoothing property) and fixes no
 * cycle; this is the library's: a V-cycle on Galerkin coarse operators of an
 * aggregation hierarchy whose smoother on every level is
 *   x += M^{-1} (b - A x),  M = L U the block ILU(0) of that level's matrix,
 * built by the sweeps of abilu_build and applied by those of abilu_apply.
 *
 * Hierarchy.  Strength ||A_ij||_F^2 (entries summed in storage order); in
 * row i, j != i is strong when it is > 0 and >= theta^2 max_{k != i}
 * ||A_ik||^2.  Pass 1 (cells ascending): an unplaced cell with a strong
 * coupling and no placed strong neighbour roots an aggregate of itself and
 * its strong neighbours; pass 2: a leftover cell joins the pass-1 aggregate of
 * its strongest placed neighbour (lowest column on ties), or stands alone.
 * Aggregates are numbered in creation order.  Transfer is piecewise constant
 * (P_{i,agg(i)} = I_4, restriction P^T) and A_c = P^T A P, coarse blocks
 * summed in ascending fine position.  Coarsening stops at max_levels levels,
 * at or below min_coarse cells, or when aggregation stops reducing the count.
 *
 * Cycle, on level l from x = 0: pre_smooth steps, b_c = P^T (b - A x), the
 * cycle on level l+1 for x_c, x += P x_c, post_smooth steps; the coarsest level
 * takes coarse_smooth steps.  Each step applies M^{-1} with apply_sweeps_lower
 * / apply_sweeps_upper triangular sweeps in `mode`; vectors are FP64, factors
 * in factor_dtype.
 */
#define ABILU_MG_MAX_LEVELS 16
typedef struct {
    int32_t max_levels;          /* 1..ABILU_MG_MAX_LEVELS */
    int32_t min_coarse;          /* stop coarsening at or below this many cells (>= 1) */
    double theta;                /* strong-coupling threshold, 0 <= theta <= 1 */
    int32_t factor_dtype;        /* abilu_dtype of every level's factors (block variant) */
    int32_t build_sweeps;        /* build sweeps per level at set-up */
    int32_t apply_sweeps_lower;  /* sweeps on L per smoothing step */
    int32_t apply_sweeps_upper;  /* sweeps on U per smoothing step */
    int32_t pre_smooth;          /* smoothing steps before the coarse correction */
    int32_t post_smooth;         /* smoothing steps after it */
    int32_t coarse_smooth;       /* smoothing steps on the coarsest level */
    int32_t mode;                /* abilu_mode of the builds and the smoothing sweeps */
    int32_t init;                /* abilu_init of the builds (warm start keeps each level's factors) */
} abilu_mg_opts;
typedef struct abilu_mg_s *abilu_mg;

/* Defaults: 10 levels, min_coarse 512, theta 0.25, FP32 factors, 4 build and
 * 2+2 apply sweeps, 1 pre-, 1 post- and 2 coarsest-level smoothing steps,
 * ABILU_SYNC, builds from A. */
void abilu_mg_default_opts(abilu_mg_opts *opts);

/*
 * abilu_mg_create: the hierarchy of pattern `p` with values `A_vals` (device,
 * double[nnzb][4][4]; they set the strengths, and the aggregation stays fixed
 * for the handle's life): coarse patterns, transfer lists, coarse values,
 * factor storage and work vectors of every level, owned by the handle.  The
 * handle keeps `p` (not a copy): destroy the handle first.  Synchronises
 * `stream`.  ABILU_EINVAL on bad options.
 * abilu_mg_setup: numeric set-up for new values on the same pattern: the
 * coarse values, then `build_sweeps` block ILU sweeps on every level (with the
 * handle's mode and init).  A_vals must stay valid while the handle applies
 * the cycle.  Asynchronous on `stream`.
 * abilu_mg_apply: z = one V-cycle applied to r (double[n][4] each, device,
 * distinct).  Asynchronous on `stream`.
 * abilu_mg_levels: host int64_t[2 * ABILU_MG_MAX_LEVELS + 1]: out[0] = levels,
 * out[1 + 2l] = cells and out[2 + 2l] = blocks of level l.
 * abilu_mg_level_data: copies level l's aggregates (agg int32[n_l], each
 * cell's aggregate on level l+1; not for the coarsest level), pattern
 * (rowptr int32[n_l+1], colind int32[nnzb_l]), values (double
 * [nnzb_l][4][4]) and block ILU factors in FP64, laid out as
 * abilu_factors_export writes them (X double[nnzb_l][4][4], Dinv
 * double[n_l][4][4]); device pointers, any may be NULL.  Level 0's pattern
 * and values are the caller's.  Asynchronous on `stream`.
 */
abilu_status abilu_mg_create(abilu_pattern p, const double *A_vals, const abilu_mg_opts *opts,
                             abilu_stream stream, abilu_mg *out);
void abilu_mg_destroy(abilu_mg mg);
abilu_status abilu_mg_setup(abilu_mg mg, const double *A_vals, abilu_stream stream);
abilu_status abilu_mg_apply(abilu_mg mg, const double *r, double *z, abilu_stream stream);
abilu_status abilu_mg_levels(abilu_mg mg, int64_t *out);
abilu_status abilu_mg_level_data(abilu_mg mg, int32_t level, int32_t *agg, int32_t *rowptr,
                                 int32_t *colind, double *vals, double *X, double *Dinv,
                                 abilu_stream stream);

/*
 * FGMRES(m) (as fgmres_solve, Sec. 2 and Sec. 6 setup) right-preconditioned
 * by one V-cycle per Arnoldi step on the level-0 pattern of `mg`.  opts->build:
 * abilu_mg_setup(mg, A_vals) inside the solve; otherwise the cycle uses the
 * values of the last set-up, and A_vals must be those same values.  The
 * smoother settings come from the handle (opts' sweep counts and mode are not
 * used).  Synchronises `stream`; statuses as fgmres_solve (singular blocks
 * counted over all levels).
 */
abilu_status fgmres_solve_mg(abilu_mg mg, const double *A_vals, const double *b, double *x,
                             const fgmres_opts *opts, fgmres_result *res, abilu_stream stream);

/*
 * Threshold block ILU by fixed-point sweeps.  The paper's closing section
 * names a parallel threshold ILU (ParILUT) as the next extension of its
 * sweeps, without an algorithm; this is the library's, in FP64:
 *   start  X = A on A's pattern, `sweeps` synchronous sweeps of Eq. (bilu);
 *   `iters` times:
 *     fill  the pattern becomes that of L U (L unit lower, U upper; it
 *           contains the current one); new blocks start at zero and A is zero
 *           outside its own pattern; `sweeps` synchronous sweeps;
 *     drop  the strictly lower blocks whose squared Frobenius norm exceeds the
 *           (budget+1)-th largest are kept (all of them if at most budget),
 *           likewise the strictly upper ones, budgets floor(fill x the counts
 *           of A's pattern); diagonal blocks always; `sweeps` synchronous
 *           sweeps on the kept pattern.
 * abilu_parilut returns a new pattern handle (the final pattern, n cells) and
 * factors on it, both owned by the caller (abilu_pattern_destroy,
 * abilu_factors_destroy): abilu_apply, abilu_factors_export (in the new
 * pattern's layout) and fgmres_solve (with opts->build = 0) take them.  The
 * factorisation runs in FP64; the returned factors are stored in
 * factor_dtype (FP32: rounded, with Dinv U for the upper sweeps, as a build
 * leaves them).
 * Synchronises `stream`.  ABILU_EINVAL on bad options or when a row of L U
 * would exceed 192 blocks.  iters = 0 gives block ILU(0) after `sweeps`
 * sweeps, on a copy of A's pattern.
 */
typedef struct {
    double fill;          /* budget factor, >= 0 (2.0: twice A's lower / upper blocks) */
    int32_t iters;        /* fill-and-drop steps, >= 0 */
    int32_t sweeps;       /* synchronous sweeps after the start and after every change, >= 0 */
    int32_t factor_dtype; /* abilu_dtype of the returned factors */
} abilu_parilut_opts;

/* Defaults: fill 2.0, 3 steps, 2 sweeps, FP64 factors. */
void abilu_parilut_default_opts(abilu_parilut_opts *opts);
abilu_status abilu_parilut(abilu_pattern p, const double *A_vals, const abilu_parilut_opts *opts,
                           abilu_stream stream, abilu_pattern *pattern_out,
                           abilu_factors *factors_out);

/*
 * Batched solves: many independent systems of uneven size (for example one
 * Jacobian per grid block or per request) handled by the same launches.  Each
 * system is the problem above, solved by the same method; the batch runs every
 * build sweep, triangular sweep and SpMV of all systems in one launch (the
 * systems form one block-diagonal pattern, each system's rows padded to a
 * multiple of 64 with identity rows), and FGMRES keeps a separate Krylov
 * state, Hessenberg, Givens rotations and convergence test per system; the
 * systems iterate in lockstep and a converged system stops contributing.
 *
 * abilu_batch_create: `n`, `nnzb` are HOST arrays [nsys]; `rowptr`, `colind`
 * are HOST arrays [nsys] of DEVICE pointers to each system's pattern (as for
 * abilu_pattern_create; copied).  Synchronises `stream`.  The batch owns the
 * concatenated values, right-hand sides, solutions, factors (in `dtype`) and
 * Krylov workspace.
 * abilu_batch_set_system: copies system s's A values (device, double
 * [nnzb_s][4][4]) and right-hand side (device, double[n_s][4]) into the batch;
 * either may be NULL to keep the current one.  Asynchronous on `stream`.
 * abilu_batch_solve: builds (if opts->build) and solves every system from
 * x0 = 0 with the options of fgmres_solve; `res` is a HOST array [nsys].
 * Synchronises `stream`.  ABILU_ENOCONV if any system did not converge.
 * abilu_batch_get_solution: copies system s's solution (device, double
 * [n_s][4]).  abilu_batch_counts: host int64_t[4] = systems, padded rows,
 * blocks, 64-row chunks.
 */
typedef struct abilu_batch_s *abilu_batch;
abilu_status abilu_batch_create(int32_t nsys, const int32_t *n, const int32_t *nnzb,
                                const int32_t *const *rowptr, const int32_t *const *colind,
                                abilu_dtype dtype, abilu_stream stream, abilu_batch *out);
void abilu_batch_destroy(abilu_batch b);
abilu_status abilu_batch_counts(abilu_batch b, int64_t *out);
abilu_status abilu_batch_set_system(abilu_batch b, int32_t s, const double *A_vals,
                                    const double *rhs, abilu_stream stream);
abilu_status abilu_batch_solve(abilu_batch b, const fgmres_opts *opts, fgmres_result *res,
                               abilu_stream stream);
abilu_status abilu_batch_get_solution(abilu_batch b, int32_t s, double *x, abilu_stream stream);
abilu_status abilu_batch_set_build_chunk(abilu_batch b, int32_t blocks);

/*
 * Continuous batching: a server whose every step solves one value update of
 * each admitted system in shared launches (the batched solve above), while
 * systems join and leave between steps.  The use it serves is the paper's:
 * each system is the Jacobian of one flow computation, its values change every
 * pseudo-time step on a fixed pattern (Sec. 2), and its factors are
 * warm-started from the previous step's (Sec. 6 setup).
 *
 * The server allocates one arena at creation, sized by abilu_server_opts (rows
 * and blocks of all admitted systems, each padded to a multiple of 64 rows with
 * identity rows; their strictly lower / upper blocks, product pairs and build
 * work items, whose defaults suit symmetric patterns; systems; the FGMRES
 * restart the Krylov workspace is sized for).  Admission and departure
 * allocate nothing in it:
 *   abilu_server_add analyses the system's pattern (rowptr/colind: device, as
 *     for abilu_pattern_create) once, into its own pattern handle, and admits
 *     it; ABILU_ENOMEM (nothing changed) when the admitted systems would no
 *     longer fit the arena.  *id (host) names the system.  Synchronises stream.
 *   abilu_server_add_pattern admits a pattern analysed beforehand by
 *     abilu_pattern_create (for example on another host thread and stream
 *     while a step runs): on success the server owns the handle (it is
 *     released with the system); on ABILU_ENOMEM the caller still owns it.
 *     No device work.
 *   abilu_server_remove releases the system's pattern handle at once; its
 *     share of the arena is free from the next step on.
 *   abilu_server_step solves, in one batched solve, one update of every
 *     admitted system: ids[k] lists each admitted system exactly once; A[q]
 *     (double[nnzb][4][4]), rhs[q] (double[n][4]) and x[q] (output, double
 *     [n][4]) are HOST arrays of pointers to device or pinned host memory.
 *     When the list differs from the previous step's, the systems are laid
 *     out again in the listed order (each analysis relocated into the arena,
 *     the factors of continuing systems moved with them).  Every step builds
 *     (opts->build must be 1) with opts' sweeps and mode: a system's first
 *     step from A, later steps from its previous factors (opts->init is not
 *     used); FGMRES from x0 = 0 per system; res[q] (host) per listed system.
 *     Synchronises stream.  Statuses as abilu_batch_solve.
 *   abilu_server_usage: host int64_t[14]: capacities (rows, blocks, L blocks,
 *     U blocks, product pairs, work items, systems), then the same quantities
 *     of the admitted systems.
 *   abilu_server_arena_bytes: the device bytes of an arena with these options
 *     (to size one to an HBM budget); no device work.
 */
typedef struct {
    int64_t max_cells;     /* rows of all admitted systems, padding included (>= 64) */
    int64_t max_blocks;    /* blocks of all admitted systems, padding included (>= 64) */
    int32_t max_systems;   /* >= 1 */
    int32_t factor_dtype;  /* abilu_dtype of the factors */
    int32_t restart;       /* the largest FGMRES(m) of the steps, 1..64 */
    int64_t max_lower;     /* strictly lower blocks; 0: max_blocks / 2 */
    int64_t max_upper;     /* strictly upper blocks; 0: max_blocks / 2 */
    int64_t max_pairs;     /* product pairs of the build; 0: max_blocks */
    int64_t max_work;      /* build work items; 0: max_blocks */
} abilu_server_opts;
typedef struct abilu_server_s *abilu_server;
abilu_status abilu_server_arena_bytes(const abilu_server_opts *opts, int64_t *bytes);
abilu_status abilu_server_create(const abilu_server_opts *opts, abilu_stream stream,
                                 abilu_server *out);
void abilu_server_destroy(abilu_server s);
abilu_status abilu_server_add(abilu_server s, int32_t n, int32_t nnzb, const int32_t *rowptr,
                              const int32_t *colind, abilu_stream stream, int32_t *id);
abilu_status abilu_server_add_pattern(abilu_server s, abilu_pattern p, int32_t *id);
abilu_status abilu_server_remove(abilu_server s, int32_t id);
abilu_status abilu_server_step(abilu_server s, int32_t k, const int32_t *ids,
                               const double *const *A, const double *const *rhs,
                               double *const *x, const fgmres_opts *opts, fgmres_result *res,
                               abilu_stream stream);
abilu_status abilu_server_usage(abilu_server s, int64_t *out);

/*
 * Orderings of the cell graph (Sec. 5), host code on host arrays.  `kind`:
 *   ABILU_ORDER_RCM       reverse Cuthill-McKee, per component (in order of
 *                         the component's lowest cell, each reversed on its
 *                         own): breadth-first from a pseudo-peripheral cell
 *                         (from the lowest cell, the last level's cell of
 *                         least degree, ties to the lowest index, while its
 *                         level structure is deeper), each cell's new
 *                         neighbours by increasing (degree, index); degrees
 *                         are those of the whole graph;
 *   ABILU_ORDER_1WD       one-way dissection: level sets of a rooted level
 *                         structure every delta = max(2, round(sqrt((3 w +
 *                         13) / 2))) levels (w = mean level width, levels
 *                         below the last) are separators; the blocks between
 *                         them, in the order of their first cell in
 *                         breadth-first order, are numbered first (each by
 *                         RCM from that cell), the separators of all
 *                         components last; a component with fewer than
 *                         2 delta + 1 levels is numbered by RCM;
 *   ABILU_ORDER_LINE      lines of strongly coupled cells (Sec. 5.1) made
 *                         contiguous, each at the position of its first cell;
 *   ABILU_ORDER_LINE_RCM, ABILU_ORDER_LINE_1WD  the graph of lines and
 *                         single cells (Sec. 5.2) ordered by RCM / 1WD, every
 *                         line expanded in place.
 * Lines: a cell is anisotropic when its strongest coupling is at least
 * `line_threshold` (> 1) times its weakest; from the most anisotropic free
 * cell (ties: lowest index) a line grows forward, then backward, to the
 * strongest-coupled free neighbour (ties: lowest index) while that coupling
 * is at least `line_threshold` times the end cell's weakest coupling and at
 * least the neighbour's strongest coupling / `line_threshold`; a cell with
 * no weak coupling (a side boundary) is measured against the line's last
 * anisotropic cell, at most two such cells in a row (a third ends the line);
 * a one-cell line is dropped; lines are numbered by their lowest cell.
 * The coupling of an edge is the larger weight of its two blocks.
 * Couplings: `weights` double[nnzb] per block (e.g. geometric), else the
 * Frobenius norms of `vals` double[nnzb][4][4]; one of them is required for
 * the line kinds, both may be NULL otherwise.  rowptr int32[n+1], colind
 * int32[nnzb] (the block pattern; symmetrised internally).  Output perm
 * int32[n]: perm[k] = the old index of the cell numbered k; line_of (may be
 * NULL) int32[n]: each old cell's line index, -1 for cells in no line.  All
 * pointers are HOST pointers; no device work.  ABILU_EINVAL on bad input.
 */
typedef enum {
    ABILU_ORDER_RCM = 0,
    ABILU_ORDER_1WD = 1,
    ABILU_ORDER_LINE = 2,
    ABILU_ORDER_LINE_RCM = 3,
    ABILU_ORDER_LINE_1WD = 4
} abilu_ordering;
abilu_status abilu_order(int32_t n, const int32_t *rowptr, const int32_t *colind,
                         const double *weights, const double *vals, int32_t kind,
                         double line_threshold, int32_t *perm, int32_t *line_of);

/*
 * The pattern renumbered by perm (as abilu_order returns it): row k of the
 * result is old row perm[k] with its columns renumbered and sorted.  HOST
 * arrays: rowptr_out int32[n+1], colind_out int32[nnzb], src_out int32[nnzb]
 * (the old position of each new block, for abilu_gather_blocks).
 */
abilu_status abilu_permute_pattern(int32_t n, const int32_t *rowptr, const int32_t *colind,
                                   const int32_t *perm, int32_t *rowptr_out, int32_t *colind_out,
                                   int32_t *src_out);

/* vals_out[p] = vals_in[src[p]] for p < nnzb (4x4 FP64 blocks), on the device:
 * the block values in a renumbered pattern.  Device pointers, distinct arrays. */
abilu_status abilu_gather_blocks(int64_t nnzb, const int32_t *src, const double *vals_in,
                                 double *vals_out, abilu_stream stream);

/*
 * abilu_add_block_diagonal — A_out = A_in + diag(d_i) on every diagonal block:
 * A_out[diag of row i][c][c] = A_in[...][c][c] + d[i][c], every other entry
 * copied.  The pseudo-time matrix M_tau + dr/dw of Sec. 2 (Eq. pseudotimestep)
 * is assembled this way each step, the shift being V_i / dtau_i (and any
 * diagonal part of the Jacobian that changes with the state).  A_in, A_out:
 * double[nnzb][4][4] in the pattern's layout (they may be the same array);
 * d: double[n][4].  Device pointers, caller-owned.  Asynchronous on `stream`.
 */
abilu_status abilu_add_block_diagonal(abilu_pattern p, const double *A_in, double *A_out,
                                      const double *d, abilu_stream stream);

/*
 * abilu_to_f32 — out[i] = in[i] rounded to FP32, round to nearest even, for
 * i < n: the conversion FGMRES uses to hand the normalised Krylov vector to
 * FP32/BF16 preconditioners, done with integer instructions only (this GPU's
 * hardware FP64->FP32 conversion runs on its FP64 pipe).  A utility outside
 * the paper's method; it gives IEEE results for every input (subnormal
 * results, overflow to Inf, quiet NaN).  in: double[n], out: float[n], device,
 * caller-owned, 8- and 4-byte aligned.  n >= 0.  Asynchronous on `stream`.
 */
abilu_status abilu_to_f32(const double *in, float *out, int64_t n, abilu_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* ABILU_H */
