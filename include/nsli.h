/*
 * nsli.h -- C ABI of the GB300 pseudo-projection solver for (non-stationary)
 * systems of linear inequalities A x <= b(t).
 *
 * Method: Sokolinsky & Sokolinskaya, "Scalable Parallel Algorithm for Solving
 * Non-stationary Systems of Linear Inequalities" (2020).
 *   Section 2, Eq. 7   positive slice  rho+_i(x) = max(<a_i,x> - b_i, 0) / ||a_i||^2 * a_i
 *   Section 2, Eq. 8   phi(x) = y / h, y = sum_i rho+_i(x), h = #non-zero slices
 *   Section 2, Eq. 10  eps-membership: for all i, r_i <= 0 or |r_i| / ||a_i|| < eps
 *   Section 2, Eq. 12  ModAP step psi(x) = lambda * phi / ||phi|| = lambda * y / ||y||
 *   Section 3, Eq. 13  the Map F_x(a_i, b_i) = rho+_i(x), then Reduce(+)
 *   Section 5          non-stationarity as a translation of the polytope
 *
 * One iteration (the "hot path"):
 *   b_i(k) = b0_i + k * rho * (A v)_i                      (tick; fused into the Map)
 *   r_i = <a_i, x> - b_i(k);  y = sum_{r_i > 0} r_i / ||a_i||^2 * a_i;  h = #{r_i > 0}
 *   stopping test on (x_k, b(k)); then
 *   RELAXED: x <- x - lambda * y / h        (Algorithm 1, Eq. 8 with relaxation lambda)
 *   MODAP:   x <- x - lambda * y / ||y||    (Eq. 12)
 *   k <- k + 1
 *
 * Conventions for every call:
 *   - Every function returns an int status (NSLI_OK = 0, > 0 informational,
 *     < 0 error) and never aborts the process.
 *   - Pointers marked "host or device" may point to host memory (pageable or
 *     pinned) or to device memory of the handle's device; the library detects
 *     which.  Arrays are dense, contiguous, in the element type stated.
 *   - All device work of a handle is issued on the stream given to
 *     nsli_create; calls that return host results synchronise that stream.
 *   - A handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef NSLI_H
#define NSLI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nsli_solver *nsli_handle;

/* element types: storage of A on the device, and source type of A */
enum {
    NSLI_F64 = 0,      /* IEEE binary64; the Map accumulates in binary64   */
    NSLI_F32 = 1,      /* IEEE binary32; the Map accumulates in binary32   */
    NSLI_BF16 = 2,     /* bfloat16 (round-to-nearest-even from binary32)   */
    NSLI_FP8E4M3 = 3   /* FP8 E4M3 codes with a power-of-two scale per row */
};

/* step rules */
enum {
    NSLI_RULE_RELAXED = 0, /* x <- x - lambda * y / h      (Eq. 8)  */
    NSLI_RULE_MODAP = 1    /* x <- x - lambda * y / ||y||  (Eq. 12) */
};

/* stopping rules, evaluated on the Map at (x_k, b(k)) at the top of each
 * iteration (STEP after the update) */
enum {
    NSLI_STOP_NONE = 0,        /* no test: run a fixed number of iterations  */
    NSLI_STOP_STEP = 1,        /* ||x_{k+1} - x_k|| < eps, or h == 0          */
    NSLI_STOP_EPSMEM = 2,      /* Eq. 10: max_i r_i / ||a_i|| < eps           */
    NSLI_STOP_MAXVIOL_REL = 3  /* max_i r_i <= eps * max_i |b_i(k)|           */
};

/* status and return codes */
enum {
    NSLI_OK = 0,
    NSLI_NOT_CONVERGED = 1,    /* max_iter reached without the stop rule     */
    NSLI_RUNNING = 2,          /* nsli_get_result only: the run goes on       */
    NSLI_CANDIDATE = 3,        /* nsli_get_result only: the stop test passed in
                                  the accumulation type; the binary64 check
                                  (nsli_residual_max) decides                */
    NSLI_ERR_ARG = -1,         /* invalid argument                           */
    NSLI_ERR_ZERO_ROW = -2,    /* a row of A is zero (the method needs a_i != 0) */
    NSLI_ERR_NONFINITE = -3,   /* NaN or Inf in A, b, Av, x or norms         */
    NSLI_ERR_OOM = -4,         /* device allocation failed                   */
    NSLI_ERR_CUDA = -5,        /* a CUDA runtime call failed (see nsli_last_error) */
    NSLI_ERR_TIMEOUT = -6,     /* a bounded device wait expired              */
    NSLI_ERR_UNSUPPORTED = -7  /* valid but outside this library's limits    */
};

typedef struct {
    double lambda;       /* step length / relaxation, > 0                          */
    int32_t rule;        /* NSLI_RULE_*                                             */
    int32_t stop;        /* NSLI_STOP_*                                             */
    double eps;          /* threshold of the stopping rule, >= 0                   */
    int64_t max_iter;    /* nsli_solve: maximum number of x-updates, >= 0           */
    int32_t block_iters; /* iterations per captured CUDA graph (0: 32); for a small
                            sparse system run on one CTA, iterations per launch
                            (0: 1024)                                                */
    int32_t reserved;    /* must be 0                                               */
    double rho;          /* translation per tick: b(k) = b0 + k * rho * Av          */
} nsli_params;

typedef struct {
    int64_t iters;            /* x-updates performed by this call               */
    int64_t tick;             /* tick k after the call                          */
    int32_t status;           /* NSLI_OK, NSLI_NOT_CONVERGED or an error code   */
    int32_t rejected;         /* nsli_solve: stop candidates of the accumulation
                                 type that the binary64 check rejected      */
    int64_t h;                /* violated rows at the final point (binary64 check) */
    double max_viol;          /* max_i (a_i.x - b_i(k)), binary64, stored A      */
    double max_viol_norm;     /* max_i (a_i.x - b_i(k)) / ||a_i||, binary64      */
    double max_abs_b;         /* max_i |b_i(k)|                                  */
    double last_step_norm;    /* ||x_k - x_{k-1}|| of the last update, binary64 */
} nsli_result;

/* Create a solver for the m x n system A x <= b0 + k rho Av.
 *   storage   NSLI_F64 / NSLI_F32 / NSLI_BF16 / NSLI_FP8E4M3: how A is held on
 *             the device.  BF16 rounds each binary32 entry to nearest even;
 *             FP8E4M3 stores e4m3(a_ij / s_i) with s_i the smallest power of
 *             two such that max_j |a_ij| / s_i <= 448 (saturating, nearest
 *             even).  The solved system is the stored one.
 *   a_dtype   NSLI_F64 or NSLI_F32: element type of the source A.  BF16 and
 *             FP8E4M3 storage need an NSLI_F32 source.
 *   A         host or device, row-major, m rows of lda elements (lda >= n);
 *             copied, not retained.
 *   b0        host or device, m doubles: right-hand side at tick 0.
 *   norms2    host or device, m doubles ||a_i||^2, or NULL to compute them
 *             in binary64 on the device from the stored entries.
 *   Av        host or device, m doubles (A v for the translation direction
 *             v), or NULL for a stationary right-hand side.
 *   x0        host or device, n doubles: the starting point.  The iterate is
 *             kept and updated in binary64; the Map reads its rounding to the
 *             accumulation type (binary32 unless storage is NSLI_F64).
 *   stream    a cudaStream_t on the current device (not the legacy default
 *             stream: iteration blocks are captured into CUDA graphs), or
 *             NULL to let the handle create and own a non-blocking stream.
 * Errors: NSLI_ERR_ARG (m, n < 1, lda < n, bad enum, NULL required pointer),
 * NSLI_ERR_ZERO_ROW, NSLI_ERR_NONFINITE, NSLI_ERR_OOM, NSLI_ERR_CUDA.  Rows
 * up to 16384 entries (binary32 / bf16 / fp8; 8192 for binary64) are held
 * in registers while streamed through shared memory; longer rows use a
 * chunked two-pass Map that re-reads violated rows from L2.  On error *out is NULL
 * and nothing is leaked.  The handle owns all its device memory until
 * nsli_destroy. */
int nsli_create(nsli_handle *out, int64_t m, int64_t n, int32_t storage,
                int32_t a_dtype, const void *A, int64_t lda, const double *b0,
                const double *norms2, const double *Av, const double *x0,
                void *stream);

/* Create a solver for a SPARSE m x n system A x <= b0 + k rho Av (the same
 * method, Sections 2, 3 and 5; the paper's test system, Section 5, has a
 * few non-zeros per row).  A is given in compressed-row form:
 *   row_ptr   host or device, m + 1 int64 offsets, row_ptr[0] = 0,
 *             non-decreasing, row_ptr[m] = nnz;
 *   col_idx   host or device, nnz int32 column indices, strictly increasing
 *             within each row (no duplicates), each in [0, n);
 *   val       host or device, nnz doubles, the entries in the same order.
 *   storage   NSLI_F64 or NSLI_F32 (entries rounded to nearest even);
 *             others give NSLI_ERR_UNSUPPORTED.
 * b0, norms2, Av, x0 and stream as for nsli_create.  The library keeps A
 * twice on the device, by rows (for the residuals) and by columns (so every
 * y_j is summed in one fixed order, rows ascending: results are bitwise
 * reproducible), about 2 nnz (4 + element size) bytes.  The structure is
 * copied and checked on the host; nothing is retained.  Every other call
 * on the handle works as for a dense one, except nsli_test_inject_timeout
 * (NSLI_ERR_UNSUPPORTED); a ModAP iteration is three kernel launches
 * instead of two.  A small system (x, the coefficients and a table of
 * lambda / h fit in one CTA's shared memory, and the matrix fits with them in
 * one SM's on-chip memory) is iterated by nsli_iterate and nsli_solve on one
 * CTA, a whole block of iterations per launch (same steps and decisions; its
 * own fixed summation order, so not bit-identical to the grid kernels, and
 * bit-identical however a run is split into launches); the environment
 * variable NSLI_SPARSE_RESIDENT=0 (=1) at creation turns this off (forces
 * it wherever the shared memory suffices).  Errors: NSLI_ERR_ARG (sizes < 1, NULL required pointer,
 * malformed offsets or indices), NSLI_ERR_UNSUPPORTED (storage, m or n
 * >= 2^31), NSLI_ERR_ZERO_ROW (an empty or all-zero row),
 * NSLI_ERR_NONFINITE, NSLI_ERR_OOM, NSLI_ERR_CUDA.  On error *out is NULL
 * and nothing is leaked. */
int nsli_create_csr(nsli_handle *out, int64_t m, int64_t n, int32_t storage,
                    int64_t nnz, const int64_t *row_ptr, const int32_t *col_idx,
                    const double *val, const double *b0, const double *norms2,
                    const double *Av, const double *x0, void *stream);

/* Replace b0 (host or device, m doubles; NULL keeps the current b0) and set
 * the tick k used by the next iteration (tick < 0 keeps the current tick).
 * Section 5: the data update step of each iteration. */
int nsli_update_b(nsli_handle h, const double *b0, int64_t tick);

/* Replace rows row0 .. row0 + rows - 1 of A (and optionally their b0)
 * between iterations: the data update step of Section 3 for a system whose
 * matrix changes with time (Eq. 1; Section 4 prices a full change at
 * (n + 1) m values).  Issued on the handle's stream after the work already
 * queued, so the next iteration sees the new rows.
 *   a_dtype  NSLI_F32 or NSLI_F64: element type of the new rows (BF16 and
 *            FP8E4M3 storage need NSLI_F32).
 *   A        host or device, row-major, rows rows of lda elements
 *            (lda >= n); row q replaces row row0 + q; copied, not retained.
 *   b0       host or device, rows doubles: new right-hand sides at tick 0 of
 *            the same rows, or NULL to keep them.
 * The rows are stored, normed (binary64, from the stored values) and their
 * records rebuilt exactly as nsli_create does.  A row that holds a NaN / Inf
 * (or whose new b0 does, or a value that rounds to infinity in bf16) or is
 * all zeros keeps its previous values; the call then returns
 * NSLI_ERR_NONFINITE or NSLI_ERR_ZERO_ROW after updating the other rows.
 * Other errors: NSLI_ERR_ARG (range outside [0, m), NULL A, lda < n,
 * dtype), NSLI_ERR_UNSUPPORTED (a sparse handle), NSLI_ERR_TIMEOUT (a
 * device copy of a source row did not arrive within the bounded wait; that
 * row keeps its previous values), NSLI_ERR_OOM / NSLI_ERR_CUDA.
 * Synchronises (it reads the row flags back). */
int nsli_update_rows(nsli_handle h, int64_t row0, int64_t rows,
                     int32_t a_dtype, const void *A, int64_t lda,
                     const double *b0);

/* Run exactly n_iter iterations (Map, Reduce, step, tick) with no stopping
 * test (p->stop is ignored); an iteration with h == 0 makes no step.  Issues
 * the work asynchronously on the handle's stream and returns without
 * synchronising.  n_iter >= 0. */
int nsli_iterate(nsli_handle h, const nsli_params *p, int64_t n_iter);

/* The same n_iter iterations as nsli_iterate, launched kernel by kernel
 * with a CUDA event pair around every kernel on the handle's stream.
 * kernel_ms[0] receives the summed device time of the Map kernels and
 * kernel_ms[1] that of the Reduce-and-step kernels, in milliseconds.
 * Synchronises.  For attributing time to kernels (roofline figures). */
int nsli_iterate_timed(nsli_handle h, const nsli_params *p, int64_t n_iter,
                       double *kernel_ms);

/* Iterate until the stopping rule holds or p->max_iter x-updates were made.
 * Tests taken in binary32 are confirmed in binary64 on the stored A (the
 * binary64 check decides; a rejected candidate costs one more iteration).
 * Synchronises.  out receives the final binary64 check.  Returns out->status. */
int nsli_solve(nsli_handle h, const nsli_params *p, nsli_result *out);

/* Binary64 feasibility check of the current x against the stored A and
 * b(k) at the current tick (Eq. 10): max_i r_i and max_i r_i / ||a_i||.
 * Either output pointer may be NULL.  Synchronises. */
int nsli_residual_max(nsli_handle h, double *max_viol, double *max_viol_norm);

/* One Map + Reduce (Eq. 13, Reduce(+)) at the current x and tick, without a
 * step: y (host or device, n doubles), the violated-row count, and
 * stats[0..2] = max r_i, max r_i / ||a_i||, max |b_i| in the accumulation
 * type.  Any output may be NULL.  Synchronises. */
int nsli_map_reduce(nsli_handle h, double *y, int64_t *violated, double *stats);

/* Copy the current x out (host or device, n doubles) / set it. Synchronise. */
int nsli_get_x(nsli_handle h, double *x);
int nsli_set_x(nsli_handle h, const double *x);

/* Diagnostics: the exact values of stored rows row0 .. row0+rows-1 as
 * doubles (FP8 storage: code * row scale), written row-major with n values
 * per row to `out` (host or device, rows * n doubles), and the binary64
 * ||a_i||^2 the solver uses (host or device, m doubles).  Synchronise. */
int nsli_get_stored_rows(nsli_handle h, int64_t row0, int64_t rows, double *out);
int nsli_get_norms2(nsli_handle h, double *out);

/* Failure-detection test (no GPU fault): one Map launch in which CTA 0 never
 * issues the bulk copy of its row slot `slot`, so its threads wait on a
 * barrier that nothing completes.  The bounded waits (about two seconds)
 * expire, the CTA records the timeout, waits (bounded) for its other copies
 * and returns.  Returns NSLI_ERR_TIMEOUT when detection works (NSLI_OK if
 * slot is beyond CTA 0's rows); the handle stays usable.  Synchronises. */
int nsli_test_inject_timeout(nsli_handle h, int32_t slot);

/* Progress of the last nsli_iterate / nsli_solve / sharded run (device
 * state): status NSLI_RUNNING while a run can go on, NSLI_CANDIDATE after a
 * stop test passed in the accumulation type and before a binary64 check
 * decided, else NSLI_OK / NSLI_NOT_CONVERGED.  The binary64 fields of out
 * are those of the last check made, or 0.  Synchronises. */
int nsli_get_result(nsli_handle h, nsli_result *out);

/* ---- Row shards: ModAPL (Section 3) ----
 * Section 3 splits the list of inequalities among workers: each worker maps
 * and reduces its own sublist, the partial results are added, and the step
 * is taken with the sums.  Here each worker is a handle created (as usual,
 * with nsli_create / nsli_create_csr) over a contiguous block of rows of
 * the whole system, with the same x0; normally one handle per GPU of a
 * process group.  One iteration is
 *   nsli_shard_map(h_w, rec_w)                 on every worker w,
 *   gather rec_0 .. rec_{R-1} into `records`   (an allgather, in worker order),
 *   nsli_shard_step(h_w, records, R, 0)        on every worker w.
 * A record is NSLI_SHARD_HEADER + n doubles: h_w, max_i r_i, max_i r_i /
 * ||a_i|| and max_i |b_i(k)| over the worker's rows (binary32 / bf16 / fp8
 * storage: accumulation-type values), then y_w (its Reduce, Eq. 7-8).  The
 * step adds the y_w in worker order in binary64 (a fixed order: identical
 * records give identical iterates on every worker, without a broadcast of
 * x), adds the h_w, takes the maxima, then makes the same stop decision and
 * step as nsli_iterate / nsli_solve (Eq. 8 relaxed or Eq. 12).  Results
 * differ from a single handle over all rows only by the order of the sums. */
#define NSLI_SHARD_HEADER 4

/* Set the run parameters of a sharded run on this worker (as a solve does:
 * iteration count 0, tick kept; p->max_iter bounds the updates; p->stop is
 * tested by nsli_shard_step on the combined values, a pass leaving status
 * "candidate" for the caller's binary64 check).  Call it with the same
 * parameters on every worker.  Allocates the step's partial sums on first
 * use.  Asynchronous. */
int nsli_shard_begin(nsli_handle h, const nsli_params *p);

/* Map and local Reduce of this worker's rows at its current x and tick;
 * writes the record to `record` (device memory of the handle's device,
 * NSLI_SHARD_HEADER + n doubles).  Runs even after a finished run.
 * Asynchronous on the handle's stream. */
int nsli_shard_map(nsli_handle h, double *record);

/* The global Reduce of `nranks` records (device memory, nranks x
 * (NSLI_SHARD_HEADER + n) doubles, worker order), the stop decision and the
 * step, on this worker's x.  Does nothing once the run has stopped (a
 * candidate, the step rule, or max_iter) unless force_step != 0, which
 * resumes the run and steps without testing (after a rejected candidate).
 * Progress is read with nsli_get_result.  Asynchronous on the handle's
 * stream: the records must be complete in stream order when it runs. */
int nsli_shard_step(nsli_handle h, const double *records, int32_t nranks, int32_t force_step);

/* Map + Reduce of a caller-held binary32 system that ALLOCATES NOTHING (the
 * paper has no counterpart; this is an interface for callers that cannot
 * allocate device memory: code under a fixed device-memory budget, and code
 * inside a host framework that owns all device memory through its own
 * allocator and does not let libraries call cudaMalloc).  With
 * r_i = <a_i, x> - b_i it writes
 *   y[j]       = sum over r_i > 0 of r_i / norms2[i] * a_ij   (n doubles),
 *   *violated  = #{i : r_i > 0},  *max_viol = max_i r_i  (binary32 sums).
 * Every pointer is a device pointer of the current device: A row-major, m
 * rows of lda >= n floats; b, norms2: m floats (norms2[i] = ||a_i||^2 > 0);
 * x: n floats.  Work is issued on `stream` (a cudaStream_t or NULL) and not
 * synchronised.  Scratch: a fixed 4 MiB array (plus 16 KiB of counters)
 * inside the library, held by every GPU that loads it until the process
 * exits; n larger than 2^20 is rejected with NSLI_ERR_UNSUPPORTED.  The
 * first call on a device looks up that array's device address (once per
 * device).  All calls share the
 * array and each call clears the part it accumulates into: calls that
 * overlap on the GPU race and must not be issued.  Calls no cudaMalloc or
 * cudaFree.  A CUDA error already pending when the call starts is left in
 * place and nothing is launched.  Returns NSLI_OK, NSLI_ERR_ARG,
 * NSLI_ERR_UNSUPPORTED or NSLI_ERR_CUDA. */
int nsli_map_reduce_noalloc(int64_t m, int64_t n, const float *A, int64_t lda,
                            const float *b, const float *norms2, const float *x,
                            double *y, int64_t *violated, double *max_viol,
                            void *stream);

/* ---- Batched form: P <= 64 problems sharing one matrix (tensor cores) ----
 * Problem p is A x <= b0 + (s_p + k) rho Av with its own x_p and tick
 * offset s_p; all problems advance one tick per batch iteration.  Each batch
 * iteration is the relaxed step of Algorithm 1 (Section 2, Eq. 7, Eq. 8)
 * for every problem, computed as two tensor-core contractions R = A X and
 * Y = A^T W over one bf16 copy of A (and its transpose), binary32
 * accumulation. */
typedef struct nsli_batch_solver *nsli_batch;

/* A: host or device, m x n binary32 (row pitch lda), stored as bf16 (round
 * to nearest even).  b0, Av (NULL: stationary): m doubles.  tick_offsets:
 * nprob int64 s_p (NULL: all 0).  X0: nprob x n doubles, row-major.  stream:
 * a non-default cudaStream_t or NULL (the handle then owns one).  Errors as
 * nsli_create; NSLI_ERR_UNSUPPORTED for nprob > 64. */
int nsli_batch_create(nsli_batch *out, int64_t m, int64_t n, int32_t nprob,
                      const float *A, int64_t lda, const double *b0,
                      const double *Av, const int64_t *tick_offsets,
                      const double *X0, void *stream);

/* n_iter batch iterations with lambda = p->lambda and rho = p->rho (RELAXED
 * only; other fields ignored), graph-replayed in blocks of p->block_iters
 * (0: 16).  Asynchronous. */
int nsli_batch_iterate(nsli_batch h, const nsli_params *p, int64_t n_iter);

/* One Map + Reduce for every problem at the current x and tick, no step:
 * Y (host or device, nprob x n doubles), violated (host, nprob), max_viol
 * (host, nprob; binary32 residuals).  Any output may be NULL.  Synchronises. */
int nsli_batch_map_reduce(nsli_batch h, double rho, double *Y, int64_t *violated,
                          double *max_viol);

/* Current iterates (host or device, nprob x n doubles).  Synchronises. */
int nsli_batch_get_x(nsli_batch h, double *X);

/* Binary64 check per problem (Eq. 10): max_viol[p] = max_i r_i of problem p
 * at its current tick (host, nprob doubles).  Synchronises. */
int nsli_batch_residual_max(nsli_batch h, double *max_viol);

int64_t nsli_batch_launch_count(nsli_batch h);
int nsli_batch_sync(nsli_batch h);
void nsli_batch_destroy(nsli_batch h);
const char *nsli_batch_last_error(nsli_batch h);

/* ---- Pool: continuous batching of many problems of mixed sizes ----------
 * Problems are admitted while they fit (the pool's byte budget and the
 * device's free memory), stay resident with their A, x and b across ticks,
 * and advance together: one round = ONE grouped Map launch over the row
 * blocks of every live problem + ONE grouped reduce-and-step launch.  Each
 * problem's row blocks and thread mapping depend only on itself, so its
 * iterates are bit-identical alone and in any mix.  Finished problems stop
 * costing work at once (their blocks return) and keep their x until
 * removed.  The paper's master-slave farm (Section 3) runs one problem; the
 * pool is this library's serving form of the same iteration. */
typedef struct nsli_pool_s *nsli_pool;

/* storage: NSLI_BF16 or NSLI_F32.  max_bytes: device-memory budget of the
 * pool (0: only free HBM limits admission).  stream as in nsli_create. */
int nsli_pool_create(nsli_pool *out, int32_t storage, int64_t max_bytes, void *stream);

/* Admit one problem (arguments as nsli_create with a binary32 A, norms
 * computed on the device) with its run parameters p (stop rule, eps,
 * max_iter, lambda, rule, rho).  *slot receives its id.  NSLI_ERR_OOM when
 * it does not fit: nothing is allocated and the pool is unchanged. */
int nsli_pool_add(nsli_pool pool, int64_t m, int64_t n, const float *A, int64_t lda,
                  const double *b0, const double *Av, const double *x0,
                  const nsli_params *p, int64_t *slot);

/* `rounds` iterations of every live problem (asynchronous). */
int nsli_pool_step(nsli_pool pool, int32_t rounds);

/* Wall-clock ticks: set tick k of the listed problems (slots/ticks: host
 * arrays of count entries); from then on their ticks change only here. */
int nsli_pool_set_ticks(nsli_pool pool, const int64_t *slots, const int64_t *ticks, int64_t count);

/* Synchronise, confirm binary32 stop candidates in binary64 (a rejected one
 * resumes with a forced step), and report every finished problem (status
 * NSLI_OK, NSLI_NOT_CONVERGED or an error) in slots/status/iters (host
 * arrays of cap entries); *count = number of finished problems (may exceed
 * cap). */
int nsli_pool_poll(nsli_pool pool, int64_t *slots, int32_t *status, int64_t *iters,
                   int64_t cap, int64_t *count);

/* Persistent serving: ONE launch iterates every live problem round after
 * round (Map items of all problems, grid barrier, Reduce-and-step items,
 * grid barrier, control) until nsli_pool_yield is called, no problem is
 * left running, max_rounds rounds have run, or max_seconds have passed.
 * The kernel is a cooperative launch with one CTA per SM.  tick_s > 0:
 * each problem's tick is its tick when the launch began (as set by
 * nsli_pool_set_ticks, which holds ticks) plus the wall-clock time since
 * the launch began in units of tick_s, advanced by the kernel itself; 0:
 * ticks advance per iteration unless held.  Problems that stop (a stop
 * candidate, the step rule, their max_iter) are published while the launch
 * runs through pinned host memory (nsli_pool_stopped).  While a launch
 * runs, only nsli_pool_yield, nsli_pool_stopped, nsli_pool_wait and the
 * counters may be called; the other pool calls return NSLI_ERR_ARG
 * (allocation calls are implicit device synchronisation points, so
 * admission and retirement happen between launches).  Asynchronous. */
int nsli_pool_launch(nsli_pool pool, int64_t max_rounds, double max_seconds, double tick_s);

/* Ask the running launch to end at its next round boundary (non-blocking;
 * no effect when none runs). */
int nsli_pool_yield(nsli_pool pool);

/* Problems that stopped during the running launch so far (non-blocking,
 * read from pinned host memory; 0 when no launch runs). */
int64_t nsli_pool_stopped(nsli_pool pool);

/* Wait for the running launch to end; *rounds (may be NULL) receives the
 * rounds it ran.  The next nsli_pool_poll reads only the problems it
 * reported.  NSLI_ERR_TIMEOUT if a bounded grid barrier wait expired. */
int nsli_pool_wait(nsli_pool pool, int64_t *rounds);

int nsli_pool_get_x(nsli_pool pool, int64_t slot, double *x);
int nsli_pool_residual_max(nsli_pool pool, int64_t slot, double *max_viol,
                           double *max_viol_norm);
/* Release a problem's device memory (its slot id becomes free). */
int nsli_pool_remove(nsli_pool pool, int64_t slot);
int64_t nsli_pool_live(nsli_pool pool);
int64_t nsli_pool_bytes_used(nsli_pool pool);
int64_t nsli_pool_launch_count(nsli_pool pool);
int nsli_pool_sync(nsli_pool pool);
void nsli_pool_destroy(nsli_pool pool);
const char *nsli_pool_last_error(nsli_pool pool);

/* Number of kernels the handle has launched so far (graph nodes included). */
int64_t nsli_launch_count(nsli_handle h);

/* Wait for all work of the handle. */
int nsli_sync(nsli_handle h);

/* Release every resource of the handle (NULL is allowed). */
void nsli_destroy(nsli_handle h);

/* Static description of a status code. */
const char *nsli_strerror(int code);

/* Text of the last error recorded on the handle ("" if none). */
const char *nsli_last_error(nsli_handle h);

#ifdef __cplusplus
}
#endif
#endif /* NSLI_H */
