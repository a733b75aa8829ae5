// nsli_internal.h -- layouts shared by the host library and the kernels.
//
// Device layout of one problem (all buffers owned by the handle):
//   A      m rows x ld elements of the storage type, row-major, each row
//          zero-padded from n to ld so that a row is a whole number of
//          16-byte vectors (the unit of the bulk copies and of the loads).
//   meta   one 32-byte record per row: b0_i, (Av)_i, 1/||a_i||^2, 1/||a_i||
//          and the FP8 row scale, in the accumulation type; the Map streams
//          it beside the row.
//   b0_64, av_64, n2_64   binary64 copies for the binary64 check.
//   x64    ld binary64 elements: the iterate itself, updated in binary64.
//   x      ld elements of the accumulation type, the rounding of x64 that the
//          Map reads (for binary64 storage the same buffer as x64).
//   part_y G x ld partial sums of the positive slices, one row per CTA of
//          the Map; part_stat G records (h, max r, max r/||a||, max |b|).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace nsli {

struct RowMeta32 {
    float b0, av, inv_n2, inv_n, scale, pad0, pad1, pad2;
};
struct RowMeta64 {
    double b0, av, inv_n2, inv_n;
};
static_assert(sizeof(RowMeta32) == 32, "row record is 32 bytes");
static_assert(sizeof(RowMeta64) == 32, "row record is 32 bytes");

struct PartStat {
    long long h;
    double maxviol, maxnorm, maxb;
};

// Device-resident state of the iteration; the kernels read the control
// fields at run time so one captured graph serves every solve.
struct DevState {
    // control, written by the host before a run
    double lambda, eps, rho;
    long long max_iter;   // absolute bound on `it`
    int rule, stop, force_step;
    int hold_tick;        // 1: ticks are set from outside (wall clock), not per iteration
    // progress, written by the kernels
    long long it;         // x-updates performed in this run
    long long tick;       // k of b(k)
    int done;             // non-zero: every kernel returns at once
    int status;           // ST_RUNNING, ST_CANDIDATE, 0 = OK, 1 = NOT_CONVERGED
    int error;            // ERRF_* bits
    unsigned int ticket;  // last-block counter of the reduce kernel
    long long h;          // stats of the last Map
    double maxviol, maxnorm, maxb;
    double dx2;           // ||dx||^2 of the last step (its root is taken by the host)
    double y_norm;
};

// The step rule ||dx|| < eps from ||dx||^2 (binary64 square roots are long
// dependency chains on GB300): the root is needed only when dx^2 is not
// above 4 eps^2, i.e. when ||dx|| could be below eps.
__host__ __device__ __forceinline__ bool step_norm_below(double dx2, double eps)
{
    const double e2 = eps * eps;
    if (dx2 > 4.0 * e2 && !(e2 < 1e-300))
        return false;
    return sqrt(dx2) < eps;
}

enum : int { ST_RUNNING = 2, ST_CANDIDATE = 3 };   // reported as NSLI_RUNNING / NSLI_CANDIDATE
enum : int { ERRF_TIMEOUT = 1 };
enum : int { PREPF_ZERO_ROW = 1, PREPF_NONFINITE = 2, PREPF_TIMEOUT = 4 };

// Result of the binary64 check: maxima kept as order-preserving integers.
struct VerOut {
    unsigned long long maxviol, maxnorm, maxb;
    unsigned long long h;
};

struct MapArgs {
    const void *A;
    const void *meta;
    const void *x;
    void *part_y;
    PartStat *part_stat;
    DevState *st;
    long long ld;          // elements per stored row
    long long m;
    long long rows_base;   // rows per CTA = rows_base (+1 for the first rows_rem)
    int rows_rem;
    int nv;                // 16-byte vectors per stored row
    int row_bytes;
    int rows_per_slot;     // R
    int nstage;
    int stage_stride;      // bytes per stage in shared memory
    int ignore_done;       // run even when the done flag is set
    int skip_slot;         // failure injection: CTA 0 never issues this slot (-1: none)
    int cluster;           // long rows on thread-block clusters: CTAs per cluster (0: not used)
    int slice_nv;          // ... 16-byte vectors of a row per CTA of a cluster
    int cluster_vpt;       // ... vectors per thread (instance of the cluster kernel)
    int cluster_lag;       // ... row groups between a group's Map and the wait for its exchange (1..3)
    int cluster_rg;        // ... rows per group (1, or 2 for bf16 / FP8)
};

struct ReduceArgs {
    const void *part_y;
    const PartStat *part_stat;
    void *x;               // accumulation-type copy read by the Map
    double *x64;           // binary64 iterate
    double *ybuf;
    double *part_dx;
    DevState *st;
    const double *rtab;    // lambda / h for h = 0..m (written when a run begins); NULL: divide
    long long ld;
    int G;
};

// Grouped launches (continuous batching): per-problem launch parameters and
// work items.  A problem's items and thread mapping depend only on itself.
struct GroupProblem {
    MapArgs map;        // rows_base / rows_rem unused; part_y has one row per item
    ReduceArgs red;     // G = number of items of the problem
    int nt, vpt;        // Map threads owning vectors, vectors per thread
    int red_blocks;     // reduce blocks of this problem
    int first_red;      // index of its first block in the grouped reduce launch
};
struct GroupItem {
    int prob;           // index into the GroupProblem array
    int part;           // index of the item within its problem
    long long row_begin, row_end;
};
struct GroupRed {
    int prob;
    int blk;            // block index within the problem
};

// Persistent serving (one launch iterates all live problems of a pool for
// many rounds).  ServeCtrl lives in pinned, mapped host memory: the host
// raises `yield`, the kernel publishes the problems that stopped (done[],
// done_count) and the rounds it ran.
struct ServeDone {
    int prob;            // index into the launch's problem table
    int status;          // ST_CANDIDATE, NSLI_OK or NSLI_NOT_CONVERGED
    long long it;        // x-updates made in the problem's run
};
constexpr int kServeMaxProblems = 4096;
struct ServeCtrl {
    int yield;                    // host -> kernel: end at the next round boundary
    int error;                    // kernel -> host: a grid barrier wait expired
    unsigned long long rounds;    // kernel -> host: rounds completed
    unsigned int done_count;      // kernel -> host: entries of done[] written
    unsigned int pad;
    ServeDone done[kServeMaxProblems];
};
// Device-side scratch of one launch (zeroed before it).
struct ServeSync {
    unsigned int bar_count, bar_gen;  // grid barrier
    unsigned int ndone;               // completions reported
    int stop;                         // decision of the control phase
    unsigned int map_next, red_next;  // next Map / Reduce item to take (reset every round)
};
struct ServeArgs {
    const GroupProblem *probs;
    const GroupItem *items;
    const GroupRed *reds;
    int nprob, nitems, nreds;
    long long *tick0;          // nprob: each problem's tick when the launch began
    int *reported;             // nprob: stop already reported (or stopped before the launch)
    ServeSync *sync;
    ServeCtrl *ctrl;           // host-mapped
    long long max_rounds;
    unsigned long long max_ns; // wall-clock bound of the launch
    unsigned long long tick_ns;  // > 0: tick = tick0 + (now - launch) / tick_ns
};

struct VerifyArgs {
    const void *A;
    const double *x64;
    const double *b0_64, *av_64, *n2_64;
    const float *scale;    // per-row FP8 scale (NULL otherwise)
    const DevState *st;
    VerOut *out;
    long long ld, m;
    int nv;
};

// ---- launchers (nsli_kernels.cu) -------------------------------------------
constexpr int kMapMaxConsumers = 512;
constexpr int kMapRowGroup = 8;      // most rows reduced per block barrier
constexpr int kReduceCols = 32;      // columns per reduce block
constexpr int kSmemHeader = 2432;    // barriers, flags, warp-sum buffers

// rows per block barrier of the Map kernel for a vectors-per-thread count;
// a ring slot always holds a multiple of it
// (eight for one vector per thread with binary32 accumulation: short rows,
// whose fixed cost per barrier would otherwise dominate; the two halves of
// the warp-sum buffer hold 1024 bytes each)
__host__ __device__ constexpr int map_rows_per_group(int vpt, int acc_bytes)
{
    return vpt >= 8 ? 1 : (vpt >= 4 ? 2 : (vpt >= 2 || acc_bytes > 4 ? 4 : 8));
}

int map_vpt_limit(int storage);      // largest vectors-per-thread instance
// guard: some thread's vectors fall outside the row (nv < threads * vpt)
cudaError_t map_prepare(int storage, int vpt, bool guard, size_t smem);
cudaError_t map_launch(int storage, int vpt, bool guard, int grid, int consumers, size_t smem,
                       cudaStream_t s, const MapArgs &a);
// long rows on clusters of C CTAs: set the kernel's shared memory and return
// how many clusters can be resident at once (0: the shape does not fit)
cudaError_t cluster_prepare(int storage, int vpt, int rg, int C, size_t smem, int *clusters);
cudaError_t reduce_launch(bool f64, int grid, cudaStream_t s, const ReduceArgs &a);
cudaError_t reduce_only_launch(bool f64, int grid, cudaStream_t s, const ReduceArgs &a,
                               double *y_out);
cudaError_t verify_launch(int storage, int grid, cudaStream_t s, const VerifyArgs &a);
// grouped launches over the problems of a pool (one storage type)
cudaError_t map_group_prepare(int storage, size_t smem);
cudaError_t map_group_launch(int storage, int items, size_t smem, cudaStream_t s, const GroupProblem *probs,
                             const GroupItem *it);
cudaError_t reduce_group_launch(bool f64, int blocks, cudaStream_t s, const GroupProblem *probs,
                                const GroupRed *tab);

// persistent serving: cooperative launch of `grid` CTAs (at most one wave)
cudaError_t serve_prepare(int storage, size_t smem, int *blocks_per_sm);
cudaError_t serve_launch(int storage, int grid, size_t smem, cudaStream_t s, const ServeArgs &a);

struct PrepArgs {
    const void *src;        // staged source rows (device), row pitch lda
    long long lda;
    int src_f64;
    void *A;                // destination rows (storage type), pitch ld
    long long ld, n;
    long long row0, rows;   // rows of this launch (global index row0)
    const double *norms_in; // optional user norms (global index)
    double *n2_64;          // receives ||a_i||^2 (global index)
    float *scale;           // FP8 row scale (global index) or NULL
    int *flags;
    int fast;               // 1: the quick norm for the row records (no binary64
                            // work per entry); 0: the binary64-accurate norm
};
cudaError_t prep_launch(int storage, cudaStream_t s, const PrepArgs &a);
// binary64-accurate ||a_i||^2 of the STORED rows (same value the set-up
// kernel gives with fast = 0), for the binary64 check (nsli_update.cu)
cudaError_t stored_norms64_launch(int storage, cudaStream_t s, const void *A, const float *scale, long long ld,
                                  long long n, long long m, double *n2_64);

// rows row0 .. row0 + rows - 1 replaced from src (device, pitch lda, binary32
// or binary64); b0_new (device, rows values) or NULL keeps b0 (nsli_update.cu)
struct UpdateArgs {
    const void *src;
    long long lda;
    int src_f64;
    void *A;
    long long ld, n;
    long long row0, rows;
    const double *b0_new;
    double *b0_64;
    const double *av_64;
    double *n2_64;       // receives the quick norm of each updated row (row records)
    float *scale;
    void *meta;
    int *flags;
};
cudaError_t update_rows_launch(int storage, cudaStream_t s, const UpdateArgs &a);

struct MetaArgs {
    void *meta;
    const double *b0_64, *av_64, *n2_64;
    const float *scale;
    long long m;            // rows [row0, row0 + m)
    int *flags;
    long long row0 = 0;
};
cudaError_t meta_launch(bool f64, cudaStream_t s, const MetaArgs &a);
// only the records' b0 (a new right-hand side)
cudaError_t meta_b0_launch(bool f64, cudaStream_t s, const MetaArgs &a);

// x64[j] = src[j] (j < n), 0 up to ld; x = x64 rounded to the accumulation type
cudaError_t x_from_f64_launch(bool f64, cudaStream_t s, const double *src, double *x64, void *x,
                              long long n, long long ld, int *flags);
cudaError_t check_finite_launch(cudaStream_t s, const double *v, long long n, int *flags);

struct StateBegin {
    double lambda, eps, rho;
    long long max_iter;
    int rule, stop;
    int reset_it;        // 1: it = 0
    int force_step;
    long long tick;      // >= 0: set the tick
    double *rtab;        // non-NULL: write lambda / h to rtab[h], h = 0..rtab_m (0 for h = 0)
    long long rtab_m;
};
cudaError_t state_begin_launch(cudaStream_t s, DevState *st, const StateBegin &b);
cudaError_t state_resume_launch(cudaStream_t s, DevState *st);
// sts[i]->tick = ticks[i] and ticks held (device arrays of count entries)
cudaError_t set_ticks_launch(cudaStream_t s, DevState *const *sts, const long long *ticks, int count);
cudaError_t stored_rows_launch(int storage, cudaStream_t s, const void *A, const float *scale, long long ld,
                               long long n, long long row0, long long rows, double *out);

// ---- row shards (nsli_shard.cu) ---------------------------------------------
// A worker's record: h, max r_i, max r_i / ||a_i||, max |b_i| (doubles),
// then y (n doubles); see include/nsli.h.
constexpr int kShardHeader = 4;
struct ShardStepArgs {
    const double *recs;   // nranks records of n + kShardHeader doubles, worker order
    int nranks;
    long long n;
    void *x;              // accumulation-type copy read by the Map
    double *x64;          // binary64 iterate
    double *ybuf;         // n doubles (ModAP: the global y)
    double *part_dx;      // shard_step_blocks(n) partial sums
    DevState *st;
};
int shard_step_blocks(long long n);
cudaError_t shard_pack_launch(cudaStream_t s, const DevState *st, const double *ybuf, long long n, double *rec);
cudaError_t shard_step_launch(bool f64, cudaStream_t s, const ShardStepArgs &a);

// ---- sparse A (nsli_sparse.cu) ----------------------------------------------
// A held as CSR (rows, for the residuals) and CSC (columns, for y), values
// in the storage type (binary64 or binary32), indices int32, offsets int64.

// One CTA's piece of a heavy row (column): entries [e0, e1) of segment seg,
// piece k of npieces; the partial sums of the segment's pieces go to slots
// first .. first + npieces - 1; hs indexes the segment's arrival counter.
struct SegPiece {
    int seg, hs, first, npieces, k, pad;
    long long e0, e1;
};
constexpr int kSparsePiece = 2048;   // entries per heavy piece
#ifndef NSLI_SPARSE_KU
#define NSLI_SPARSE_KU 4
#endif
constexpr int kSparseU = NSLI_SPARSE_KU;  // independent loads per lane per chunk

struct SparseArgs {
    const long long *rp;      // m + 1 row offsets
    const int *ci;            // nnz column indices, ascending within a row
    const void *va;           // nnz values in row order
    const long long *cp;      // n + 1 column offsets
    const int *ri;            // nnz row indices, ascending within a column
    const void *vc;           // nnz values in column order
    const void *meta;         // m row records (RowMeta32 / RowMeta64)
    const SegPiece *row_pieces;  // pieces of rows longer than heavy_thr_row
    const SegPiece *col_pieces;  // pieces of columns longer than heavy_thr_col
    void *row_slots, *col_slots; // partial sums of the pieces (accumulation type)
    int *row_cnt, *col_cnt;      // per heavy segment arrival counters (zero between launches)
    void *coef;               // m: max(r_i, 0) / ||a_i||^2, accumulation type
    void *x;                  // n, accumulation type
    double *x64;              // n, the binary64 iterate
    double *ybuf;             // n: y (ModAP, and the Map-only call)
    PartStat *part_stat;      // one record per row-pass CTA
    double *part_dx;          // one partial sum per column / step CTA
    DevState *st;
    long long m, n;
    long long light_rows_per_cta, light_cols_per_cta;
    long long heavy_thr_row, heavy_thr_col;
    int n_row_pieces, n_col_pieces;
    int row_light_ctas, col_light_ctas, step_ctas;
    int w_row, w_col;         // lanes per row / column (1, 2, 4, ..., 32)
    int ignore_done;          // run even when the done flag is set
    int mode;                 // 0: iteration; 1: Map and y only (no decision, no step)
    const double *rtab;       // lambda / h for h = 0..m (written when a run begins)
    // one-CTA runs of small systems (sparse_resident_kernel): the rows and
    // columns with more than kResLong entries, taken by one warp each
    const int *res_long_rows, *res_long_cols;
    int n_res_long_rows, n_res_long_cols;
};
// resident CTAs per SM of the row / column kernel instances for these widths
void sparse_blocks_per_sm(bool f64, int w_row, int w_col, int *row_bps, int *col_bps);
cudaError_t sparse_row_launch(bool f64, cudaStream_t s, const SparseArgs &a);
cudaError_t sparse_col_launch(bool f64, cudaStream_t s, const SparseArgs &a);
cudaError_t sparse_step_launch(bool f64, cudaStream_t s, const SparseArgs &a);
cudaError_t sparse_norms_launch(bool f64, int grid, cudaStream_t s, const SparseArgs &a, double *n2, int *flags);
cudaError_t sparse_verify_launch(bool f64, int grid, cudaStream_t s, const SparseArgs &a, const VerifyArgs &v);
cudaError_t sparse_rows_launch(bool f64, cudaStream_t s, const SparseArgs &a, long long row0, long long rows,
                               double *out);

// Small systems: a block of up to `iters` iterations (mode 0) in one launch
// of one CTA whose shared memory holds x64, y, x and c.
constexpr int kResThreads = 256;
constexpr int kResLong = 32;             // longer rows / columns go to a warp each
constexpr size_t kResSmemMax = 216 * 1024;
constexpr int kResBlock = 1024;          // iterations per launch unless block_iters says otherwise
size_t sparse_resident_smem(bool f64, long long m, long long n);
cudaError_t sparse_resident_prepare(bool f64, size_t smem);
cudaError_t sparse_resident_launch(bool f64, cudaStream_t s, const SparseArgs &a, size_t smem, int iters);

}  // namespace nsli
