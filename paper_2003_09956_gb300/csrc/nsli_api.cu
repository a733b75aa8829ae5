// nsli_api.cu -- host side of the C ABI declared in include/nsli.h.
//
// Owns the device buffers of one problem, picks the launch shape of the Map
// kernel from n and the storage type, captures blocks of iterations into
// CUDA graphs, and runs the solve loop (graph block, read 64-byte state,
// binary64 confirmation of candidate stops).
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "nsli.h"
#include "nsli_internal.h"

using namespace nsli;

namespace {
// An NVTX range around each ABI call, named after it, so a profiler's
// timeline shows which call issued which kernels (free without a profiler).
struct Trace {
    explicit Trace(const char *name) { nvtxRangePushA(name); }
    ~Trace() { nvtxRangePop(); }
    Trace(const Trace &) = delete;
    Trace &operator=(const Trace &) = delete;
};
}  // namespace

struct nsli_solver {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int storage = NSLI_F32;
    long long m = 0, n = 0, ld = 0;
    int elem_bytes = 4, epv = 4, row_bytes = 0, nv = 0;
    int vpt = 1, consumers = 32, R = 1, nstage = 2, stage_stride = 0;
    int cluster = 0, slice_nv = 0, cluster_vpt = 0, cluster_lag = 1, cluster_rg = 1;   // long rows on clusters
    bool guard = true;
    size_t smem = 0;
    int G = 1, red_grid = 1, num_sms = 1;
    long long rows_base = 0;
    int rows_rem = 0;

    void *A = nullptr, *meta = nullptr, *x = nullptr, *part_y = nullptr;
    double *b0_64 = nullptr, *av_64 = nullptr, *n2_64 = nullptr, *part_dx = nullptr, *ybuf = nullptr,
           *dtmp = nullptr, *x64 = nullptr;
    // ||a_i||^2 behind the row records (binary32 / bf16 / fp8 storage: the
    // quick double-float sum; otherwise the same array as n2_64), and whether
    // the binary64 norms n2_64 are up to date (they are computed from the
    // stored rows when the binary64 check or nsli_get_norms2 needs them)
    double *n2_meta = nullptr;
    bool n2_64_valid = true;
    float *scale = nullptr;
    PartStat *part_stat = nullptr;
    DevState *st = nullptr;
    VerOut *ver = nullptr;
    int *flags = nullptr;

    // lambda / h, h = 0..m, for the relaxed step (filled when a run begins
    // with a step size other than the one it holds)
    double *rtab = nullptr;
    double rtab_lambda = std::nan("");

    DevState *st_host = nullptr;  // pinned
    VerOut *ver_host = nullptr;   // pinned
    int *flags_host = nullptr;    // pinned

    // sparse A (nsli_create_csr): CSR + CSC copies, see nsli_sparse.cu
    bool sparse = false;
    long long nnz = 0;
    long long *rp = nullptr, *cp = nullptr;
    int *ci = nullptr, *ri = nullptr, *row_cnt = nullptr, *col_cnt = nullptr;
    SegPiece *row_pieces = nullptr, *col_pieces = nullptr;
    void *va = nullptr, *vc = nullptr, *coef = nullptr, *row_slots = nullptr, *col_slots = nullptr;
    SparseArgs sp{};
    // small systems: whole iteration blocks in one CTA (sparse_resident_kernel)
    bool resident = false;
    size_t res_smem = 0;
    int *res_rows = nullptr, *res_cols = nullptr;

    // row-sharded runs (nsli_shard_*): partial sums of the exchange step
    double *shard_dx = nullptr;

    cudaGraphExec_t graph = nullptr;
    int graph_iters = 0;
    int graph_rule = -1;
    long long launches = 0;

    nsli_result last_check{};
    std::string last_error;
};

namespace {

int set_err(nsli_solver *h, int code, const std::string &msg)
{
    if (h)
        h->last_error = msg;
    return code;
}

int cuda_err(nsli_solver *h, cudaError_t e, const char *what)
{
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation)
        return set_err(h, NSLI_ERR_OOM, msg);
    return set_err(h, NSLI_ERR_CUDA, msg);
}

#define CK(call, what)                                                                                       \
    do {                                                                                                     \
        cudaError_t e_ = (call);                                                                             \
        if (e_ != cudaSuccess)                                                                               \
            return cuda_err(h, e_, what);                                                                    \
    } while (0)

long long round_up(long long a, long long b) { return (a + b - 1) / b * b; }

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void free_all(nsli_solver *h)
{
    if (!h)
        return;
    if (h->graph)
        cudaGraphExecDestroy(h->graph);
    void *dev[] = {h->A, h->meta, h->x, h->part_y, h->b0_64, h->av_64, h->n2_64, h->part_dx, h->ybuf, h->shard_dx,
                   h->dtmp, h->scale, h->part_stat, h->st, h->ver, h->flags,
                   (h->x64 != h->x) ? (void *)h->x64 : nullptr,
                   (h->n2_meta != h->n2_64) ? (void *)h->n2_meta : nullptr,
                   h->rp, h->cp, h->ci, h->ri, h->row_cnt, h->col_cnt, h->row_pieces, h->col_pieces,
                   h->va, h->vc, h->coef, h->row_slots, h->col_slots, h->res_rows, h->res_cols, h->rtab};
    for (void *p : dev)
        if (p)
            cudaFree(p);
    if (h->st_host)
        cudaFreeHost(h->st_host);
    if (h->ver_host)
        cudaFreeHost(h->ver_host);
    if (h->flags_host)
        cudaFreeHost(h->flags_host);
    if (h->own_stream && h->stream)
        cudaStreamDestroy(h->stream);
}

// Launch shape of the Map kernel (see nsli_kernels.cu): rows are padded to
// whole 16-byte vectors; each consumer thread owns vpt vectors of every row.
int choose_config(nsli_solver *h)
{
    switch (h->storage) {
    case NSLI_F64: h->elem_bytes = 8; h->epv = 2; break;
    case NSLI_F32: h->elem_bytes = 4; h->epv = 4; break;
    case NSLI_BF16: h->elem_bytes = 2; h->epv = 8; break;
    case NSLI_FP8E4M3: h->elem_bytes = 1; h->epv = 16; break;
    default: return set_err(h, NSLI_ERR_ARG, "unknown storage type");
    }
    h->ld = round_up(h->n, h->epv);
    h->row_bytes = (int)(h->ld * h->elem_bytes);
    h->nv = h->row_bytes / 16;
    const int vlim = map_vpt_limit(h->storage);
    h->vpt = 0;
    for (int v = 1; v <= vlim; v *= 2) {
        if ((h->nv + v - 1) / v <= kMapMaxConsumers) {
            h->vpt = v;
            break;
        }
    }
    if (h->vpt == 0) {
        // long rows: thread-block clusters that split the columns
        // (NSLI_LONG_CLUSTER=0 selects the two-pass kernel): the fewest CTAs
        // per cluster (2, 4, 8; NSLI_LONG_CLUSTER_SIZE forces one) whose
        // column slice each CTA holds in registers, with a ring of at least
        // three row slices per CTA.  Measured at n = 54000 (108001 rows):
        // binary32 4.72 ms per Map on clusters of four against 7.52 ms
        // two-pass, bf16 3.57 against 4.06 ms.
        const char *cenv = std::getenv("NSLI_LONG_CLUSTER");
        const bool use_cluster = !(cenv && cenv[0] == '0');
        if (use_cluster) {
            const long long per_cta = (long long)vlim * kMapMaxConsumers;
            int forced = 0;
            if (const char *cs = std::getenv("NSLI_LONG_CLUSTER_SIZE")) {
                const int v = std::atoi(cs);
                if (v == 2 || v == 4 || v == 8)
                    forced = v;
            }
            int C = 0;
            for (int c = 2; c <= 8 && !C; c *= 2)
                if ((h->nv + c - 1) / c <= per_cta && (!forced || c == forced))
                    C = c;
            const int slice = C ? (int)((h->nv + C - 1) / C) : 0;
            const int stride = C ? (int)round_up((long long)slice * 16 + 32, 128) : 1;
            const int ns = C ? std::min(16, (232448 - kSmemHeader) / stride) : 0;
            if (C && ns >= 3) {
                int cv = 1;
                while ((long long)cv * kMapMaxConsumers < slice)
                    cv *= 2;
                // rows per block barrier: up to four for FP8 and two for
                // bf16 (short row slices, whose per-row fixed cost
                // dominates) where the ring holds the two groups in use and
                // one more, 3 x rg stages (NSLI_LONG_CLUSTER_RG forces 1, 2
                // or 4 within those limits)
                const int rg_max = h->storage == NSLI_FP8E4M3 ? 4 : (h->storage == NSLI_BF16 ? 2 : 1);
                int rg = 1;
                for (int v = rg_max; v >= 2; v /= 2)
                    if (ns >= 3 * v) {
                        rg = v;
                        break;
                    }
                if (const char *rs = std::getenv("NSLI_LONG_CLUSTER_RG")) {
                    const int v = std::atoi(rs);
                    if ((v == 1 || v == 2 || v == 4) && v <= rg_max && ns >= 3 * v)
                        rg = v;
                }
                int clusters = 0;
                const size_t smem = (size_t)kSmemHeader + (size_t)ns * stride;
                if (cluster_prepare(h->storage, cv, rg, C, smem, &clusters) == cudaSuccess && clusters > 0) {
                    h->cluster = C;
                    h->slice_nv = slice;
                    h->cluster_vpt = cv;
                    h->cluster_rg = rg;
                    // groups between a group's Map and the wait for its
                    // exchange: the ring holds D + 1 groups in use and at
                    // least one prefetched (measured best: 2 at four
                    // binary32 stages)
                    const int ng = ns / rg;
                    h->cluster_lag = std::max(1, std::min(rg == 1 ? 2 : 1, ng - 2));
                    if (const char *ls = std::getenv("NSLI_LONG_CLUSTER_LAG")) {
                        const int v = std::atoi(ls);   // 1..3, leaving a group to prefetch
                        if (v >= 1 && v <= 3 && v <= ng - 2)
                            h->cluster_lag = v;
                    }
                    h->consumers = kMapMaxConsumers;
                    h->guard = true;
                    h->nstage = ns;
                    h->stage_stride = stride;
                    h->R = 1;
                    h->smem = smem;
                    h->G = (int)std::min<long long>(clusters, h->m);
                    h->rows_base = h->m / h->G;
                    h->rows_rem = (int)(h->m % h->G);
                    h->red_grid = (int)((h->ld + kReduceCols - 1) / kReduceCols);
                    return NSLI_OK;
                }
                cudaGetLastError();   // a shape the device cannot take: use the two-pass kernel
            }
        }
        // long rows: the chunked two-pass kernel (no shared-memory ring).
        // R = rows per group: the largest of 4, 2, 1 whose rows, over all
        // CTAs, take at most 160 MB between the two passes (measured at
        // n = 54000: four rows per group beat fewer even where part of them
        // must come back from DRAM); the partial-sum row goes to shared
        // memory when it fits in 220 KB.
        h->consumers = 512;
        h->guard = true;
        h->nstage = 0;
        h->stage_stride = 0;
        h->G = (int)std::min<long long>(h->num_sms, h->m);
        long long budget = 160ll << 20;   // NSLI_LONG_L2_MB (8..512) overrides it
        if (const char *env = std::getenv("NSLI_LONG_L2_MB")) {
            const long long mb = std::atoll(env);
            if (mb >= 8 && mb <= 512)
                budget = mb << 20;
        }
        h->R = 4;
        while (h->R > 1 && (long long)h->G * h->R * h->row_bytes > budget)
            h->R /= 2;
        const size_t ybytes = (size_t)h->ld * (h->storage == NSLI_F64 ? 8 : 4);
        h->smem = ybytes <= 220 * 1024 ? ybytes : 0;
        h->rows_base = h->m / h->G;
        h->rows_rem = (int)(h->m % h->G);
        h->red_grid = (int)((h->ld + kReduceCols - 1) / kReduceCols);
        return NSLI_OK;
    }
    h->consumers = (int)round_up((h->nv + h->vpt - 1) / h->vpt, 32);
    // bytes of A per ring slot: 64 KiB unless NSLI_MAP_SLOT_KB (4..96) overrides it
    int slot_target = 65536;
    if (const char *env = std::getenv("NSLI_MAP_SLOT_KB")) {
        const int kb = std::atoi(env);
        if (kb >= 4 && kb <= 96)
            slot_target = kb * 1024;
    }
    h->guard = (long long)h->consumers * h->vpt != h->nv;
    const int rg = map_rows_per_group(h->vpt, h->storage == NSLI_F64 ? 8 : 4);
    h->R = rg * std::max(1, std::min(64 / rg, slot_target / (h->row_bytes * rg)));
    h->stage_stride = (int)round_up((long long)h->R * h->row_bytes + (long long)h->R * 32, 128);
    const int budget = 232448 - kSmemHeader;
    h->nstage = std::min(8, budget / h->stage_stride);
    if (h->nstage < 2)
        return set_err(h, NSLI_ERR_UNSUPPORTED, "row does not fit two shared-memory stages");
    h->smem = (size_t)kSmemHeader + (size_t)h->nstage * h->stage_stride;
    h->G = (int)std::min<long long>(h->num_sms, h->m);
    h->rows_base = h->m / h->G;
    h->rows_rem = (int)(h->m % h->G);
    h->red_grid = (int)((h->ld + kReduceCols - 1) / kReduceCols);
    return NSLI_OK;
}

MapArgs map_args(nsli_solver *h)
{
    MapArgs a;
    a.A = h->A;
    a.meta = h->meta;
    a.x = h->x;
    a.part_y = h->part_y;
    a.part_stat = h->part_stat;
    a.st = h->st;
    a.ld = h->ld;
    a.m = h->m;
    a.rows_base = h->rows_base;
    a.rows_rem = h->rows_rem;
    a.nv = h->nv;
    a.row_bytes = h->row_bytes;
    a.rows_per_slot = h->R;
    a.nstage = h->nstage;
    a.stage_stride = h->stage_stride;
    a.ignore_done = 0;
    a.skip_slot = -1;
    a.cluster = h->cluster;
    a.slice_nv = h->slice_nv;
    a.cluster_vpt = h->cluster_vpt;
    a.cluster_lag = h->cluster_lag;
    a.cluster_rg = h->cluster_rg;
    return a;
}

ReduceArgs reduce_args(nsli_solver *h)
{
    ReduceArgs a;
    a.part_y = h->part_y;
    a.part_stat = h->part_stat;
    a.x = h->x;
    a.x64 = h->x64;
    a.ybuf = h->ybuf;
    a.part_dx = h->part_dx;
    a.st = h->st;
    a.rtab = h->rtab;
    a.ld = h->ld;
    a.G = h->G;
    return a;
}

// kernels per iteration: Map + Reduce/step; a sparse A adds the ModAP step
int launches_per_iteration(const nsli_solver *h, int rule)
{
    return (h->sparse && rule == NSLI_RULE_MODAP) ? 3 : 2;
}

cudaError_t launch_iteration(nsli_solver *h, int rule)
{
    if (h->sparse) {
        const bool f64 = h->storage == NSLI_F64;
        cudaError_t e = sparse_row_launch(f64, h->stream, h->sp);
        if (e == cudaSuccess)
            e = sparse_col_launch(f64, h->stream, h->sp);
        if (e == cudaSuccess && rule == NSLI_RULE_MODAP)
            e = sparse_step_launch(f64, h->stream, h->sp);
        return e;
    }
    cudaError_t e = map_launch(h->storage, h->vpt, h->guard, h->G, h->consumers, h->smem, h->stream, map_args(h));
    if (e != cudaSuccess)
        return e;
    return reduce_launch(h->storage == NSLI_F64, h->red_grid, h->stream, reduce_args(h));
}

int ensure_graph(nsli_solver *h, int iters, int rule)
{
    // the dense kernels read the rule at run time; the sparse ModAP graph
    // holds one more kernel per iteration
    const int key = h->sparse ? rule : -1;
    if (h->graph && h->graph_iters == iters && h->graph_rule == key)
        return NSLI_OK;
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t err = cudaSuccess;
    for (int i = 0; i < iters && err == cudaSuccess; ++i)
        err = launch_iteration(h, rule);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    if (err != cudaSuccess) {
        if (g)
            cudaGraphDestroy(g);
        return cuda_err(h, err, "capture iteration block");
    }
    CK(e2, "end capture");
    cudaError_t e3 = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    CK(e3, "instantiate iteration graph");
    h->graph_iters = iters;
    h->graph_rule = key;
    return NSLI_OK;
}

int validate_params(nsli_solver *h, const nsli_params *p)
{
    if (!p)
        return set_err(h, NSLI_ERR_ARG, "params is NULL");
    if (!(p->lambda > 0.0) || !std::isfinite(p->lambda))
        return set_err(h, NSLI_ERR_ARG, "lambda must be finite and > 0");
    if (p->rule != NSLI_RULE_RELAXED && p->rule != NSLI_RULE_MODAP)
        return set_err(h, NSLI_ERR_ARG, "unknown rule");
    if (p->stop < NSLI_STOP_NONE || p->stop > NSLI_STOP_MAXVIOL_REL)
        return set_err(h, NSLI_ERR_ARG, "unknown stop rule");
    if (!(p->eps >= 0.0) || !std::isfinite(p->eps))
        return set_err(h, NSLI_ERR_ARG, "eps must be finite and >= 0");
    if (p->max_iter < 0 || p->block_iters < 0 || p->block_iters > 4096 || p->reserved != 0)
        return set_err(h, NSLI_ERR_ARG, "bad max_iter / block_iters / reserved");
    if (!std::isfinite(p->rho))
        return set_err(h, NSLI_ERR_ARG, "rho must be finite");
    return NSLI_OK;
}

int read_flags(nsli_solver *h)
{
    CK(cudaMemcpyAsync(h->flags_host, h->flags, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "read flags");
    CK(cudaStreamSynchronize(h->stream), "synchronize");
    const int f = *h->flags_host;
    if (f & PREPF_TIMEOUT)
        return set_err(h, NSLI_ERR_TIMEOUT, "a row copy did not arrive within the wait limit");
    if (f & PREPF_NONFINITE)
        return set_err(h, NSLI_ERR_NONFINITE, "NaN or Inf in the input");
    if (f & PREPF_ZERO_ROW)
        return set_err(h, NSLI_ERR_ZERO_ROW, "A has a zero row (the method needs a_i != 0)");
    return NSLI_OK;
}

double ord_dec(unsigned long long u)
{
    unsigned long long bits = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
    double d;
    std::memcpy(&d, &bits, sizeof d);
    return d;
}

// The binary64 norms of the stored rows, if rows changed since they were
// last taken (dense binary32 / bf16 / fp8 storage).
int ensure_norms64(nsli_solver *h)
{
    if (h->n2_64_valid)
        return NSLI_OK;
    CK(stored_norms64_launch(h->storage, h->stream, h->A, h->scale, h->ld, h->n, h->m, h->n2_64),
       "binary64 row norms");
    h->launches += 1;
    h->n2_64_valid = true;
    return NSLI_OK;
}

// Binary64 check at the current x and tick; fills h->last_check fields.
int run_verify(nsli_solver *h)
{
    int rc = ensure_norms64(h);
    if (rc != NSLI_OK)
        return rc;
    CK(cudaMemsetAsync(h->ver, 0, sizeof(VerOut), h->stream), "clear check");
    VerifyArgs a;
    a.A = h->A;
    a.x64 = h->x64;
    a.b0_64 = h->b0_64;
    a.av_64 = h->av_64;
    a.n2_64 = h->n2_64;
    a.scale = h->scale;
    a.st = h->st;
    a.out = h->ver;
    a.ld = h->ld;
    a.m = h->m;
    a.nv = h->nv;
    const int grid = std::max(1, std::min<int>(h->num_sms * 8, (int)((h->m + 7) / 8)));
    if (h->sparse)
        CK(sparse_verify_launch(h->storage == NSLI_F64, grid, h->stream, h->sp, a), "launch binary64 check");
    else
        CK(verify_launch(h->storage, grid, h->stream, a), "launch binary64 check");
    h->launches += 1;
    CK(cudaMemcpyAsync(h->ver_host, h->ver, sizeof(VerOut), cudaMemcpyDeviceToHost, h->stream), "read check");
    CK(cudaStreamSynchronize(h->stream), "synchronize");
    h->last_check.max_viol = ord_dec(h->ver_host->maxviol);
    h->last_check.max_viol_norm = ord_dec(h->ver_host->maxnorm);
    h->last_check.max_abs_b = ord_dec(h->ver_host->maxb);
    h->last_check.h = (int64_t)h->ver_host->h;
    return NSLI_OK;
}

int read_state(nsli_solver *h)
{
    CK(cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream), "read state");
    CK(cudaStreamSynchronize(h->stream), "synchronize");
    if (h->st_host->error & ERRF_TIMEOUT)
        return set_err(h, NSLI_ERR_TIMEOUT, "a bounded device wait expired");
    return NSLI_OK;
}

int begin_run(nsli_solver *h, const nsli_params *p, int stop, long long max_iter)
{
    StateBegin b;
    b.lambda = p->lambda;
    b.eps = p->eps;
    b.rho = p->rho;
    b.max_iter = max_iter;
    b.rule = p->rule;
    b.stop = stop;
    b.reset_it = 1;
    b.force_step = 0;
    b.tick = -1;
    const bool fill = h->rtab && !(h->rtab_lambda == p->lambda);
    b.rtab = fill ? h->rtab : nullptr;
    b.rtab_m = h->m;
    CK(state_begin_launch(h->stream, h->st, b), "begin run");
    if (fill)
        h->rtab_lambda = p->lambda;
    h->launches += 1;
    return NSLI_OK;
}

}  // namespace

extern "C" {

const char *nsli_strerror(int code)
{
    switch (code) {
    case NSLI_OK: return "ok";
    case NSLI_NOT_CONVERGED: return "maximum number of iterations reached";
    case NSLI_RUNNING: return "running";
    case NSLI_CANDIDATE: return "stop test passed, binary64 check pending";
    case NSLI_ERR_ARG: return "invalid argument";
    case NSLI_ERR_ZERO_ROW: return "zero row in A";
    case NSLI_ERR_NONFINITE: return "NaN or Inf in the input";
    case NSLI_ERR_OOM: return "device memory allocation failed";
    case NSLI_ERR_CUDA: return "CUDA runtime error";
    case NSLI_ERR_TIMEOUT: return "bounded device wait expired";
    case NSLI_ERR_UNSUPPORTED: return "outside the limits of this library";
    default: return "unknown status";
    }
}

const char *nsli_last_error(nsli_handle h) { return h ? h->last_error.c_str() : ""; }

int64_t nsli_launch_count(nsli_handle h) { return h ? (int64_t)h->launches : 0; }

int nsli_create(nsli_handle *out, int64_t m, int64_t n, int32_t storage, int32_t a_dtype, const void *A,
                int64_t lda, const double *b0, const double *norms2, const double *Av, const double *x0,
                void *stream)
{
    Trace trace_("nsli_create");
    if (!out)
        return NSLI_ERR_ARG;
    *out = nullptr;
    if (m < 1 || n < 1 || lda < n || !A || !b0 || !x0)
        return NSLI_ERR_ARG;
    if (a_dtype != NSLI_F32 && a_dtype != NSLI_F64)
        return NSLI_ERR_ARG;
    if (storage < NSLI_F64 || storage > NSLI_FP8E4M3)
        return NSLI_ERR_ARG;
    if ((storage == NSLI_BF16 || storage == NSLI_FP8E4M3) && a_dtype != NSLI_F32)
        return NSLI_ERR_ARG;
    if (m > (1ll << 40) || n > (1ll << 31))
        return NSLI_ERR_UNSUPPORTED;

    nsli_solver *h = new nsli_solver();
    h->storage = storage;
    h->m = m;
    h->n = n;
    int rc = NSLI_OK;
    auto fail = [&](int code) {
        free_all(h);
        delete h;
        return code;
    };
#define CKC(call, what)                                                                                      \
    do {                                                                                                     \
        cudaError_t e_ = (call);                                                                             \
        if (e_ != cudaSuccess)                                                                               \
            return fail(cuda_err(h, e_, what));                                                              \
    } while (0)

    CKC(cudaGetDevice(&h->device), "get device");
    CKC(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device), "SM count");
    if ((rc = choose_config(h)) != NSLI_OK)
        return fail(rc);
    if (stream) {
        h->stream = static_cast<cudaStream_t>(stream);
    } else {
        CKC(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking), "create stream");
        h->own_stream = true;
    }
    cudaStream_t s = h->stream;

    const size_t accb = (storage == NSLI_F64) ? 8 : 4;
    const size_t meta_bytes = 32;
    CKC(cudaMalloc(&h->A, (size_t)m * h->row_bytes), "allocate A");
    CKC(cudaMalloc(&h->meta, (size_t)m * meta_bytes), "allocate row records");
    CKC(cudaMalloc((void **)&h->b0_64, (size_t)m * 8), "allocate b0");
    CKC(cudaMalloc((void **)&h->av_64, (size_t)m * 8), "allocate Av");
    CKC(cudaMalloc((void **)&h->n2_64, (size_t)m * 8), "allocate norms");
    if (storage == NSLI_F64)
        h->n2_meta = h->n2_64;
    else
        CKC(cudaMalloc((void **)&h->n2_meta, (size_t)m * 8), "allocate record norms");
    if (storage == NSLI_FP8E4M3)
        CKC(cudaMalloc((void **)&h->scale, (size_t)m * 4), "allocate row scales");
    CKC(cudaMalloc(&h->x, (size_t)h->ld * accb), "allocate x");
    if (storage == NSLI_F64)
        h->x64 = static_cast<double *>(h->x);
    else
        CKC(cudaMalloc((void **)&h->x64, (size_t)h->ld * 8), "allocate binary64 x");
    CKC(cudaMalloc(&h->part_y, (size_t)h->G * h->ld * accb), "allocate partial sums");
    CKC(cudaMalloc((void **)&h->part_stat, (size_t)h->G * sizeof(PartStat)), "allocate partial stats");
    CKC(cudaMalloc((void **)&h->rtab, (size_t)(m + 1) * 8), "allocate step table");
    CKC(cudaMalloc((void **)&h->part_dx, (size_t)h->red_grid * 8), "allocate step partials");
    CKC(cudaMalloc((void **)&h->ybuf, (size_t)h->ld * 8), "allocate y");
    CKC(cudaMalloc((void **)&h->dtmp, (size_t)std::max<long long>(m, h->ld) * 8), "allocate staging");
    CKC(cudaMalloc((void **)&h->st, sizeof(DevState)), "allocate state");
    CKC(cudaMalloc((void **)&h->ver, sizeof(VerOut)), "allocate check");
    CKC(cudaMalloc((void **)&h->flags, sizeof(int)), "allocate flags");
    CKC(cudaMallocHost((void **)&h->st_host, sizeof(DevState)), "allocate pinned state");
    CKC(cudaMallocHost((void **)&h->ver_host, sizeof(VerOut)), "allocate pinned check");
    CKC(cudaMallocHost((void **)&h->flags_host, sizeof(int)), "allocate pinned flags");

    CKC(cudaMemsetAsync(h->st, 0, sizeof(DevState), s), "clear state");
    CKC(cudaMemsetAsync(h->flags, 0, sizeof(int), s), "clear flags");
    CKC(cudaMemsetAsync(h->ybuf, 0, (size_t)h->ld * 8, s), "clear y");
    CKC(cudaMemcpyAsync(h->b0_64, b0, (size_t)m * 8, cudaMemcpyDefault, s), "copy b0");
    if (Av)
        CKC(cudaMemcpyAsync(h->av_64, Av, (size_t)m * 8, cudaMemcpyDefault, s), "copy Av");
    else
        CKC(cudaMemsetAsync(h->av_64, 0, (size_t)m * 8, s), "clear Av");
    CKC(check_finite_launch(s, h->b0_64, m, h->flags), "check b0");
    CKC(check_finite_launch(s, h->av_64, m, h->flags), "check Av");
    h->launches += 2;

    // x0 -> accumulation type (the staging buffer is reused for the norms
    // only after this kernel has consumed it, in stream order)
    CKC(cudaMemcpyAsync(h->dtmp, x0, (size_t)n * 8, cudaMemcpyDefault, s), "copy x0");
    CKC(x_from_f64_launch(storage == NSLI_F64, s, h->dtmp, h->x64, h->x, n, h->ld, h->flags), "convert x0");
    h->launches += 1;

    const double *norms_dev = nullptr;
    double *norms_buf = nullptr;
    if (norms2) {
        CKC(cudaMalloc((void **)&norms_buf, (size_t)m * 8), "allocate norms input");
        cudaError_t e = cudaMemcpyAsync(norms_buf, norms2, (size_t)m * 8, cudaMemcpyDefault, s);
        if (e != cudaSuccess) {
            cudaFree(norms_buf);
            return fail(cuda_err(h, e, "copy norms"));
        }
        norms_dev = norms_buf;
    }

    // A: quantise / copy row blocks into the padded device layout
    const size_t src_eb = (a_dtype == NSLI_F64) ? 8 : 4;
    const bool a_on_device = is_device_ptr(A);
    long long chunk = std::max<long long>(1, (256ll << 20) / (long long)(lda * src_eb));
    chunk = std::min<long long>(chunk, m);
    void *stage = nullptr;
    if (!a_on_device) {
        cudaError_t e = cudaMalloc(&stage, (size_t)chunk * lda * src_eb);
        if (e != cudaSuccess) {
            if (norms_buf)
                cudaFree(norms_buf);
            return fail(cuda_err(h, e, "allocate staging for A"));
        }
    }
    cudaError_t err = cudaSuccess;
    for (long long r0 = 0; r0 < m && err == cudaSuccess; r0 += chunk) {
        const long long rows = std::min(chunk, m - r0);
        PrepArgs pa;
        if (a_on_device) {
            pa.src = static_cast<const unsigned char *>(A) + (size_t)r0 * lda * src_eb;
        } else {
            err = cudaMemcpy2DAsync(stage, (size_t)lda * src_eb,
                                    static_cast<const unsigned char *>(A) + (size_t)r0 * lda * src_eb,
                                    (size_t)lda * src_eb, (size_t)n * src_eb, (size_t)rows, cudaMemcpyDefault, s);
            if (err != cudaSuccess)
                break;
            pa.src = stage;
        }
        pa.lda = lda;
        pa.src_f64 = (a_dtype == NSLI_F64) ? 1 : 0;
        pa.A = h->A;
        pa.ld = h->ld;
        pa.n = n;
        pa.row0 = r0;
        pa.rows = rows;
        pa.norms_in = norms_dev;
        pa.n2_64 = h->n2_meta;
        pa.scale = h->scale;
        pa.flags = h->flags;
        pa.fast = 1;
        err = prep_launch(storage, s, pa);
        h->launches += 1;
        if (!a_on_device && err == cudaSuccess)
            err = cudaStreamSynchronize(s);  // the staging buffer is reused
    }
    if (err == cudaSuccess) {
        MetaArgs ma;
        ma.meta = h->meta;
        ma.b0_64 = h->b0_64;
        ma.av_64 = h->av_64;
        ma.n2_64 = h->n2_meta;
        ma.scale = h->scale;
        ma.m = m;
        ma.flags = h->flags;
        err = meta_launch(storage == NSLI_F64, s, ma);
        h->launches += 1;
    }
    // binary64 norms: the same array for binary64 storage, the user's norms
    // if given, else taken from the stored rows when first needed
    if (err == cudaSuccess && h->n2_meta != h->n2_64) {
        if (norms2)
            err = cudaMemcpyAsync(h->n2_64, h->n2_meta, (size_t)m * 8, cudaMemcpyDeviceToDevice, s);
        else
            h->n2_64_valid = false;
    }
    if (err == cudaSuccess)
        err = cudaStreamSynchronize(s);
    if (stage)
        cudaFree(stage);
    if (norms_buf)
        cudaFree(norms_buf);
    if (err != cudaSuccess)
        return fail(cuda_err(h, err, "prepare A"));
    if ((rc = read_flags(h)) != NSLI_OK)
        return fail(rc);
    if (h->cluster == 0)
        CKC(map_prepare(storage, h->vpt, h->guard, h->smem), "configure Map kernel");
#undef CKC
    *out = h;
    return NSLI_OK;
}

int nsli_create_csr(nsli_handle *out, int64_t m, int64_t n, int32_t storage, int64_t nnz, const int64_t *row_ptr,
                    const int32_t *col_idx, const double *val, const double *b0, const double *norms2,
                    const double *Av, const double *x0, void *stream)
{
    Trace trace_("nsli_create_csr");
    if (!out)
        return NSLI_ERR_ARG;
    *out = nullptr;
    if (m < 1 || n < 1 || nnz < 1 || !row_ptr || !col_idx || !val || !b0 || !x0)
        return NSLI_ERR_ARG;
    if (storage != NSLI_F64 && storage != NSLI_F32)
        return NSLI_ERR_UNSUPPORTED;
    if (m >= (1ll << 31) || n >= (1ll << 31) || nnz > (1ll << 40))
        return NSLI_ERR_UNSUPPORTED;

    nsli_solver *h = new nsli_solver();
    h->sparse = true;
    h->storage = storage;
    h->m = m;
    h->n = n;
    h->ld = n;
    h->nnz = nnz;
    h->elem_bytes = storage == NSLI_F64 ? 8 : 4;
    auto fail = [&](int code) {
        free_all(h);
        delete h;
        return code;
    };
#define CKC(call, what)                                                                                      \
    do {                                                                                                     \
        cudaError_t e_ = (call);                                                                             \
        if (e_ != cudaSuccess)                                                                               \
            return fail(cuda_err(h, e_, what));                                                              \
    } while (0)

    CKC(cudaGetDevice(&h->device), "get device");
    CKC(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device), "SM count");

    // host copies of the structure (the inputs may be device memory); the
    // column-major copy is built by a stable counting sort, so the rows of
    // every column stay ascending
    std::vector<long long> rp((size_t)m + 1);
    std::vector<int> ci((size_t)nnz);
    std::vector<double> va((size_t)nnz);
    CKC(cudaMemcpy(rp.data(), row_ptr, (size_t)(m + 1) * 8, cudaMemcpyDefault), "copy row offsets");
    CKC(cudaMemcpy(ci.data(), col_idx, (size_t)nnz * 4, cudaMemcpyDefault), "copy column indices");
    CKC(cudaMemcpy(va.data(), val, (size_t)nnz * 8, cudaMemcpyDefault), "copy values");
    if (rp[0] != 0 || rp[m] != nnz)
        return fail(set_err(h, NSLI_ERR_ARG, "row offsets must start at 0 and end at nnz"));
    for (long long i = 0; i < m; ++i) {
        if (rp[i + 1] < rp[i])
            return fail(set_err(h, NSLI_ERR_ARG, "row offsets must not decrease"));
        for (long long e = rp[i]; e < rp[i + 1]; ++e) {
            if (ci[e] < 0 || ci[e] >= n)
                return fail(set_err(h, NSLI_ERR_ARG, "column index out of range"));
            if (e > rp[i] && ci[e] <= ci[e - 1])
                return fail(set_err(h, NSLI_ERR_ARG, "column indices must increase strictly within a row"));
            if (!std::isfinite(va[e]))
                return fail(set_err(h, NSLI_ERR_NONFINITE, "NaN or Inf in the input"));
        }
    }
    std::vector<long long> cp((size_t)n + 1, 0);
    for (long long e = 0; e < nnz; ++e)
        cp[(size_t)ci[e] + 1] += 1;
    for (long long j = 0; j < n; ++j)
        cp[j + 1] += cp[j];
    std::vector<long long> fill(cp.begin(), cp.end() - 1);
    std::vector<int> ri((size_t)nnz);
    std::vector<double> vcol((size_t)nnz);
    for (long long i = 0; i < m; ++i)
        for (long long e = rp[i]; e < rp[i + 1]; ++e) {
            const long long k = fill[ci[e]]++;
            ri[k] = (int)i;
            vcol[k] = va[e];
        }

    // lanes per row / column from the median length (a few very long rows or
    // columns do not set it): W lanes x kSparseU loads cover a typical one in
    // one chunk; those needing more than 4 chunks are cut into pieces of
    // kSparsePiece entries, one CTA each
    auto median_len = [](const std::vector<long long> &off) {
        std::vector<long long> len(off.size() - 1);
        for (size_t i = 0; i + 1 < off.size(); ++i)
            len[i] = off[i + 1] - off[i];
        std::nth_element(len.begin(), len.begin() + len.size() / 2, len.end());
        return (double)len[len.size() / 2];
    };
    auto pick_w = [](double typical) {
        int w = 1;
        while (w < 32 && (double)kSparseU * w < typical)
            w *= 2;
        return w;
    };
    auto make_pieces = [](const std::vector<long long> &off, long long thr, std::vector<SegPiece> &pcs,
                          long long *nseg, long long *nslots) {
        long long hs = 0, slot = 0;
        for (size_t q = 0; q + 1 < off.size(); ++q) {
            const long long len = off[q + 1] - off[q];
            if (len <= thr)
                continue;
            const int np = (int)((len + kSparsePiece - 1) / kSparsePiece);
            for (int k = 0; k < np; ++k) {
                SegPiece pc;
                pc.seg = (int)q;
                pc.hs = (int)hs;
                pc.first = (int)slot;
                pc.npieces = np;
                pc.k = k;
                pc.pad = 0;
                pc.e0 = off[q] + (long long)k * kSparsePiece;
                pc.e1 = std::min(off[q + 1], pc.e0 + kSparsePiece);
                pcs.push_back(pc);
            }
            slot += np;
            hs += 1;
        }
        *nseg = hs;
        *nslots = slot;
    };
    // One CTA runs whole blocks of iterations when its shared memory holds
    // x64, y, x and c and the matrix (both orders) fits, with them, in the
    // SM's 256 KB of L1 and shared memory: then an iteration reads nothing
    // from L2.  NSLI_SPARSE_RESIDENT=0 never takes this path, =1 takes it
    // whenever the shared memory suffices.
    const size_t res_smem = sparse_resident_smem(storage == NSLI_F64, m, n);
    const size_t res_total = res_smem + (size_t)nnz * 2 * (h->elem_bytes + 4) + (size_t)(m + n + 2) * 8;
    {
        const char *env = std::getenv("NSLI_SPARSE_RESIDENT");
        const int force = env ? std::atoi(env) : -1;
        h->resident = res_smem <= kResSmemMax && force != 0 && (force == 1 || res_total <= (200u << 10));
        h->res_smem = res_smem;
    }
    std::vector<int> long_rows, long_cols;
    if (h->resident) {
        for (long long i = 0; i < m; ++i)
            if (rp[i + 1] - rp[i] > kResLong)
                long_rows.push_back((int)i);
        for (long long j = 0; j < n; ++j)
            if (cp[j + 1] - cp[j] > kResLong)
                long_cols.push_back((int)j);
    }

    SparseArgs &sp = h->sp;
    sp = SparseArgs{};
    sp.m = m;
    sp.n = n;
    sp.w_row = pick_w(median_len(rp));
    sp.w_col = pick_w(median_len(cp));
    sp.heavy_thr_row = 4ll * kSparseU * sp.w_row;
    sp.heavy_thr_col = 4ll * kSparseU * sp.w_col;
    std::vector<SegPiece> hr, hc;
    long long nseg_r = 0, nslot_r = 0, nseg_c = 0, nslot_c = 0;
    make_pieces(rp, sp.heavy_thr_row, hr, &nseg_r, &nslot_r);
    make_pieces(cp, sp.heavy_thr_col, hc, &nseg_c, &nslot_c);
    if (hr.size() > (size_t)INT_MAX / 2 || hc.size() > (size_t)INT_MAX / 2)
        return fail(set_err(h, NSLI_ERR_UNSUPPORTED, "too many heavy pieces"));
    sp.n_row_pieces = (int)hr.size();
    sp.n_col_pieces = (int)hc.size();
    int row_bps = 0, col_bps = 0;
    sparse_blocks_per_sm(storage == NSLI_F64, sp.w_row, sp.w_col, &row_bps, &col_bps);
    auto split = [&](long long items, int w, int bps, int *ctas, long long *per) {
        const long long groups = 256 / w;
        const long long cap = (long long)h->num_sms * std::max(1, bps);
        long long c = (items + groups - 1) / groups;
        c = std::max<long long>(1, std::min<long long>(c, cap));
        *per = (items + c - 1) / c;
        *ctas = (int)((items + *per - 1) / *per);
    };
    split(m, sp.w_row, row_bps, &sp.row_light_ctas, &sp.light_rows_per_cta);
    split(n, sp.w_col, col_bps, &sp.col_light_ctas, &sp.light_cols_per_cta);
    sp.step_ctas = (int)std::max<long long>(1, std::min<long long>((n + 1023) / 1024, (long long)h->num_sms * 4));
    const long long g_row = sp.n_row_pieces + sp.row_light_ctas;
    const long long g_col = std::max<long long>(sp.n_col_pieces + sp.col_light_ctas, sp.step_ctas);
    h->G = (int)g_row;

    if (stream) {
        h->stream = static_cast<cudaStream_t>(stream);
    } else {
        CKC(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking), "create stream");
        h->own_stream = true;
    }
    cudaStream_t s = h->stream;
    const size_t eb = (size_t)h->elem_bytes;
    CKC(cudaMalloc((void **)&h->rp, (size_t)(m + 1) * 8), "allocate row offsets");
    CKC(cudaMalloc((void **)&h->ci, (size_t)nnz * 4), "allocate column indices");
    CKC(cudaMalloc(&h->va, (size_t)nnz * eb), "allocate row values");
    CKC(cudaMalloc((void **)&h->cp, (size_t)(n + 1) * 8), "allocate column offsets");
    CKC(cudaMalloc((void **)&h->ri, (size_t)nnz * 4), "allocate row indices");
    CKC(cudaMalloc(&h->vc, (size_t)nnz * eb), "allocate column values");
    if (!hr.empty()) {
        CKC(cudaMalloc((void **)&h->row_pieces, hr.size() * sizeof(SegPiece)), "allocate heavy row pieces");
        CKC(cudaMalloc(&h->row_slots, (size_t)nslot_r * eb), "allocate heavy row slots");
        CKC(cudaMalloc((void **)&h->row_cnt, (size_t)nseg_r * 4), "allocate heavy row counters");
    }
    if (!hc.empty()) {
        CKC(cudaMalloc((void **)&h->col_pieces, hc.size() * sizeof(SegPiece)), "allocate heavy column pieces");
        CKC(cudaMalloc(&h->col_slots, (size_t)nslot_c * eb), "allocate heavy column slots");
        CKC(cudaMalloc((void **)&h->col_cnt, (size_t)nseg_c * 4), "allocate heavy column counters");
    }
    CKC(cudaMalloc(&h->coef, (size_t)m * eb), "allocate slice coefficients");
    CKC(cudaMalloc(&h->meta, (size_t)m * 32), "allocate row records");
    CKC(cudaMalloc((void **)&h->b0_64, (size_t)m * 8), "allocate b0");
    CKC(cudaMalloc((void **)&h->av_64, (size_t)m * 8), "allocate Av");
    CKC(cudaMalloc((void **)&h->n2_64, (size_t)m * 8), "allocate norms");
    CKC(cudaMalloc(&h->x, (size_t)n * eb), "allocate x");
    if (storage == NSLI_F64)
        h->x64 = static_cast<double *>(h->x);
    else
        CKC(cudaMalloc((void **)&h->x64, (size_t)n * 8), "allocate binary64 x");
    CKC(cudaMalloc((void **)&h->part_stat, (size_t)g_row * sizeof(PartStat)), "allocate partial stats");
    CKC(cudaMalloc((void **)&h->rtab, (size_t)(m + 1) * 8), "allocate step table");
    CKC(cudaMalloc((void **)&h->part_dx, (size_t)g_col * 8), "allocate step partials");
    CKC(cudaMalloc((void **)&h->ybuf, (size_t)n * 8), "allocate y");
    CKC(cudaMalloc((void **)&h->dtmp, (size_t)std::max<long long>(m, n) * 8), "allocate staging");
    CKC(cudaMalloc((void **)&h->st, sizeof(DevState)), "allocate state");
    CKC(cudaMalloc((void **)&h->ver, sizeof(VerOut)), "allocate check");
    CKC(cudaMalloc((void **)&h->flags, sizeof(int)), "allocate flags");
    CKC(cudaMallocHost((void **)&h->st_host, sizeof(DevState)), "allocate pinned state");
    CKC(cudaMallocHost((void **)&h->ver_host, sizeof(VerOut)), "allocate pinned check");
    CKC(cudaMallocHost((void **)&h->flags_host, sizeof(int)), "allocate pinned flags");

    // values in the storage type (binary32: rounded to nearest, ties to even)
    std::vector<float> va32, vc32;
    const void *va_src = va.data(), *vc_src = vcol.data();
    if (storage == NSLI_F32) {
        va32.assign(va.begin(), va.end());
        vc32.assign(vcol.begin(), vcol.end());
        va_src = va32.data();
        vc_src = vc32.data();
    }
    CKC(cudaMemcpyAsync(h->rp, rp.data(), (size_t)(m + 1) * 8, cudaMemcpyHostToDevice, s), "upload row offsets");
    CKC(cudaMemcpyAsync(h->ci, ci.data(), (size_t)nnz * 4, cudaMemcpyHostToDevice, s), "upload column indices");
    CKC(cudaMemcpyAsync(h->va, va_src, (size_t)nnz * eb, cudaMemcpyHostToDevice, s), "upload row values");
    CKC(cudaMemcpyAsync(h->cp, cp.data(), (size_t)(n + 1) * 8, cudaMemcpyHostToDevice, s), "upload column offsets");
    CKC(cudaMemcpyAsync(h->ri, ri.data(), (size_t)nnz * 4, cudaMemcpyHostToDevice, s), "upload row indices");
    CKC(cudaMemcpyAsync(h->vc, vc_src, (size_t)nnz * eb, cudaMemcpyHostToDevice, s), "upload column values");
    if (!hr.empty()) {
        CKC(cudaMemcpyAsync(h->row_pieces, hr.data(), hr.size() * sizeof(SegPiece), cudaMemcpyHostToDevice, s),
            "upload heavy row pieces");
        CKC(cudaMemsetAsync(h->row_cnt, 0, (size_t)nseg_r * 4, s), "clear heavy row counters");
    }
    if (!hc.empty()) {
        CKC(cudaMemcpyAsync(h->col_pieces, hc.data(), hc.size() * sizeof(SegPiece), cudaMemcpyHostToDevice, s),
            "upload heavy column pieces");
        CKC(cudaMemsetAsync(h->col_cnt, 0, (size_t)nseg_c * 4, s), "clear heavy column counters");
    }

    sp.rp = h->rp;
    sp.ci = h->ci;
    sp.va = h->va;
    sp.cp = h->cp;
    sp.ri = h->ri;
    sp.vc = h->vc;
    sp.meta = h->meta;
    sp.row_pieces = h->row_pieces;
    sp.col_pieces = h->col_pieces;
    sp.row_slots = h->row_slots;
    sp.col_slots = h->col_slots;
    sp.row_cnt = h->row_cnt;
    sp.col_cnt = h->col_cnt;
    sp.coef = h->coef;
    sp.x = h->x;
    sp.x64 = h->x64;
    sp.ybuf = h->ybuf;
    sp.part_stat = h->part_stat;
    sp.part_dx = h->part_dx;
    sp.st = h->st;
    sp.ignore_done = 0;
    sp.mode = 0;
    sp.rtab = h->rtab;
    if (h->resident) {
        if (!long_rows.empty()) {
            CKC(cudaMalloc((void **)&h->res_rows, long_rows.size() * 4), "allocate long row list");
            CKC(cudaMemcpyAsync(h->res_rows, long_rows.data(), long_rows.size() * 4, cudaMemcpyHostToDevice, s),
                "upload long row list");
        }
        if (!long_cols.empty()) {
            CKC(cudaMalloc((void **)&h->res_cols, long_cols.size() * 4), "allocate long column list");
            CKC(cudaMemcpyAsync(h->res_cols, long_cols.data(), long_cols.size() * 4, cudaMemcpyHostToDevice, s),
                "upload long column list");
        }
        sp.res_long_rows = h->res_rows;
        sp.res_long_cols = h->res_cols;
        sp.n_res_long_rows = (int)long_rows.size();
        sp.n_res_long_cols = (int)long_cols.size();
        CKC(sparse_resident_prepare(storage == NSLI_F64, h->res_smem), "configure one-CTA kernel");
    }

    CKC(cudaMemsetAsync(h->st, 0, sizeof(DevState), s), "clear state");
    CKC(cudaMemsetAsync(h->flags, 0, sizeof(int), s), "clear flags");
    CKC(cudaMemsetAsync(h->ybuf, 0, (size_t)n * 8, s), "clear y");
    CKC(cudaMemsetAsync(h->coef, 0, (size_t)m * eb, s), "clear coefficients");
    CKC(cudaMemcpyAsync(h->b0_64, b0, (size_t)m * 8, cudaMemcpyDefault, s), "copy b0");
    if (Av)
        CKC(cudaMemcpyAsync(h->av_64, Av, (size_t)m * 8, cudaMemcpyDefault, s), "copy Av");
    else
        CKC(cudaMemsetAsync(h->av_64, 0, (size_t)m * 8, s), "clear Av");
    CKC(check_finite_launch(s, h->b0_64, m, h->flags), "check b0");
    CKC(check_finite_launch(s, h->av_64, m, h->flags), "check Av");
    CKC(cudaMemcpyAsync(h->dtmp, x0, (size_t)n * 8, cudaMemcpyDefault, s), "copy x0");
    CKC(x_from_f64_launch(storage == NSLI_F64, s, h->dtmp, h->x64, h->x, n, n, h->flags), "convert x0");
    const int ngrid = (int)std::max<long long>(1, std::min<long long>((long long)h->num_sms * 8, (m + 7) / 8));
    h->n2_meta = h->n2_64;   // sparse rows: the binary64 norms serve the records too
    CKC(sparse_norms_launch(storage == NSLI_F64, ngrid, s, sp, h->n2_64, h->flags), "row norms");
    if (norms2)
        CKC(cudaMemcpyAsync(h->n2_64, norms2, (size_t)m * 8, cudaMemcpyDefault, s), "copy norms");
    MetaArgs ma;
    ma.meta = h->meta;
    ma.b0_64 = h->b0_64;
    ma.av_64 = h->av_64;
    ma.n2_64 = h->n2_64;
    ma.scale = nullptr;
    ma.m = m;
    ma.flags = h->flags;
    CKC(meta_launch(storage == NSLI_F64, s, ma), "row records");
    h->launches += 5;
    CKC(cudaStreamSynchronize(s), "synchronize");
    int rc = read_flags(h);
    if (rc != NSLI_OK)
        return fail(rc);
#undef CKC
    *out = h;
    return NSLI_OK;
}

void nsli_destroy(nsli_handle h)
{
    if (!h)
        return;
    if (h->stream)
        cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

int nsli_sync(nsli_handle h)
{
    if (!h)
        return NSLI_ERR_ARG;
    CK(cudaStreamSynchronize(h->stream), "synchronize");
    return NSLI_OK;
}

int nsli_update_b(nsli_handle h, const double *b0, int64_t tick)
{
    Trace trace_("nsli_update_b");
    if (!h)
        return NSLI_ERR_ARG;
    if (b0) {
        CK(cudaMemsetAsync(h->flags, 0, sizeof(int), h->stream), "clear flags");
        CK(cudaMemcpyAsync(h->b0_64, b0, (size_t)h->m * 8, cudaMemcpyDefault, h->stream), "copy b0");
        MetaArgs ma;
        ma.meta = h->meta;
        ma.b0_64 = h->b0_64;
        ma.av_64 = h->av_64;
        ma.n2_64 = h->n2_meta;
        ma.scale = h->scale;
        ma.m = h->m;
        ma.flags = h->flags;
        CK(meta_b0_launch(h->storage == NSLI_F64, h->stream, ma), "update row records");
        h->launches += 1;
    }
    if (tick >= 0) {
        const long long t = tick;  // pageable source: staged before the call returns
        CK(cudaMemcpyAsync(&h->st->tick, &t, sizeof t, cudaMemcpyHostToDevice, h->stream), "set tick");
    }
    if (b0)
        return read_flags(h);
    return NSLI_OK;
}

int nsli_update_rows(nsli_handle h, int64_t row0, int64_t rows, int32_t a_dtype, const void *A, int64_t lda,
                     const double *b0)
{
    Trace trace_("nsli_update_rows");
    if (!h)
        return NSLI_ERR_ARG;
    if (h->sparse)
        return set_err(h, NSLI_ERR_UNSUPPORTED, "rows of a sparse matrix are not replaced in place");
    if (row0 < 0 || rows < 0 || row0 + rows > h->m || (rows > 0 && (!A || lda < h->n)))
        return set_err(h, NSLI_ERR_ARG, "bad row range, source or lda");
    if (a_dtype != NSLI_F32 && a_dtype != NSLI_F64)
        return set_err(h, NSLI_ERR_ARG, "source must be binary32 or binary64");
    if ((h->storage == NSLI_BF16 || h->storage == NSLI_FP8E4M3) && a_dtype != NSLI_F32)
        return set_err(h, NSLI_ERR_ARG, "bf16 / fp8 storage needs a binary32 source");
    if (rows == 0)
        return NSLI_OK;
    cudaStream_t s = h->stream;
    CK(cudaMemsetAsync(h->flags, 0, sizeof(int), s), "clear flags");
    const size_t src_eb = a_dtype == NSLI_F64 ? 8 : 4;
    const bool on_device = is_device_ptr(A);
    // rows per launch: all of them for a device source, else a staged chunk
    long long chunk = on_device ? rows : std::max<long long>(1, (256ll << 20) / (long long)(lda * src_eb));
    chunk = std::min<long long>(chunk, rows);
    void *stage = nullptr;
    if (!on_device)
        CK(cudaMalloc(&stage, (size_t)chunk * lda * src_eb), "allocate staging for rows");
    cudaError_t err = cudaSuccess;
    for (long long r0 = 0; r0 < rows && err == cudaSuccess; r0 += chunk) {
        const long long cnt = std::min(chunk, rows - r0);
        UpdateArgs ua;
        if (on_device) {
            ua.src = static_cast<const unsigned char *>(A) + (size_t)r0 * lda * src_eb;
        } else {
            err = cudaMemcpy2DAsync(stage, (size_t)lda * src_eb,
                                    static_cast<const unsigned char *>(A) + (size_t)r0 * lda * src_eb,
                                    (size_t)lda * src_eb, (size_t)h->n * src_eb, (size_t)cnt, cudaMemcpyDefault, s);
            if (err != cudaSuccess)
                break;
            ua.src = stage;
        }
        ua.b0_new = nullptr;
        if (b0) {
            // the new right-hand sides go through the staging buffer (m doubles)
            err = cudaMemcpyAsync(h->dtmp, b0 + r0, (size_t)cnt * 8, cudaMemcpyDefault, s);
            if (err != cudaSuccess)
                break;
            ua.b0_new = h->dtmp;
        }
        ua.lda = lda;
        ua.src_f64 = a_dtype == NSLI_F64 ? 1 : 0;
        ua.A = h->A;
        ua.ld = h->ld;
        ua.n = h->n;
        ua.row0 = row0 + r0;
        ua.rows = cnt;
        ua.b0_64 = h->b0_64;
        ua.av_64 = h->av_64;
        ua.n2_64 = h->n2_meta;
        ua.scale = h->scale;
        ua.meta = h->meta;
        ua.flags = h->flags;
        err = update_rows_launch(h->storage, s, ua);
        h->launches += 1;
        if (err == cudaSuccess && (!on_device || b0) && r0 + cnt < rows)
            err = cudaStreamSynchronize(s);  // staging buffers are reused
    }
    if (err == cudaSuccess) {
        // the records of the rows (rejected rows: rebuilt from their
        // unchanged norm, b0 and scale), as at creation
        MetaArgs ma;
        ma.meta = h->meta;
        ma.b0_64 = h->b0_64;
        ma.av_64 = h->av_64;
        ma.n2_64 = h->n2_meta;
        ma.scale = h->scale;
        ma.m = rows;
        ma.row0 = row0;
        ma.flags = h->flags;
        err = meta_launch(h->storage == NSLI_F64, s, ma);
        h->launches += 1;
    }
    if (stage) {
        if (err == cudaSuccess)
            err = cudaStreamSynchronize(s);
        cudaFree(stage);
    }
    CK(err, "update rows");
    if (h->n2_meta != h->n2_64)
        h->n2_64_valid = false;   // taken again from the stored rows when needed
    return read_flags(h);
}

int nsli_iterate(nsli_handle h, const nsli_params *p, int64_t n_iter)
{
    Trace trace_("nsli_iterate");
    if (!h)
        return NSLI_ERR_ARG;
    int rc = validate_params(h, p);
    if (rc != NSLI_OK)
        return rc;
    if (n_iter < 0)
        return set_err(h, NSLI_ERR_ARG, "n_iter < 0");
    if ((rc = begin_run(h, p, NSLI_STOP_NONE, LLONG_MAX)) != NSLI_OK)
        return rc;
    if (h->resident) {
        const int B = p->block_iters > 0 ? p->block_iters : kResBlock;
        for (long long done = 0; done < n_iter; done += B) {
            CK(sparse_resident_launch(h->storage == NSLI_F64, h->stream, h->sp, h->res_smem,
                                      (int)std::min<long long>(B, n_iter - done)),
               "launch one-CTA iterations");
            h->launches += 1;
        }
        return NSLI_OK;
    }
    const int B = p->block_iters > 0 ? p->block_iters : 32;
    const long long full = n_iter / B;
    const long long rem = n_iter % B;
    const int per = launches_per_iteration(h, p->rule);
    if (full > 0) {
        if ((rc = ensure_graph(h, B, p->rule)) != NSLI_OK)
            return rc;
        for (long long i = 0; i < full; ++i) {
            CK(cudaGraphLaunch(h->graph, h->stream), "launch iteration graph");
            h->launches += (long long)per * B;
        }
    }
    for (long long i = 0; i < rem; ++i) {
        CK(launch_iteration(h, p->rule), "launch iteration");
        h->launches += per;
    }
    return NSLI_OK;
}

int nsli_iterate_timed(nsli_handle h, const nsli_params *p, int64_t n_iter, double *kernel_ms)
{
    Trace trace_("nsli_iterate_timed");
    if (!h || !kernel_ms)
        return NSLI_ERR_ARG;
    int rc = validate_params(h, p);
    if (rc != NSLI_OK)
        return rc;
    if (n_iter < 0 || n_iter > 100000)
        return set_err(h, NSLI_ERR_ARG, "n_iter out of range for the timed run");
    if ((rc = begin_run(h, p, NSLI_STOP_NONE, LLONG_MAX)) != NSLI_OK)
        return rc;
    kernel_ms[0] = 0.0;
    kernel_ms[1] = 0.0;
    const int batch = 64;  // iterations per event batch
    cudaEvent_t ev[3 * batch];
    for (int i = 0; i < 3 * batch; ++i)
        CK(cudaEventCreate(&ev[i]), "create event");
    cudaError_t err = cudaSuccess;
    for (long long done = 0; done < n_iter && err == cudaSuccess; done += batch) {
        const int cnt = (int)std::min<long long>(batch, n_iter - done);
        for (int i = 0; i < cnt && err == cudaSuccess; ++i) {
            cudaEventRecord(ev[3 * i], h->stream);
            if (h->sparse)
                err = sparse_row_launch(h->storage == NSLI_F64, h->stream, h->sp);
            else
                err = map_launch(h->storage, h->vpt, h->guard, h->G, h->consumers, h->smem, h->stream,
                                 map_args(h));
            if (err != cudaSuccess)
                break;
            cudaEventRecord(ev[3 * i + 1], h->stream);
            if (h->sparse) {
                err = sparse_col_launch(h->storage == NSLI_F64, h->stream, h->sp);
                if (err == cudaSuccess && p->rule == NSLI_RULE_MODAP)
                    err = sparse_step_launch(h->storage == NSLI_F64, h->stream, h->sp);
            } else {
                err = reduce_launch(h->storage == NSLI_F64, h->red_grid, h->stream, reduce_args(h));
            }
            cudaEventRecord(ev[3 * i + 2], h->stream);
            h->launches += launches_per_iteration(h, p->rule);
        }
        if (err == cudaSuccess)
            err = cudaStreamSynchronize(h->stream);
        for (int i = 0; i < cnt && err == cudaSuccess; ++i) {
            float a = 0.f, b = 0.f;
            err = cudaEventElapsedTime(&a, ev[3 * i], ev[3 * i + 1]);
            if (err == cudaSuccess)
                err = cudaEventElapsedTime(&b, ev[3 * i + 1], ev[3 * i + 2]);
            kernel_ms[0] += a;
            kernel_ms[1] += b;
        }
    }
    for (int i = 0; i < 3 * batch; ++i)
        cudaEventDestroy(ev[i]);
    CK(err, "timed iterations");
    return read_state(h);
}

int nsli_solve(nsli_handle h, const nsli_params *p, nsli_result *out)
{
    Trace trace_("nsli_solve");
    if (!h)
        return NSLI_ERR_ARG;
    int rc = validate_params(h, p);
    if (rc != NSLI_OK)
        return rc;
    if ((rc = begin_run(h, p, p->stop, p->max_iter)) != NSLI_OK)
        return rc;
    const int B = p->block_iters > 0 ? p->block_iters : (h->resident ? kResBlock : 32);
    if (!h->resident && (rc = ensure_graph(h, B, p->rule)) != NSLI_OK)
        return rc;
    const int per = launches_per_iteration(h, p->rule);
    int status = NSLI_NOT_CONVERGED;
    // every block either makes B updates or ends the run; a rejected
    // candidate forces one update, so this bound is never reached
    const long long max_blocks = p->max_iter / B + p->max_iter + 4;
    bool finished = false;
    int rejected = 0;
    for (long long blk = 0; blk < max_blocks && !finished; ++blk) {
        if (h->resident) {
            CK(sparse_resident_launch(h->storage == NSLI_F64, h->stream, h->sp, h->res_smem, B),
               "launch one-CTA iterations");
            h->launches += 1;
        } else {
            CK(cudaGraphLaunch(h->graph, h->stream), "launch iteration graph");
            h->launches += (long long)per * B;
        }
        if ((rc = read_state(h)) != NSLI_OK)
            return rc;
        const int sst = h->st_host->status;
        if (sst == ST_RUNNING)
            continue;
        if (sst == ST_CANDIDATE) {
            if ((rc = run_verify(h)) != NSLI_OK)
                return rc;
            bool accept;
            if (p->stop == NSLI_STOP_EPSMEM)
                accept = h->last_check.max_viol_norm < p->eps;
            else if (p->stop == NSLI_STOP_MAXVIOL_REL)
                accept = h->last_check.max_viol <= p->eps * h->last_check.max_abs_b;
            else
                accept = h->last_check.h == 0;
            if (accept) {
                status = NSLI_OK;
                finished = true;
            } else {
                CK(state_resume_launch(h->stream, h->st), "resume");
                h->launches += 1;
                rejected += 1;
            }
            continue;
        }
        status = sst;  // NSLI_OK (step rule) or NSLI_NOT_CONVERGED
        finished = true;
    }
    if ((rc = read_state(h)) != NSLI_OK)
        return rc;
    if ((rc = run_verify(h)) != NSLI_OK)
        return rc;
    nsli_result r = h->last_check;
    r.iters = h->st_host->it;
    r.tick = h->st_host->tick;
    r.status = status;
    r.rejected = rejected;
    r.last_step_norm = std::sqrt(h->st_host->dx2);
    h->last_check = r;
    if (out)
        *out = r;
    return status;
}

int nsli_residual_max(nsli_handle h, double *max_viol, double *max_viol_norm)
{
    Trace trace_("nsli_residual_max");
    if (!h)
        return NSLI_ERR_ARG;
    int rc = run_verify(h);
    if (rc != NSLI_OK)
        return rc;
    if (max_viol)
        *max_viol = h->last_check.max_viol;
    if (max_viol_norm)
        *max_viol_norm = h->last_check.max_viol_norm;
    return NSLI_OK;
}

int nsli_map_reduce(nsli_handle h, double *y, int64_t *violated, double *stats)
{
    Trace trace_("nsli_map_reduce");
    if (!h)
        return NSLI_ERR_ARG;
    if (h->sparse) {
        SparseArgs sa = h->sp;
        sa.ignore_done = 1;
        sa.mode = 1;
        CK(sparse_row_launch(h->storage == NSLI_F64, h->stream, sa), "launch Map");
        CK(sparse_col_launch(h->storage == NSLI_F64, h->stream, sa), "launch Reduce");
    } else {
        MapArgs ma = map_args(h);
        ma.ignore_done = 1;  // also after a finished run
        CK(map_launch(h->storage, h->vpt, h->guard, h->G, h->consumers, h->smem, h->stream, ma), "launch Map");
        CK(reduce_only_launch(h->storage == NSLI_F64, h->red_grid, h->stream, reduce_args(h), h->ybuf),
           "launch Reduce");
    }
    h->launches += 2;
    if (y)
        CK(cudaMemcpyAsync(y, h->ybuf, (size_t)h->n * 8, cudaMemcpyDefault, h->stream), "copy y");
    int rc = read_state(h);
    if (rc != NSLI_OK)
        return rc;
    if (violated)
        *violated = h->st_host->h;
    if (stats) {
        stats[0] = h->st_host->maxviol;
        stats[1] = h->st_host->maxnorm;
        stats[2] = h->st_host->maxb;
    }
    return NSLI_OK;
}

int nsli_get_x(nsli_handle h, double *x)
{
    Trace trace_("nsli_get_x");
    if (!h || !x)
        return NSLI_ERR_ARG;
    CK(cudaMemcpyAsync(x, h->x64, (size_t)h->n * 8, cudaMemcpyDefault, h->stream), "copy x");
    CK(cudaStreamSynchronize(h->stream), "synchronize");
    return NSLI_OK;
}

int nsli_set_x(nsli_handle h, const double *x)
{
    Trace trace_("nsli_set_x");
    if (!h || !x)
        return NSLI_ERR_ARG;
    CK(cudaMemsetAsync(h->flags, 0, sizeof(int), h->stream), "clear flags");
    CK(cudaMemcpyAsync(h->dtmp, x, (size_t)h->n * 8, cudaMemcpyDefault, h->stream), "copy x");
    CK(x_from_f64_launch(h->storage == NSLI_F64, h->stream, h->dtmp, h->x64, h->x, h->n, h->ld, h->flags),
       "convert x");
    h->launches += 1;
    return read_flags(h);
}

int nsli_test_inject_timeout(nsli_handle h, int32_t slot)
{
    if (!h || slot < 0)
        return NSLI_ERR_ARG;
    if (h->sparse || h->vpt == 0)
        return set_err(h, NSLI_ERR_UNSUPPORTED, "only the dense register-resident Map streams bulk copies");
    MapArgs ma = map_args(h);
    ma.ignore_done = 1;
    ma.skip_slot = slot;
    CK(cudaMemsetAsync(&h->st->error, 0, sizeof(int), h->stream), "clear error");
    CK(map_launch(h->storage, h->vpt, h->guard, h->G, h->consumers, h->smem, h->stream, ma), "launch Map");
    h->launches += 1;
    int rc = read_state(h);
    CK(cudaMemsetAsync(&h->st->error, 0, sizeof(int), h->stream), "clear error");
    CK(cudaStreamSynchronize(h->stream), "synchronize");
    return rc;
}

int nsli_get_stored_rows(nsli_handle h, int64_t row0, int64_t rows, double *out)
{
    if (!h || !out || row0 < 0 || rows < 0 || row0 + rows > h->m)
        return NSLI_ERR_ARG;
    if (rows == 0)
        return NSLI_OK;
    double *tmp = nullptr;
    CK(cudaMalloc((void **)&tmp, (size_t)rows * h->n * 8), "allocate row copy");
    cudaError_t e;
    if (h->sparse) {
        e = cudaMemsetAsync(tmp, 0, (size_t)rows * h->n * 8, h->stream);
        if (e == cudaSuccess)
            e = sparse_rows_launch(h->storage == NSLI_F64, h->stream, h->sp, row0, rows, tmp);
    } else {
        e = stored_rows_launch(h->storage, h->stream, h->A, h->scale, h->ld, h->n, row0, rows, tmp);
    }
    h->launches += 1;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, tmp, (size_t)rows * h->n * 8, cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(h->stream);
    cudaFree(tmp);
    CK(e, "copy stored rows");
    return NSLI_OK;
}

int nsli_get_norms2(nsli_handle h, double *out)
{
    if (!h || !out)
        return NSLI_ERR_ARG;
    int rc = ensure_norms64(h);
    if (rc != NSLI_OK)
        return rc;
    CK(cudaMemcpyAsync(out, h->n2_64, (size_t)h->m * 8, cudaMemcpyDefault, h->stream), "copy norms");
    CK(cudaStreamSynchronize(h->stream), "synchronize");
    return NSLI_OK;
}

int nsli_get_result(nsli_handle h, nsli_result *out)
{
    if (!h || !out)
        return NSLI_ERR_ARG;
    int rc = read_state(h);
    if (rc != NSLI_OK)
        return rc;
    nsli_result r = h->last_check;
    r.iters = h->st_host->it;
    r.tick = h->st_host->tick;
    const int sst = h->st_host->status;
    r.status = sst == ST_RUNNING ? NSLI_RUNNING : (sst == ST_CANDIDATE ? NSLI_CANDIDATE : sst);
    r.last_step_norm = std::sqrt(h->st_host->dx2);
    *out = r;
    return NSLI_OK;
}

// ---- row shards (ModAPL, Section 3) ----------------------------------------

int nsli_shard_begin(nsli_handle h, const nsli_params *p)
{
    Trace trace_("nsli_shard_begin");
    if (!h)
        return NSLI_ERR_ARG;
    int rc = validate_params(h, p);
    if (rc != NSLI_OK)
        return rc;
    if (!h->shard_dx)
        CK(cudaMalloc((void **)&h->shard_dx, (size_t)shard_step_blocks(h->n) * 8), "allocate exchange partials");
    return begin_run(h, p, p->stop, p->max_iter);
}

int nsli_shard_map(nsli_handle h, double *record)
{
    Trace trace_("nsli_shard_map");
    if (!h || !record)
        return NSLI_ERR_ARG;
    if (h->sparse) {
        SparseArgs sa = h->sp;
        sa.ignore_done = 1;
        sa.mode = 1;
        CK(sparse_row_launch(h->storage == NSLI_F64, h->stream, sa), "launch Map");
        CK(sparse_col_launch(h->storage == NSLI_F64, h->stream, sa), "launch local Reduce");
    } else {
        MapArgs ma = map_args(h);
        ma.ignore_done = 1;
        CK(map_launch(h->storage, h->vpt, h->guard, h->G, h->consumers, h->smem, h->stream, ma), "launch Map");
        CK(reduce_only_launch(h->storage == NSLI_F64, h->red_grid, h->stream, reduce_args(h), h->ybuf),
           "launch local Reduce");
    }
    CK(shard_pack_launch(h->stream, h->st, h->ybuf, h->n, record), "write the record");
    h->launches += 3;
    return NSLI_OK;
}

int nsli_shard_step(nsli_handle h, const double *records, int32_t nranks, int32_t force_step)
{
    Trace trace_("nsli_shard_step");
    if (!h || !records || nranks < 1)
        return NSLI_ERR_ARG;
    if (!h->shard_dx)
        return set_err(h, NSLI_ERR_ARG, "nsli_shard_begin has not been called on this handle");
    if (force_step) {
        CK(state_resume_launch(h->stream, h->st), "resume");
        h->launches += 1;
    }
    ShardStepArgs a;
    a.recs = records;
    a.nranks = nranks;
    a.n = h->n;
    a.x = h->x;
    a.x64 = h->x64;
    a.ybuf = h->ybuf;
    a.part_dx = h->shard_dx;
    a.st = h->st;
    CK(shard_step_launch(h->storage == NSLI_F64, h->stream, a), "launch exchange step");
    h->launches += 1;
    return NSLI_OK;
}

}  // extern "C"

// ============================================================== pool ======
//
// Continuous batching of many problems: each problem is an nsli_solver
// (its own device buffers, state and ring configuration); a round is one
// grouped Map launch over the work items of every live problem and one
// grouped reduce-and-step launch.  A problem's items (row blocks) and
// thread mapping depend only on that problem, so its iterates are the same
// alone and in any mix.

struct nsli_pool_s {
    int storage = NSLI_BF16;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 1;
    long long max_bytes = 0, used_bytes = 0;
    std::vector<nsli_solver *> slots;       // slot id -> problem (nullptr when free)
    std::vector<long long> slot_bytes;
    std::vector<int> slot_items;
    bool dirty = true;
    int n_items = 0, n_red = 0, n_live = 0;
    size_t smem = 0;
    GroupProblem *d_probs = nullptr;
    GroupItem *d_items = nullptr;
    GroupRed *d_red = nullptr;
    size_t cap_probs = 0, cap_items = 0, cap_red = 0;
    DevState **d_sts = nullptr;
    long long *d_ticks = nullptr;
    size_t cap_ticks = 0;
    DevState *h_states = nullptr;            // pinned mirror for polling
    size_t cap_states = 0;
    std::vector<int> live_order;             // slot ids in the current tables
    long long launches = 0;
    std::string last_error;

    // persistent launches (nsli_pool_launch): host-mapped control block,
    // device scratch, and what the last launch reported
    ServeCtrl *ctrl_host = nullptr;          // pinned, mapped
    ServeCtrl *ctrl_dev = nullptr;           // its device address
    ServeSync *d_sync = nullptr;
    long long *d_tick0 = nullptr;
    int *d_reported = nullptr;
    size_t cap_serve = 0;
    size_t serve_smem = 0;
    int serve_bps = 0;
    bool running = false;
    bool have_done_list = false;             // poll may restrict itself to done_slots
    std::vector<int> done_slots;
};

namespace {

int perr(nsli_pool p, int code, const std::string &msg)
{
    if (p)
        p->last_error = msg;
    return code;
}
#define PCK(call, what)                                                                                      \
    do {                                                                                                     \
        cudaError_t e_ = (call);                                                                             \
        if (e_ != cudaSuccess)                                                                               \
            return perr(p, e_ == cudaErrorMemoryAllocation ? NSLI_ERR_OOM : NSLI_ERR_CUDA,                  \
                        std::string(what) + ": " + cudaGetErrorString(e_));                                  \
    } while (0)

// device bytes a problem will take (A, records, vectors, partials)
long long problem_bytes(int storage, long long m, long long n, int num_sms)
{
    const int eb = storage == NSLI_F64 ? 8 : storage == NSLI_F32 ? 4 : storage == NSLI_BF16 ? 2 : 1;
    const long long ld = n + 16;
    const long long G = std::min<long long>(num_sms, m);
    return m * ld * eb + m * (32 + 5 * 8 + 4) + G * ld * 8 + ld * 40 + (1 << 16);
}

int items_of(nsli_solver *h)
{
    // about 1 MiB of A per item, at most one item per Map CTA of the handle
    const long long bytes = h->m * (long long)h->row_bytes;
    const long long want = (bytes + (1ll << 20) - 1) >> 20;
    return (int)std::max<long long>(1, std::min<long long>(want, h->G));
}

template <typename T> int grow(nsli_pool p, T **buf, size_t *cap, size_t need)
{
    if (*cap >= need)
        return NSLI_OK;
    size_t c = std::max<size_t>(need, *cap * 2 + 16);
    if (*buf)
        cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    PCK(cudaMalloc((void **)buf, c * sizeof(T)), "grow pool table");
    *cap = c;
    return NSLI_OK;
}

int rebuild_tables(nsli_pool p)
{
    std::vector<GroupProblem> probs;
    std::vector<GroupItem> items;
    std::vector<GroupRed> reds;
    p->live_order.clear();
    size_t smem = kSmemHeader;
    for (size_t sid = 0; sid < p->slots.size(); ++sid) {
        nsli_solver *h = p->slots[sid];
        if (!h)
            continue;
        const int pi = (int)probs.size();
        const int nitems = p->slot_items[sid];
        GroupProblem gp;
        gp.map = map_args(h);
        gp.red = reduce_args(h);
        gp.red.G = nitems;
        gp.nt = h->consumers;
        gp.vpt = h->vpt;
        gp.red_blocks = h->red_grid;
        gp.first_red = (int)reds.size();
        probs.push_back(gp);
        const long long base = h->m / nitems, rem = h->m % nitems;
        long long r = 0;
        for (int q = 0; q < nitems; ++q) {
            const long long cnt = base + (q < rem ? 1 : 0);
            items.push_back(GroupItem{pi, q, r, r + cnt});
            r += cnt;
        }
        for (int b = 0; b < h->red_grid; ++b)
            reds.push_back(GroupRed{pi, b});
        smem = std::max(smem, h->smem);
        p->live_order.push_back((int)sid);
    }
    // The persistent launch takes the items in table order from a shared
    // counter: longest first (list scheduling by longest processing time),
    // so the long items start early and the short ones fill the end of the
    // phase.  An item's time is estimated as its bytes of A over the share
    // of the CTA's threads its rows occupy.  Which CTA maps an item changes
    // no result.
    auto est = [&probs](const GroupItem &it) {
        const GroupProblem &gp = probs[it.prob];
        return (double)(it.row_end - it.row_begin) * (double)gp.map.row_bytes * (double)kMapMaxConsumers /
               (double)std::max(1, gp.nt);
    };
    std::stable_sort(items.begin(), items.end(),
                     [&est](const GroupItem &a, const GroupItem &b) { return est(a) > est(b); });
    int rc;
    if ((rc = grow(p, &p->d_probs, &p->cap_probs, std::max<size_t>(1, probs.size()))) != NSLI_OK)
        return rc;
    if ((rc = grow(p, &p->d_items, &p->cap_items, std::max<size_t>(1, items.size()))) != NSLI_OK)
        return rc;
    if ((rc = grow(p, &p->d_red, &p->cap_red, std::max<size_t>(1, reds.size()))) != NSLI_OK)
        return rc;
    PCK(cudaStreamSynchronize(p->stream), "synchronize");
    if (!probs.empty()) {
        PCK(cudaMemcpy(p->d_probs, probs.data(), probs.size() * sizeof(GroupProblem), cudaMemcpyHostToDevice),
            "upload problems");
        PCK(cudaMemcpy(p->d_items, items.data(), items.size() * sizeof(GroupItem), cudaMemcpyHostToDevice),
            "upload items");
        PCK(cudaMemcpy(p->d_red, reds.data(), reds.size() * sizeof(GroupRed), cudaMemcpyHostToDevice),
            "upload reduce table");
    }
    if (smem > p->smem) {
        PCK(map_group_prepare(p->storage, smem), "configure grouped Map");
        p->smem = smem;
    }
    p->n_items = (int)items.size();
    p->n_red = (int)reds.size();
    p->n_live = (int)probs.size();
    p->dirty = false;
    return NSLI_OK;
}

}  // namespace

extern "C" {

int nsli_pool_create(nsli_pool *out, int32_t storage, int64_t max_bytes, void *stream)
{
    if (!out || (storage != NSLI_BF16 && storage != NSLI_F32) || max_bytes < 0)
        return NSLI_ERR_ARG;
    *out = nullptr;
    nsli_pool p = new nsli_pool_s();
    p->storage = storage;
    p->max_bytes = max_bytes;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete p;
        return NSLI_ERR_CUDA;
    }
    if (stream) {
        p->stream = static_cast<cudaStream_t>(stream);
    } else {
        if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete p;
            return NSLI_ERR_CUDA;
        }
        p->own_stream = true;
    }
    *out = p;
    return NSLI_OK;
}

void nsli_pool_destroy(nsli_pool p)
{
    if (!p)
        return;
    cudaStreamSynchronize(p->stream);
    for (nsli_solver *h : p->slots)
        if (h) {
            h->stream = nullptr;  // the pool's stream is not the handle's to destroy
            h->own_stream = false;
            free_all(h);
            delete h;
        }
    void *bufs[] = {p->d_probs, p->d_items, p->d_red, p->d_sts, p->d_ticks, p->d_sync, p->d_tick0, p->d_reported};
    for (void *b : bufs)
        if (b)
            cudaFree(b);
    if (p->h_states)
        cudaFreeHost(p->h_states);
    if (p->ctrl_host)
        cudaFreeHost(p->ctrl_host);
    if (p->own_stream)
        cudaStreamDestroy(p->stream);
    delete p;
}

int nsli_pool_add(nsli_pool p, int64_t m, int64_t n, const float *A, int64_t lda, const double *b0,
                  const double *Av, const double *x0, const nsli_params *prm, int64_t *slot)
{
    Trace trace_("nsli_pool_add");
    if (!p || !slot || !prm)
        return NSLI_ERR_ARG;
    if (p && p->running)
        return perr(p, NSLI_ERR_ARG, "a persistent launch is running: call nsli_pool_wait first");
    if (m < 1 || n < 1 || lda < n || !A || !b0 || !x0)
        return perr(p, NSLI_ERR_ARG, "bad problem arguments");
    // admission by memory: the pool's budget and the device's free HBM
    const long long need = problem_bytes(p->storage, m, n, p->num_sms);
    if (p->max_bytes > 0 && p->used_bytes + need > p->max_bytes)
        return perr(p, NSLI_ERR_OOM, "problem does not fit the pool's memory budget");
    size_t freeb = 0, totalb = 0;
    PCK(cudaMemGetInfo(&freeb, &totalb), "query free memory");
    if ((long long)freeb < need + (256ll << 20))
        return perr(p, NSLI_ERR_OOM, "problem does not fit the free device memory");
    nsli_handle h = nullptr;
    int rc = nsli_create(&h, m, n, p->storage, NSLI_F32, A, lda, b0, nullptr, Av, x0, p->stream);
    if (rc != NSLI_OK)
        return perr(p, rc, "create problem");
    if (h->vpt == 0) {
        h->stream = nullptr;
        free_all(h);
        delete h;
        return perr(p, NSLI_ERR_UNSUPPORTED, "the pool serves rows up to the register-resident limit");
    }
    // control state of the problem's run
    if ((rc = validate_params(h, prm)) != NSLI_OK || (rc = begin_run(h, prm, prm->stop, prm->max_iter)) != NSLI_OK) {
        h->stream = nullptr;
        free_all(h);
        delete h;
        return perr(p, rc, "problem parameters");
    }
    size_t sid = 0;
    while (sid < p->slots.size() && p->slots[sid])
        ++sid;
    if (sid == p->slots.size()) {
        p->slots.push_back(nullptr);
        p->slot_bytes.push_back(0);
        p->slot_items.push_back(0);
    }
    p->slots[sid] = h;
    p->slot_bytes[sid] = need;
    p->slot_items[sid] = items_of(h);
    p->used_bytes += need;
    p->launches += h->launches;
    p->dirty = true;
    *slot = (int64_t)sid;
    return NSLI_OK;
}

int nsli_pool_remove(nsli_pool p, int64_t slot)
{
    if (p && p->running)
        return perr(p, NSLI_ERR_ARG, "a persistent launch is running: call nsli_pool_wait first");
    if (!p || slot < 0 || slot >= (int64_t)p->slots.size() || !p->slots[slot])
        return NSLI_ERR_ARG;
    PCK(cudaStreamSynchronize(p->stream), "synchronize");
    nsli_solver *h = p->slots[slot];
    h->stream = nullptr;
    h->own_stream = false;
    free_all(h);
    delete h;
    p->slots[slot] = nullptr;
    p->used_bytes -= p->slot_bytes[slot];
    p->dirty = true;
    return NSLI_OK;
}

int nsli_pool_step(nsli_pool p, int32_t rounds)
{
    Trace trace_("nsli_pool_step");
    if (!p || rounds < 0)
        return NSLI_ERR_ARG;
    if (p && p->running)
        return perr(p, NSLI_ERR_ARG, "a persistent launch is running: call nsli_pool_wait first");
    if (p->dirty) {
        int rc = rebuild_tables(p);
        if (rc != NSLI_OK)
            return rc;
    }
    if (p->n_live == 0)
        return NSLI_OK;
    const bool f64 = p->storage == NSLI_F64;
    for (int r = 0; r < rounds; ++r) {
        PCK(map_group_launch(p->storage, p->n_items, p->smem, p->stream, p->d_probs, p->d_items), "grouped Map");
        PCK(reduce_group_launch(f64, p->n_red, p->stream, p->d_probs, p->d_red), "grouped reduce");
        p->launches += 2;
    }
    return NSLI_OK;
}

int nsli_pool_set_ticks(nsli_pool p, const int64_t *slots, const int64_t *ticks, int64_t count)
{
    if (p && p->running)
        return perr(p, NSLI_ERR_ARG, "a persistent launch is running: call nsli_pool_wait first");
    if (!p || count < 0 || (count > 0 && (!slots || !ticks)))
        return NSLI_ERR_ARG;
    if (count == 0)
        return NSLI_OK;
    std::vector<DevState *> sts((size_t)count);
    for (int64_t i = 0; i < count; ++i) {
        if (slots[i] < 0 || slots[i] >= (int64_t)p->slots.size() || !p->slots[slots[i]])
            return perr(p, NSLI_ERR_ARG, "no problem in that slot");
        sts[i] = p->slots[slots[i]]->st;
    }
    int rc;
    size_t cap_sts = p->cap_ticks, cap_vals = p->cap_ticks;
    if ((rc = grow(p, &p->d_sts, &cap_sts, (size_t)count)) != NSLI_OK)
        return rc;
    if ((rc = grow(p, &p->d_ticks, &cap_vals, (size_t)count)) != NSLI_OK)
        return rc;
    p->cap_ticks = std::min(cap_sts, cap_vals);
    PCK(cudaStreamSynchronize(p->stream), "synchronize");
    PCK(cudaMemcpy(p->d_sts, sts.data(), (size_t)count * sizeof(DevState *), cudaMemcpyHostToDevice), "upload states");
    PCK(cudaMemcpy(p->d_ticks, ticks, (size_t)count * 8, cudaMemcpyHostToDevice), "upload ticks");
    PCK(set_ticks_launch(p->stream, p->d_sts, p->d_ticks, (int)count), "set ticks");
    p->launches += 1;
    return NSLI_OK;
}

int nsli_pool_poll(nsli_pool p, int64_t *slots, int32_t *status, int64_t *iters, int64_t cap, int64_t *count)
{
    Trace trace_("nsli_pool_poll");
    if (p && p->running)
        return perr(p, NSLI_ERR_ARG, "a persistent launch is running: call nsli_pool_wait first");
    if (!p || !count || cap < 0 || (cap > 0 && (!slots || !status || !iters)))
        return NSLI_ERR_ARG;
    *count = 0;
    const size_t ns = p->slots.size();
    if (p->cap_states < ns) {
        if (p->h_states)
            cudaFreeHost(p->h_states);
        p->h_states = nullptr;
        PCK(cudaMallocHost((void **)&p->h_states, std::max<size_t>(ns, 16) * sizeof(DevState)), "pinned states");
        p->cap_states = std::max<size_t>(ns, 16);
    }
    // after a persistent launch only the problems it reported can have
    // stopped; otherwise every live problem is read
    std::vector<int> check;
    if (p->have_done_list) {
        check = p->done_slots;
    } else {
        for (size_t sid = 0; sid < ns; ++sid)
            if (p->slots[sid])
                check.push_back((int)sid);
    }
    p->have_done_list = false;
    for (int sid : check)
        if (p->slots[sid])
            PCK(cudaMemcpyAsync(&p->h_states[sid], p->slots[sid]->st, sizeof(DevState), cudaMemcpyDeviceToHost,
                                p->stream),
                "read state");
    PCK(cudaStreamSynchronize(p->stream), "synchronize");
    for (int sid : check) {
        nsli_solver *h = p->slots[sid];
        if (!h)
            continue;
        DevState &s = p->h_states[sid];
        int st = s.status;
        if (s.error & ERRF_TIMEOUT)
            st = NSLI_ERR_TIMEOUT;
        if (st == ST_CANDIDATE) {
            p->launches += 1;
            int rc = run_verify(h);
            if (rc != NSLI_OK)
                return perr(p, rc, "binary64 check");
            bool accept;
            if (s.stop == NSLI_STOP_EPSMEM)
                accept = h->last_check.max_viol_norm < s.eps;
            else if (s.stop == NSLI_STOP_MAXVIOL_REL)
                accept = h->last_check.max_viol <= s.eps * h->last_check.max_abs_b;
            else
                accept = h->last_check.h == 0;
            if (accept) {
                st = NSLI_OK;
                const int ok = NSLI_OK;  // record the confirmed stop on the device
                PCK(cudaMemcpyAsync(&h->st->status, &ok, sizeof ok, cudaMemcpyHostToDevice, p->stream),
                    "record status");
            } else {
                PCK(state_resume_launch(p->stream, h->st), "resume");
                p->launches += 1;
                continue;
            }
        }
        if (st == ST_RUNNING)
            continue;
        if (*count < cap) {
            slots[*count] = (int64_t)sid;
            status[*count] = st;
            iters[*count] = s.it;
        }
        ++*count;
    }
    return NSLI_OK;
}

int nsli_pool_launch(nsli_pool p, int64_t max_rounds, double max_seconds, double tick_s)
{
    Trace trace_("nsli_pool_launch");
    if (!p || max_rounds < 0 || !(max_seconds > 0.0) || !std::isfinite(max_seconds) || !(tick_s >= 0.0) ||
        !std::isfinite(tick_s))
        return NSLI_ERR_ARG;
    if (p->running)
        return perr(p, NSLI_ERR_ARG, "a persistent launch is already running");
    if (p->dirty) {
        int rc = rebuild_tables(p);
        if (rc != NSLI_OK)
            return rc;
    }
    if (p->n_live == 0)
        return NSLI_OK;
    if (p->n_live > kServeMaxProblems)
        return perr(p, NSLI_ERR_UNSUPPORTED, "more live problems than one persistent launch serves");
    if (!p->ctrl_host) {
        PCK(cudaHostAlloc((void **)&p->ctrl_host, sizeof(ServeCtrl), cudaHostAllocMapped), "pinned control block");
        PCK(cudaHostGetDevicePointer((void **)&p->ctrl_dev, p->ctrl_host, 0), "map control block");
        PCK(cudaMalloc((void **)&p->d_sync, sizeof(ServeSync)), "allocate grid barrier");
    }
    int rc;
    size_t cap_t = p->cap_serve, cap_r = p->cap_serve;
    if ((rc = grow(p, &p->d_tick0, &cap_t, (size_t)p->n_live)) != NSLI_OK)
        return rc;
    if ((rc = grow(p, &p->d_reported, &cap_r, (size_t)p->n_live)) != NSLI_OK)
        return rc;
    p->cap_serve = std::min(cap_t, cap_r);
    // the reduce phase keeps its shared block in the ring's stage area
    const size_t smem = std::max<size_t>(p->smem, 16384);
    if (smem != p->serve_smem || p->serve_bps == 0) {
        int bps = 0;
        PCK(serve_prepare(p->storage, smem, &bps), "configure persistent kernel");
        if (bps < 1)
            return perr(p, NSLI_ERR_UNSUPPORTED, "the persistent kernel does not fit an SM");
        p->serve_bps = bps;
        p->serve_smem = smem;
    }
    // the launch's control block and barrier start from zero
    p->ctrl_host->yield = 0;
    p->ctrl_host->error = 0;
    p->ctrl_host->rounds = 0;
    p->ctrl_host->done_count = 0;
    PCK(cudaMemsetAsync(p->d_sync, 0, sizeof(ServeSync), p->stream), "clear grid barrier");
    ServeArgs a;
    a.probs = p->d_probs;
    a.items = p->d_items;
    a.reds = p->d_red;
    a.nprob = p->n_live;
    a.nitems = p->n_items;
    a.nreds = p->n_red;
    a.tick0 = p->d_tick0;
    a.reported = p->d_reported;
    a.sync = p->d_sync;
    a.ctrl = p->ctrl_dev;
    a.max_rounds = max_rounds;
    a.max_ns = (unsigned long long)(max_seconds * 1e9);
    a.tick_ns = (unsigned long long)(tick_s * 1e9);
    if (tick_s > 0.0 && a.tick_ns == 0)
        a.tick_ns = 1;
    const int grid = p->serve_bps * p->num_sms;
    PCK(serve_launch(p->storage, grid, smem, p->stream, a), "persistent launch");
    p->launches += 1;
    p->running = true;
    return NSLI_OK;
}

int nsli_pool_yield(nsli_pool p)
{
    if (!p)
        return NSLI_ERR_ARG;
    if (p->running) {
        std::atomic_thread_fence(std::memory_order_seq_cst);
        *(volatile int *)&p->ctrl_host->yield = 1;
        std::atomic_thread_fence(std::memory_order_seq_cst);
    }
    return NSLI_OK;
}

int64_t nsli_pool_stopped(nsli_pool p)
{
    if (!p || !p->running)
        return 0;
    const unsigned int c = *(volatile unsigned int *)&p->ctrl_host->done_count;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    return (int64_t)c;
}

int nsli_pool_wait(nsli_pool p, int64_t *rounds)
{
    Trace trace_("nsli_pool_wait");
    if (!p)
        return NSLI_ERR_ARG;
    if (!p->running) {
        if (rounds)
            *rounds = 0;
        return NSLI_OK;
    }
    const cudaError_t e = cudaStreamSynchronize(p->stream);
    p->running = false;
    if (e != cudaSuccess)
        return perr(p, NSLI_ERR_CUDA, std::string("persistent launch: ") + cudaGetErrorString(e));
    std::atomic_thread_fence(std::memory_order_seq_cst);
    ServeCtrl *c = p->ctrl_host;
    if (rounds)
        *rounds = (int64_t)c->rounds;
    p->done_slots.clear();
    const unsigned int nd = std::min<unsigned int>(c->done_count, (unsigned int)kServeMaxProblems);
    for (unsigned int k = 0; k < nd; ++k) {
        const int q = c->done[k].prob;
        if (q >= 0 && q < (int)p->live_order.size())
            p->done_slots.push_back(p->live_order[q]);
    }
    p->have_done_list = true;
    if (c->error)
        return perr(p, NSLI_ERR_TIMEOUT, "a grid barrier wait of the persistent launch expired");
    return NSLI_OK;
}

int nsli_pool_get_x(nsli_pool p, int64_t slot, double *x)
{
    if (p && p->running)
        return perr(p, NSLI_ERR_ARG, "a persistent launch is running: call nsli_pool_wait first");
    if (!p || slot < 0 || slot >= (int64_t)p->slots.size() || !p->slots[slot])
        return NSLI_ERR_ARG;
    return nsli_get_x(p->slots[slot], x);
}

int nsli_pool_residual_max(nsli_pool p, int64_t slot, double *max_viol, double *max_viol_norm)
{
    if (p && p->running)
        return perr(p, NSLI_ERR_ARG, "a persistent launch is running: call nsli_pool_wait first");
    if (!p || slot < 0 || slot >= (int64_t)p->slots.size() || !p->slots[slot])
        return NSLI_ERR_ARG;
    return nsli_residual_max(p->slots[slot], max_viol, max_viol_norm);
}

int64_t nsli_pool_live(nsli_pool p)
{
    if (!p)
        return 0;
    int64_t c = 0;
    for (nsli_solver *h : p->slots)
        c += h ? 1 : 0;
    return c;
}

int64_t nsli_pool_bytes_used(nsli_pool p) { return p ? (int64_t)p->used_bytes : 0; }

int64_t nsli_pool_launch_count(nsli_pool p) { return p ? (int64_t)p->launches : 0; }

int nsli_pool_sync(nsli_pool p)
{
    if (!p)
        return NSLI_ERR_ARG;
    PCK(cudaStreamSynchronize(p->stream), "synchronize");
    return NSLI_OK;
}

const char *nsli_pool_last_error(nsli_pool p) { return p ? p->last_error.c_str() : ""; }

}  // extern "C"
