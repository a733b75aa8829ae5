// nsli_shard.cu -- the exchange step of the row-sharded form (ModAPL).
//
// Section 3 splits the list of inequalities into sublists, one per worker:
// every worker runs the Map and a local Reduce over its own rows, the
// partial sums are added, the step is taken and the new x is used by all.
// Here a worker is one handle holding a contiguous block of rows (normally
// one GPU of a process group).  Its Map and local Reduce are the usual
// kernels; shard_pack_kernel writes their outputs as a "record"
//   [ h, max r_i, max r_i / ||a_i||, max |b_i|, y_0 .. y_{n-1} ]   (doubles)
// that the caller gathers from every worker (an allgather) into one array
// of R records in worker order.  shard_step_kernel then takes, on every
// worker alike, the global Reduce -- y = sum over workers w = 0..R-1 in
// that order (binary64), h = sum of the h_w, the maxima of the maxima --
// the stop decision and the step, exactly as the single-handle reduce
// kernel does.  Identical records give identical bits on every worker, so
// the iterates of all workers stay equal without a broadcast of x.
#include "nsli.h"
#include "nsli_internal.h"

namespace nsli {
namespace {

constexpr int kShardThreads = 256;

template <typename T> __device__ __forceinline__ T shard_warp_sum(T v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Record of one worker after its Map and local Reduce (y in ybuf, counts
// and maxima in the state).
__global__ void __launch_bounds__(kShardThreads) shard_pack_kernel(const DevState *st, const double *ybuf,
                                                                   long long n, double *rec)
{
    const long long j = (long long)blockIdx.x * kShardThreads + threadIdx.x;
    if (j == 0) {
        rec[0] = (double)st->h;
        rec[1] = st->maxviol;
        rec[2] = st->maxnorm;
        rec[3] = st->maxb;
    }
    if (j < n)
        rec[kShardHeader + j] = ybuf[j];
}

struct ShardShared {
    long long h;
    double mv, mn, mb;
    double red[kShardThreads / 32];
    int last;
};

template <typename Acc>
__global__ void __launch_bounds__(kShardThreads) shard_step_kernel(const ShardStepArgs p)
{
    DevState *st = p.st;
    if (*(volatile int *)&st->done)
        return;
    __shared__ ShardShared sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long len = p.n + kShardHeader;
    if (threadIdx.x == 0) {
        // counts and maxima of all workers, in worker order (exact)
        long long h = 0;
        double mv = -INFINITY, mn = -INFINITY, mb = 0.0;
        for (int w = 0; w < p.nranks; ++w) {
            const double *r = p.recs + (long long)w * len;
            h += (long long)r[0];
            mv = fmax(mv, r[1]);
            mn = fmax(mn, r[2]);
            mb = fmax(mb, r[3]);
        }
        sh.h = h;
        sh.mv = mv;
        sh.mn = mn;
        sh.mb = mb;
    }
    __syncthreads();
    const long long h = sh.h;
    const double mv = sh.mv, mn = sh.mn, mb = sh.mb;
    const int stop = st->stop;
    const double eps = st->eps;
    const bool force = st->force_step != 0;
    const bool pass = !force && ((stop != NSLI_STOP_NONE && h == 0) || (stop == NSLI_STOP_EPSMEM && mn < eps) ||
                                 (stop == NSLI_STOP_MAXVIOL_REL && mv <= eps * mb));
    const bool at_max = !pass && (st->it >= st->max_iter);
    const bool step = !pass && !at_max;
    const int rule = st->rule;
    const double lambda = st->lambda;
    const long long j = (long long)blockIdx.x * kShardThreads + threadIdx.x;

    double val = 0.0;
    if (step && j < p.n) {
        double y = 0.0;
        for (int w = 0; w < p.nranks; ++w)          // the global Reduce, worker order
            y += p.recs[(long long)w * len + kShardHeader + j];
        if (rule == NSLI_RULE_MODAP) {
            p.ybuf[j] = y;
            val = y * y;
        } else {
            const double s = h > 0 ? lambda / (double)h : 0.0;
            const double xo = p.x64[j];
            const double xn = xo - s * y;
            p.x64[j] = xn;
            static_cast<Acc *>(p.x)[j] = (Acc)xn;
            const double d = xn - xo;
            val = d * d;
        }
    }
    val = shard_warp_sum(val);
    if (lane == 0)
        sh.red[warp] = val;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kShardThreads / 32; ++w)
            t += sh.red[w];
        p.part_dx[blockIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int t = atomicAdd(&st->ticket, 1u);
        sh.last = (t == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!sh.last)
        return;
    __threadfence();

    double dx2 = 0.0, ynorm = 0.0;
    if (step) {
        if (warp == 0) {
            double v = 0.0;
            for (unsigned int q = lane; q < gridDim.x; q += 32)
                v += __ldcg(p.part_dx + q);
            v = shard_warp_sum(v);
            if (lane == 0)
                sh.red[0] = v;
        }
        __syncthreads();
        const double tot = sh.red[0];
        __syncthreads();
        if (rule == NSLI_RULE_MODAP) {
            ynorm = sqrt(tot);
            const double s = ynorm > 0.0 ? lambda / ynorm : 0.0;
            Acc *x = static_cast<Acc *>(p.x);
            double v = 0.0;
            for (long long q = threadIdx.x; q < p.n; q += kShardThreads) {
                const double xo = p.x64[q];
                const double xn = xo - s * __ldcg(p.ybuf + q);
                p.x64[q] = xn;
                x[q] = (Acc)xn;
                const double d = xn - xo;
                v += d * d;
            }
            v = shard_warp_sum(v);
            if (lane == 0)
                sh.red[warp] = v;
            __syncthreads();
            double t = 0.0;
            for (int w = 0; w < kShardThreads / 32; ++w)
                t += sh.red[w];
            dx2 = t;
        } else {
            dx2 = tot;
        }
    }
    if (threadIdx.x == 0) {
        st->h = h;
        st->maxviol = mv;
        st->maxnorm = mn;
        st->maxb = mb;
        if (pass) {
            st->status = ST_CANDIDATE;
            st->done = 1;
        } else if (at_max) {
            st->status = NSLI_NOT_CONVERGED;
            st->done = 1;
        } else {
            st->it += 1;
            if (!st->hold_tick)
                st->tick += 1;
            st->dx2 = dx2;
            st->y_norm = ynorm;
            if (stop == NSLI_STOP_STEP && step_norm_below(dx2, eps)) {
                st->status = NSLI_OK;
                st->done = 1;
            }
        }
        st->force_step = 0;
        st->ticket = 0u;
    }
}

}  // namespace

cudaError_t shard_pack_launch(cudaStream_t s, const DevState *st, const double *ybuf, long long n, double *rec)
{
    const unsigned int grid = (unsigned int)((n + kShardThreads - 1) / kShardThreads);
    shard_pack_kernel<<<grid, kShardThreads, 0, s>>>(st, ybuf, n, rec);
    return cudaGetLastError();
}

int shard_step_blocks(long long n) { return (int)((n + kShardThreads - 1) / kShardThreads); }

cudaError_t shard_step_launch(bool f64, cudaStream_t s, const ShardStepArgs &a)
{
    const unsigned int grid = (unsigned int)shard_step_blocks(a.n);
    if (f64)
        shard_step_kernel<double><<<grid, kShardThreads, 0, s>>>(a);
    else
        shard_step_kernel<float><<<grid, kShardThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace nsli
