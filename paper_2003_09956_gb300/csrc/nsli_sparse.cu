// nsli_sparse.cu -- the Map / Reduce / step for a sparse A.
//
// Same method as the dense kernels (Section 2 and 3: residuals, positive
// slices rho+_i of Eq. 7, their sum y, h of Eq. 8, the step of Eq. 8 or
// Eq. 12, the tick b(k) = b0 + k rho Av of Section 5), for A held twice:
// compressed rows (CSR) for the residuals and compressed columns (CSC) for
// y = sum_i c_i a_i, c_i = max(r_i, 0) / ||a_i||^2.  Reading A a second time
// by columns makes every y_j a sum in one fixed order (rows ascending) with
// no atomics, so results are bitwise reproducible, at twice the streamed
// bytes of a single pass.
//
// One iteration is three launches (the third only for the ModAP rule):
//   sparse_row_kernel   r_i, c_i, per-CTA (h, max r, max r/||a||, max |b|);
//                       the last CTA to finish (ticket) folds the CTA
//                       records and takes the stop decision.
//   sparse_col_kernel   y_j in CSC order; the relaxed step x_j -= lambda y_j / h
//                       in place, or y_j kept for ModAP; per-CTA sums of
//                       dx^2 (or y^2) folded by the last CTA.
//   sparse_step_kernel  ModAP only: x_j -= lambda y_j / ||y||.
// Rows (columns) up to a length threshold are "light": fixed ranges of them
// per CTA, W lanes per row, each lane issuing kU independent loads of
// indices and entries (evict-first: they are read once per iteration), then
// kU gathers of x (of the coefficients) from L2.  Longer ones are "heavy":
// cut into pieces of kPiece entries, one CTA per piece at the front of the
// grid; a piece stores its partial sum in a fixed slot and the last piece of
// a row to finish (per-row counter) adds the slots (the block's threads in a
// fixed tree), so the sums stay independent of timing.  Binary64 sums are
// trees or independent running sums throughout: a dependent binary64
// operation costs about 435 cycles on GB300.
//
// Small systems (x, y, the coefficients and a lambda / h table fit one CTA's
// shared memory, the matrix its L1) run instead on sparse_resident_kernel:
// one CTA, a whole block of iterations per launch (further below).
#include <cstdint>

#include "nsli.h"
#include "nsli_internal.h"

namespace nsli {
namespace {

constexpr int kThreads = 256;
constexpr int kU = kSparseU;
static_assert(kU > 0 && (kU & (kU - 1)) == 0, "loads per lane: a power of two");

template <typename T> struct SpTraits;
template <> struct SpTraits<double> {
    using Meta = RowMeta64;
};
template <> struct SpTraits<float> {
    using Meta = RowMeta32;
};

template <int W, typename T> __device__ __forceinline__ T group_sum(T v)
{
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

template <typename T> __device__ __forceinline__ T warp_total(T v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Block sum in a fixed tree: warp butterflies, then a pairwise tree over the
// 8 warp sums (GB300 takes about 435 cycles per dependent binary64 add, so
// every sum here is a tree rather than a chain).
template <typename T> __device__ __forceinline__ T block_sum(T v, T *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_total(v);
    __syncthreads();
    if (lane == 0)
        sh[warp] = v;
    __syncthreads();
    constexpr int NW = kThreads / 32;
    T t[NW];
#pragma unroll
    for (int q = 0; q < NW; ++q)
        t[q] = sh[q];
#pragma unroll
    for (int w = NW / 2; w > 0; w >>= 1)
#pragma unroll
        for (int q = 0; q < w; ++q)
            t[q] += t[q + w];
    return t[0];
}

// sum over e in [e0, e1) of val[e] * g[idx[e]] for lane l of a group of W
// lanes: chunks of W * kU entries, lane l taking e = c + l + u W, the kU
// loads of a chunk issued before any of its products; binary64 adds slot u
// of every chunk into running sum u and the kU sums in a fixed tree,
// binary32 adds everything into one running sum in lane-local order.
template <typename T, int W>
__device__ __forceinline__ T seg_dot(long long e0, long long e1, const int *idx, const T *val, const T *g, int l)
{
    T acc[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u)
        acc[u] = T(0);
    for (long long c = e0; c < e1; c += (long long)W * kU) {
        int id[kU];
        T v[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const long long e = c + l + (long long)u * W;
            const bool ok = e < e1;
            id[u] = ok ? __ldcs(idx + e) : 0;
            v[u] = ok ? __ldcs(val + e) : T(0);
        }
        T gv[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u)
            gv[u] = __ldg(g + id[u]);
        if constexpr (sizeof(T) == 8) {
#pragma unroll
            for (int u = 0; u < kU; ++u)
                acc[u] = fma(v[u], gv[u], acc[u]);
        } else {
#pragma unroll
            for (int u = 0; u < kU; ++u)
                acc[0] = fma(v[u], gv[u], acc[0]);
        }
    }
    // binary64: the kU running sums (one per load slot) in a fixed pairwise
    // tree; binary32 keeps one running sum (its latency is short)
#pragma unroll
    for (int w = kU / 2; w > 0; w >>= 1)
#pragma unroll
        for (int u = 0; u < w; ++u)
            acc[u] += acc[u + w];
    return acc[0];
}

// One piece of a heavy row / column: the block's sum over the piece, then
// (pieces > 1) the slot write and the per-segment counter.  Returns true in
// every thread when this block holds the finished segment sum in *total.
template <typename T>
__device__ __forceinline__ bool heavy_piece(const SegPiece &pc, const int *idx, const T *val, const T *g, T *slots,
                                            int *cnt, T *sh_sum, int *sh_flag, T *total)
{
    const T acc = seg_dot<T, kThreads>(pc.e0, pc.e1, idx, val, g, threadIdx.x);
    const T part = block_sum(acc, sh_sum);
    if (pc.npieces == 1) {
        *total = part;
        return true;
    }
    if (threadIdx.x == 0) {
        slots[pc.first + pc.k] = part;
        __threadfence();
        const int old = atomicAdd(cnt + pc.hs, 1);
        *sh_flag = (old == pc.npieces - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!*sh_flag)
        return false;
    __threadfence();
    // the segment's piece sums: thread t adds pieces t, t + kThreads, ...,
    // then the block tree (the same order whichever block finishes last)
    T t = T(0);
    for (int q = threadIdx.x; q < pc.npieces; q += kThreads)
        t += __ldcg(slots + pc.first + q);
    *total = block_sum(t, sh_sum);
    if (threadIdx.x == 0)
        cnt[pc.hs] = 0;   // ready for the next launch
    return true;
}

struct StatAcc {
    long long h;
    double mv, mn, mb;
};

// Order-preserving integer image of a binary64 value (and back): maxima
// folded on the integer pipe are exact and add no binary64 latency.
__device__ __forceinline__ unsigned long long stat_enc(double d)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double stat_dec(unsigned long long u)
{
    const unsigned long long bits = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
    return __longlong_as_double((long long)bits);
}

// Fold per-thread stats into one record (exact: integer sum and maxima).
__device__ StatAcc block_stats(StatAcc s, StatAcc *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long mv = stat_enc(s.mv), mn = stat_enc(s.mn), mb = stat_enc(s.mb);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        s.h += __shfl_xor_sync(0xffffffffu, s.h, off);
        mv = max(mv, __shfl_xor_sync(0xffffffffu, mv, off));
        mn = max(mn, __shfl_xor_sync(0xffffffffu, mn, off));
        mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, off));
    }
    __syncthreads();
    if (lane == 0)
        sh[warp] = StatAcc{s.h, stat_dec(mv), stat_dec(mn), stat_dec(mb)};
    __syncthreads();
    long long h = 0;
    mv = stat_enc(-INFINITY);
    mn = mv;
    mb = stat_enc(0.0);
#pragma unroll
    for (int q = 0; q < kThreads / 32; ++q) {
        h += sh[q].h;
        mv = max(mv, stat_enc(sh[q].mv));
        mn = max(mn, stat_enc(sh[q].mn));
        mb = max(mb, stat_enc(sh[q].mb));
    }
    return StatAcc{h, stat_dec(mv), stat_dec(mn), stat_dec(mb)};
}

// Per-thread stats in the accumulation type: maxima of binary32 values are
// exact in binary32, and widened once per thread (StatLoc::wide) rather
// than per row (a binary64 instruction occupies GB300's FP64 pipe for a
// whole warp, however few of its lanes are active).
template <typename T> struct StatLoc {
    long long h = 0;
    T mv = -INFINITY, mn = -INFINITY, mb = T(0);
    __device__ StatAcc wide() const { return StatAcc{h, (double)mv, (double)mn, (double)mb}; }
};

// r_i from a finished dot; writes c_i and folds the row into the stats.
template <typename T>
__device__ __forceinline__ void finish_row(const SparseArgs &p, long long i, T dot, T tk,
                                           const typename SpTraits<T>::Meta &md, StatLoc<T> &s)
{
    const T bi = fma(tk, (T)md.av, (T)md.b0);
    const T ri = dot - bi;
    const bool viol = ri > T(0);
    static_cast<T *>(p.coef)[i] = viol ? ri * (T)md.inv_n2 : T(0);
    s.h += viol ? 1 : 0;
    const T rn = ri * (T)md.inv_n;
    s.mv = ri > s.mv ? ri : s.mv;
    s.mn = rn > s.mn ? rn : s.mn;
    const T ab = bi < T(0) ? -bi : bi;
    s.mb = ab > s.mb ? ab : s.mb;
}

// Stop decision of the iteration whose Map just finished (same rules and
// order as the dense reduce kernel): candidate stop, iteration cap, or step.
__device__ void decide(DevState *st, const StatAcc &t, int mode)
{
    st->h = t.h;
    st->maxviol = t.mv;
    st->maxnorm = t.mn;
    st->maxb = t.mb;
    if (mode != 0)
        return;
    const int stop = st->stop;
    const double eps = st->eps;
    const bool force = st->force_step != 0;
    const bool pass = !force && ((stop != NSLI_STOP_NONE && t.h == 0) || (stop == NSLI_STOP_EPSMEM && t.mn < eps) ||
                                 (stop == NSLI_STOP_MAXVIOL_REL && t.mv <= eps * t.mb));
    const bool at_max = !pass && (st->it >= st->max_iter);
    if (pass) {
        st->status = ST_CANDIDATE;
        st->done = 1;
    } else if (at_max) {
        st->status = NSLI_NOT_CONVERGED;
        st->done = 1;
    }
    st->force_step = 0;
}

// Bookkeeping after a step (the dense reduce kernel's, in the same order).
__device__ void finish_step(DevState *st, double dx2, double ynorm)
{
    st->it += 1;
    if (!st->hold_tick)
        st->tick += 1;
    st->dx2 = dx2;
    st->y_norm = ynorm;
    if (st->stop == NSLI_STOP_STEP && step_norm_below(dx2, st->eps)) {
        st->status = NSLI_OK;
        st->done = 1;
    }
}

// Ticket: true in exactly one thread block, the last to arrive.
__device__ __forceinline__ bool last_block(DevState *st, int nblk, int *sh_last)
{
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int t = atomicAdd(&st->ticket, 1u);
        *sh_last = (t == (unsigned int)nblk - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!*sh_last)
        return false;
    __threadfence();
    return true;
}

// At most 48 registers (five 256-thread CTAs per SM): the row pass is bound
// by its gathers, so the loads in flight per SM set its speed.
template <typename T, int W> __global__ void __launch_bounds__(kThreads, 5) sparse_row_kernel(const SparseArgs p)
{
    using Meta = typename SpTraits<T>::Meta;
    DevState *st = p.st;
    if (!p.ignore_done && *(volatile int *)&st->done)
        return;
    __shared__ StatAcc sh_stat[kThreads / 32];
    __shared__ T sh_sum[kThreads / 32];
    __shared__ int sh_last, sh_flag;
    const T *va = static_cast<const T *>(p.va);
    const T *x = static_cast<const T *>(p.x);
    const T tk = (T)((double)st->tick * st->rho);
    StatLoc<T> s;
    const int nblk = p.n_row_pieces + p.row_light_ctas;

    if ((int)blockIdx.x < p.n_row_pieces) {
        const SegPiece pc = p.row_pieces[blockIdx.x];
        T dot;
        if (heavy_piece(pc, p.ci, va, x, static_cast<T *>(p.row_slots), p.row_cnt, sh_sum, &sh_flag, &dot) &&
            threadIdx.x == 0)
            finish_row(p, pc.seg, dot, tk, static_cast<const Meta *>(p.meta)[pc.seg], s);
    } else {
        const long long b = blockIdx.x - p.n_row_pieces;
        const long long r0 = b * p.light_rows_per_cta;
        const long long r1 = min(r0 + p.light_rows_per_cta, p.m);
        constexpr int groups = kThreads / W;
        const int g = threadIdx.x / W, l = threadIdx.x % W;
        // every group makes the same number of passes, so the shuffles
        // below always see all 32 lanes of a warp
        for (long long base = r0; base < r1; base += groups) {
            const long long i = base + g;
            T acc = T(0);
            bool valid = i < r1;
            long long e0 = 0, e1 = 0;
            Meta md{};
            if (valid) {
                e0 = p.rp[i];
                e1 = p.rp[i + 1];
                if (l == 0)
                    md = static_cast<const Meta *>(p.meta)[i];   // in flight with the entries
                valid = (e1 - e0) <= p.heavy_thr_row;
            }
            if (valid)
                acc = seg_dot<T, W>(e0, e1, p.ci, va, x, l);
            const T dot = group_sum<W>(acc);
            if (valid && l == 0)
                finish_row(p, i, dot, tk, md, s);
        }
    }
    const StatAcc t = block_stats(s.wide(), sh_stat);
    if (threadIdx.x == 0) {
        PartStat ps;
        ps.h = t.h;
        ps.maxviol = t.mv;
        ps.maxnorm = t.mn;
        ps.maxb = t.mb;
        p.part_stat[blockIdx.x] = ps;
    }
    if (!last_block(st, nblk, &sh_last))
        return;
    long long uh = 0;
    unsigned long long umv = stat_enc(-INFINITY), umn = umv, umb = stat_enc(0.0);
    for (int q = threadIdx.x; q < nblk; q += kThreads) {
        const PartStat *ps = p.part_stat + q;
        uh += __ldcg(&ps->h);
        umv = max(umv, stat_enc(__ldcg(&ps->maxviol)));
        umn = max(umn, stat_enc(__ldcg(&ps->maxnorm)));
        umb = max(umb, stat_enc(__ldcg(&ps->maxb)));
    }
    const StatAcc tot = block_stats(StatAcc{uh, stat_dec(umv), stat_dec(umn), stat_dec(umb)}, sh_stat);
    if (threadIdx.x == 0) {
        decide(st, tot, p.mode);
        st->ticket = 0u;
    }
}

// y_j = sum over the column's entries (rows ascending) of c_i a_ij.
template <typename T>
__device__ __forceinline__ double col_update(const SparseArgs &p, long long j, T y, double s_relaxed, int rule,
                                             double xo)
{
    if (p.mode != 0) {
        p.ybuf[j] = (double)y;
        return 0.0;
    }
    if (rule == NSLI_RULE_MODAP) {
        const double yd = (double)y;
        p.ybuf[j] = yd;
        return yd * yd;
    }
    const double xn = xo - s_relaxed * (double)y;
    p.x64[j] = xn;
    static_cast<T *>(p.x)[j] = (T)xn;
    const double d = xn - xo;
    return d * d;
}

template <typename T, int W> __global__ void __launch_bounds__(kThreads) sparse_col_kernel(const SparseArgs p)
{
    DevState *st = p.st;
    if (!p.ignore_done && *(volatile int *)&st->done)
        return;
    __shared__ T sh_sum[kThreads / 32];
    __shared__ double sh_d[kThreads / 32];
    __shared__ int sh_last, sh_flag;
    const T *vc = static_cast<const T *>(p.vc);
    const T *coef = static_cast<const T *>(p.coef);
    const long long h = st->h;
    const int rule = st->rule;
    const double s_relaxed = h > 0 ? (p.rtab ? __ldg(p.rtab + h) : st->lambda / (double)h) : 0.0;
    const int nblk = p.n_col_pieces + p.col_light_ctas;
    double part = 0.0;

    if ((int)blockIdx.x < p.n_col_pieces) {
        const SegPiece pc = p.col_pieces[blockIdx.x];
        T y;
        if (heavy_piece(pc, p.ri, vc, coef, static_cast<T *>(p.col_slots), p.col_cnt, sh_sum, &sh_flag, &y) &&
            threadIdx.x == 0)
            part = col_update(p, pc.seg, y, s_relaxed, rule, p.x64[pc.seg]);
    } else {
        const long long b = blockIdx.x - p.n_col_pieces;
        const long long c0 = b * p.light_cols_per_cta;
        const long long c1 = min(c0 + p.light_cols_per_cta, p.n);
        constexpr int groups = kThreads / W;
        constexpr int GW = 32 / W;   // columns a warp finishes per pass
        const int g = threadIdx.x / W, l = threadIdx.x % W;
        const int lane = threadIdx.x & 31;
        const long long wfirst = (long long)(threadIdx.x >> 5) * GW;
        // The binary64 step of a column (col_update) is taken for 32 columns
        // at once, one per lane: after pass t of every W passes, lane
        // t * GW + q holds the y and index of the column of the warp's group
        // q (a binary64 instruction occupies the FP64 pipe for a whole warp,
        // so one lane per column would cost 32 times as much).
        T ybuf = T(0);
        long long jbuf = -1;
        int t = 0;
        for (long long base = c0; base < c1; base += groups) {
            const long long j = base + g;
            T acc = T(0);
            bool valid = j < c1;
            long long e0 = 0, e1 = 0;
            if (valid) {
                e0 = p.cp[j];
                e1 = p.cp[j + 1];
                valid = (e1 - e0) <= p.heavy_thr_col;
            }
            if (valid)
                acc = seg_dot<T, W>(e0, e1, p.ri, vc, coef, l);
            const T y = group_sum<W>(acc);
            const int src = (lane % GW) * W;
            const T yq = __shfl_sync(0xffffffffu, y, src);
            const int vq = __shfl_sync(0xffffffffu, valid ? 1 : 0, src);
            if (lane / GW == t) {
                ybuf = yq;
                jbuf = vq ? base + wfirst + lane % GW : -1;
            }
            if (++t == W) {
                if (jbuf >= 0)
                    part += col_update(p, jbuf, ybuf, s_relaxed, rule,
                                       (p.mode == 0 && rule != NSLI_RULE_MODAP) ? p.x64[jbuf] : 0.0);
                t = 0;
                jbuf = -1;
            }
        }
        if (t > 0 && jbuf >= 0)
            part += col_update(p, jbuf, ybuf, s_relaxed, rule,
                               (p.mode == 0 && rule != NSLI_RULE_MODAP) ? p.x64[jbuf] : 0.0);
    }
    const double bsum = block_sum(part, sh_d);
    if (threadIdx.x == 0)
        p.part_dx[blockIdx.x] = bsum;
    if (!last_block(st, nblk, &sh_last))
        return;
    double v = 0.0;
    for (int q = threadIdx.x; q < nblk; q += kThreads)
        v += __ldcg(p.part_dx + q);
    const double tot = block_sum(v, sh_d);
    if (threadIdx.x == 0) {
        if (p.mode == 0) {
            if (rule == NSLI_RULE_MODAP)
                st->y_norm = sqrt(tot);
            else
                finish_step(st, tot, 0.0);
        }
        st->ticket = 0u;
    }
}

template <typename T> __global__ void __launch_bounds__(kThreads) sparse_step_kernel(const SparseArgs p)
{
    DevState *st = p.st;
    if (*(volatile int *)&st->done || st->rule != NSLI_RULE_MODAP)
        return;
    __shared__ double sh_d[kThreads / 32];
    __shared__ int sh_last;
    const double ynorm = st->y_norm;
    const double s = ynorm > 0.0 ? st->lambda / ynorm : 0.0;
    T *x = static_cast<T *>(p.x);
    double v = 0.0;
    for (long long j = (long long)blockIdx.x * kThreads + threadIdx.x; j < p.n; j += (long long)gridDim.x * kThreads) {
        const double xo = p.x64[j];
        const double xn = xo - s * __ldcg(p.ybuf + j);
        p.x64[j] = xn;
        x[j] = (T)xn;
        const double d = xn - xo;
        v += d * d;
    }
    const double bsum = block_sum(v, sh_d);
    if (threadIdx.x == 0)
        p.part_dx[blockIdx.x] = bsum;
    if (!last_block(st, gridDim.x, &sh_last))
        return;
    double w = 0.0;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += kThreads)
        w += __ldcg(p.part_dx + q);
    const double tot = block_sum(w, sh_d);
    if (threadIdx.x == 0) {
        finish_step(st, tot, ynorm);
        st->ticket = 0u;
    }
}

// ---- set-up and the binary64 check -----------------------------------------

__device__ __forceinline__ unsigned long long sp_ord_enc(double d)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// One warp per row: binary64 ||a_i||^2 of the stored values (fixed tree),
// zero-row and finiteness flags.
template <typename T> __global__ void __launch_bounds__(kThreads) sparse_norms_kernel(const SparseArgs p, double *n2,
                                                                                   int *flags)
{
    const int lane = threadIdx.x & 31;
    const long long w = ((long long)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * kThreads) >> 5;
    const T *va = static_cast<const T *>(p.va);
    for (long long i = w; i < p.m; i += nw) {
        double s = 0.0;
        int bad = 0;
        for (long long e = p.rp[i] + lane; e < p.rp[i + 1]; e += 32) {
            const double a = (double)va[e];
            if (!isfinite(a))
                bad = 1;
            s = fma(a, a, s);
        }
        s = warp_total(s);
        bad = __any_sync(0xffffffffu, bad);
        if (lane == 0) {
            n2[i] = s;
            if (bad)
                atomicOr(flags, PREPF_NONFINITE);
            else if (s == 0.0)
                atomicOr(flags, PREPF_ZERO_ROW);
        }
    }
}

// One warp per row: r_i in binary64 from the stored values and x64; maxima
// by order-preserving integer atomics (exact, schedule-independent).
template <typename T> __global__ void __launch_bounds__(kThreads) sparse_verify_kernel(const SparseArgs p,
                                                                                    const VerifyArgs v)
{
    const int lane = threadIdx.x & 31;
    const long long w = ((long long)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * kThreads) >> 5;
    const T *va = static_cast<const T *>(p.va);
    const double kr = __dmul_rn((double)v.st->tick, v.st->rho);
    double mv = -INFINITY, mn = -INFINITY, mb = 0.0;
    unsigned long long h = 0;
    for (long long i = w; i < p.m; i += nw) {
        double s = 0.0;
        for (long long e = p.rp[i] + lane; e < p.rp[i + 1]; e += 32)
            s = fma((double)va[e], v.x64[p.ci[e]], s);
        s = warp_total(s);
        const double bi = __dadd_rn(v.b0_64[i], __dmul_rn(kr, v.av_64[i]));
        const double ri = s - bi;
        mv = fmax(mv, ri);
        mn = fmax(mn, ri / sqrt(v.n2_64[i]));
        mb = fmax(mb, fabs(bi));
        h += (ri > 0.0) ? 1ull : 0ull;
    }
    if (lane == 0) {
        atomicMax(&v.out->maxviol, sp_ord_enc(mv));
        atomicMax(&v.out->maxnorm, sp_ord_enc(mn));
        atomicMax(&v.out->maxb, sp_ord_enc(mb));
        atomicAdd(&v.out->h, h);
    }
}

// Dense copies of stored rows row0 .. row0+rows-1 (out zeroed by the caller).
template <typename T> __global__ void sparse_rows_kernel(const SparseArgs p, long long row0, long long rows,
                                                         double *out)
{
    const long long r = blockIdx.x;
    if (r >= rows)
        return;
    const long long i = row0 + r;
    const T *va = static_cast<const T *>(p.va);
    for (long long e = p.rp[i] + threadIdx.x; e < p.rp[i + 1]; e += blockDim.x)
        out[r * p.n + p.ci[e]] = (double)va[e];
}

// ---- small systems: a whole block of iterations in one CTA --------------------
//
// When the binary64 iterate, y, x and the coefficients c in the
// accumulation type, and a table of lambda / h fit in one CTA's shared
// memory, one CTA on one SM runs up to `iters` iterations per launch: an
// iteration costs a few block barriers instead of two or three launches and
// their grid-wide hand-offs.  The steps and decisions are those of the grid
// kernels above, in an order of their own: short rows one per thread in CSR
// order, two rows at a time (rows longer than kResLong on warps of their
// own: lane-strided running sums, a tree, a butterfly); the row counts and
// maxima folded exactly (integers and order-preserving encodings); the stop
// decision by thread 0 while the other threads gather y_j in CSC order over
// the violated rows (long columns by warps); the relaxed step, or ||y|| and
// ModAP's step; the terms of ||dx|| after the step's barrier, folded in a
// fixed order.  Only x, x64 and DevState persist between launches (global
// memory), so launches of any size give identical results.  The statistics
// a stop rule does not read are not formed: DevState keeps h and max r_i
// always, max r_i / ||a_i|| only under EPSMEM and max |b_i| only under
// MAXVIOL_REL (-inf / 0 otherwise).

__device__ __forceinline__ double sp_ord_dec(unsigned long long u)
{
    const unsigned long long bits = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b)
{
    return a > b ? a : b;
}

// Running maximum for the row statistics.  Binary64: kept as the
// order-preserving integer encoding, so no comparison goes to GB300's narrow
// binary64 pipe; binary32: a plain fmaxf, encoded once at the end.
template <typename T> struct ResMax;
template <> struct ResMax<double> {
    unsigned long long u;
    __device__ __forceinline__ explicit ResMax(double init) : u(sp_ord_enc(init)) {}
    __device__ __forceinline__ void add(double v) { u = umax64(u, sp_ord_enc(v)); }
    __device__ __forceinline__ unsigned long long enc() const { return u; }
};
template <> struct ResMax<float> {
    float f;
    __device__ __forceinline__ explicit ResMax(double init) : f((float)init) {}
    __device__ __forceinline__ void add(float v) { f = fmaxf(f, v); }
    __device__ __forceinline__ unsigned long long enc() const { return sp_ord_enc((double)f); }
};

// r_i > 0 from the bit pattern (integer pipe); the same as the comparison
// for every value but NaN, which the inputs exclude
__device__ __forceinline__ bool positive(double v) { return __double_as_longlong(v) > 0; }
__device__ __forceinline__ bool positive(float v) { return __float_as_int(v) > 0; }

// Fixed-order sum of the block's per-thread values (called by warp 0):
// a pairwise tree over each lane's kResThreads / 32 values, then a butterfly.
__device__ __forceinline__ double res_fold(const double *part, int lane)
{
    constexpr int NW = kResThreads / 32;
    double t[NW];
#pragma unroll
    for (int q = 0; q < NW; ++q)
        t[q] = part[lane + 32 * q];
#pragma unroll
    for (int w = NW / 2; w > 0; w >>= 1)
#pragma unroll
        for (int q = 0; q < w; ++q)
            t[q] += t[q + w];
    return warp_total(t[0]);
}

// |v| as an integer that orders like |v| (the bits of a non-negative binary64)
__device__ __forceinline__ long long abs_bits(double v) { return __double_as_longlong(v) & 0x7fffffffffffffffll; }

// GB300 executes a dependent binary64 operation in about 435 cycles (a
// measured chain of FMAs on one SM, against about 12 for binary32), so an
// iteration's time is set by the depth of its binary64 dependency chain, and
// the kernel is arranged to keep that chain short: rows longer than
// kResLong go to warps of their own (lanes hold four partial sums added in a
// tree) while the other warps take the short rows two at a time; the tick
// term of the next Map is formed during this one; the scalar decision uses a
// table of lambda / h instead of a division; and the terms of ||dx||, which
// no later step of the iteration needs, are formed after the barrier that
// ends the step, their sum only when the step rule can hold (and for the
// last step of a launch).

// acc + a * v where acc is still the exact zero it started as: for a = +1 or
// -1 (bound rows and columns) the product is v or -v exactly and no binary64
// operation is needed; the coefficient is recognised from its bit pattern.
__device__ __forceinline__ double first_term(double a, double v)
{
    const long long b = __double_as_longlong(a);
    if (b == 0x3ff0000000000000ll)
        return v;
    if (b == (long long)0xbff0000000000000ull)
        return -v;
    return a * v;
}
__device__ __forceinline__ float first_term(float a, float v)
{
    const int b = __float_as_int(a);
    if (b == 0x3f800000)
        return v;
    if (b == (int)0xbf800000u)
        return -v;
    return a * v;
}

template <typename T>
__global__ void __launch_bounds__(kResThreads, 1) sparse_resident_kernel(const SparseArgs p, int iters)
{
    using Meta = typename SpTraits<T>::Meta;
    DevState *st = p.st;
    if (*(volatile int *)&st->done || iters <= 0)
        return;
    extern __shared__ __align__(16) unsigned char res_smem[];
    const long long n = p.n, m = p.m;
    double *x64s = reinterpret_cast<double *>(res_smem);
    double *ys = x64s + n;                  // y_j; after the step, x_j before it
    double *rtab = ys + n;                  // lambda / h for h = 0..m (0 for h = 0)
    T *xs = reinterpret_cast<T *>(rtab + m + 1);
    T *cs = xs + n;
    constexpr int NW = kResThreads / 32;
    __shared__ int sh_wh[NW];
    __shared__ unsigned long long sh_wmv[NW], sh_wmn[NW], sh_wmb[NW];
    __shared__ double sh_part[2][kResThreads];   // dx^2 (y^2) partials, by iteration parity
    __shared__ long long sh_dmax[2][NW];         // max |dx_j| per warp (bits), by parity
    // broadcast by thread 0: the run has ended, the step scale, the tick
    // term of each Map (by iteration parity)
    __shared__ int sh_done;
    __shared__ double sh_scale;
    __shared__ T sh_tk[2];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const T *va = static_cast<const T *>(p.va);
    const T *vc = static_cast<const T *>(p.vc);
    const Meta *meta = static_cast<const Meta *>(p.meta);
    T *xg = static_cast<T *>(p.x);

    // the run's control values; its progress is kept by thread 0
    const double lambda = st->lambda, eps = st->eps, rho = st->rho;
    const long long max_iter = st->max_iter;
    const int rule = st->rule, stop = st->stop, hold = st->hold_tick;
    const bool modap = rule == NSLI_RULE_MODAP;
    const bool want_mn = stop == NSLI_STOP_EPSMEM, want_mb = stop == NSLI_STOP_MAXVIOL_REL;
    for (long long j = tid; j < n; j += kResThreads) {
        x64s[j] = p.x64[j];
        xs[j] = xg[j];
    }
    for (long long h = tid; h <= m; h += kResThreads)
        rtab[h] = h > 0 ? lambda / (double)h : 0.0;   // the grid kernels' lambda / h
    // warps of their own for the long rows (columns), the last ones
    const int lw_r = min(NW / 2, p.n_res_long_rows), lw_c = min(NW / 2, p.n_res_long_cols);
    const int nt_r = (NW - lw_r) * 32, nt_c = (NW - lw_c) * 32;
    // ||dx|| < eps is possible only if no |dx_j| exceeds eps (1e-6 of margin
    // covers the rounding of the sum and the root)
    const double gate = eps * (1.0 + 1e-6);
    int force = 0, status = 0, done = 0;
    long long it = 0, tick = 0, h_last = 0;
    double mv_last = 0, mn_last = 0, mb_last = 0, yn = 0;
    int last_par = -1;   // parity of the last step's dx^2 partials (thread 0)
    double dx2_0 = 0;
    if (tid == 0) {
        force = st->force_step;
        status = st->status;
        it = st->it;
        tick = st->tick;
        h_last = st->h;
        mv_last = st->maxviol;
        mn_last = st->maxnorm;
        mb_last = st->maxb;
        dx2_0 = st->dx2;
        yn = st->y_norm;
        sh_tk[0] = (T)((double)tick * rho);
        sh_done = 0;
    }
    __syncthreads();

    // warp 0: does the step rule hold after the step whose terms carry parity q?
    auto step_rule = [&](int q) -> bool {
        long long dm = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w)
            dm = max(dm, sh_dmax[q][w]);
        if (stop != NSLI_STOP_STEP || __longlong_as_double(dm) > gate)
            return false;
        return step_norm_below(res_fold(sh_part[q], lane), eps);
    };

    for (int k = 0; k < iters; ++k) {
        const int par = k & 1;
        // ---- rows: r_i, c_i and the statistics of this thread's rows
        const T tk = sh_tk[par];
        const bool tk0 = tk == T(0);   // b_i = fma(0, Av_i, b0_i) = b0_i
        if (tid == 0)                  // the next Map's tick term
            sh_tk[par ^ 1] = (T)((double)(hold ? tick : tick + 1) * rho);
        int hc = 0;
        ResMax<T> mv(-INFINITY), mn(-INFINITY), mb(0.0);
        auto row_done = [&](long long i, T dot) {
            const Meta md = meta[i];
            const T bi = tk0 ? (T)md.b0 : fma(tk, (T)md.av, (T)md.b0);
            const T ri = dot - bi;
            const bool viol = positive(ri);
            T c = T(0);
            if (viol)
                c = ri * (T)md.inv_n2;
            cs[i] = c;
            hc += viol ? 1 : 0;
            mv.add(ri);
            if (want_mn)
                mn.add(ri * (T)md.inv_n);
            if (want_mb)
                mb.add(bi < T(0) ? -bi : bi);
        };
        if (tid < nt_r) {
            // short rows, two at a time (independent chains)
            for (long long i0 = tid; i0 < m; i0 += 2 * (long long)nt_r) {
                const long long i1 = i0 + nt_r;
                const long long a0 = __ldg(p.rp + i0), b0 = __ldg(p.rp + i0 + 1);
                long long a1 = 0, b1 = 0;
                if (i1 < m) {
                    a1 = __ldg(p.rp + i1);
                    b1 = __ldg(p.rp + i1 + 1);
                }
                const bool ok0 = b0 - a0 <= kResLong, ok1 = i1 < m && b1 - a1 <= kResLong;
                const long long l0 = ok0 ? b0 - a0 : 0, l1 = ok1 ? b1 - a1 : 0;
                T s0 = T(0), s1 = T(0);
                if (l0 > 0)
                    s0 = first_term(__ldg(va + a0), xs[__ldg(p.ci + a0)]);
                if (l1 > 0)
                    s1 = first_term(__ldg(va + a1), xs[__ldg(p.ci + a1)]);
                for (long long q = 1; q < max(l0, l1); ++q) {
                    if (q < l0)
                        s0 = fma(__ldg(va + a0 + q), xs[__ldg(p.ci + a0 + q)], s0);
                    if (q < l1)
                        s1 = fma(__ldg(va + a1 + q), xs[__ldg(p.ci + a1 + q)], s1);
                }
                if (ok0)
                    row_done(i0, s0);
                if (ok1)
                    row_done(i1, s1);
            }
        } else {
            // long rows: four partial sums per lane, a tree, a butterfly
            for (int q = warp - (NW - lw_r); q < p.n_res_long_rows; q += lw_r) {
                const long long i = __ldg(p.res_long_rows + q);
                const long long e0 = __ldg(p.rp + i), e1 = __ldg(p.rp + i + 1);
                T a4[4] = {T(0), T(0), T(0), T(0)};
                for (long long c = e0 + lane; c < e1; c += 128) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const long long e = c + 32 * u;
                        if (e < e1)
                            a4[u] = fma(__ldg(va + e), xs[__ldg(p.ci + e)], a4[u]);
                    }
                }
                T acc = (a4[0] + a4[1]) + (a4[2] + a4[3]);
                acc = warp_total(acc);
                if (lane == 0)
                    row_done(i, acc);
            }
        }
        // exact folds: integer sum, maxima as order-preserving integers
        unsigned long long umv = mv.enc(), umn = mn.enc(), umb = mb.enc();
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            hc += __shfl_xor_sync(0xffffffffu, hc, off);
            umv = umax64(umv, __shfl_xor_sync(0xffffffffu, umv, off));
            if (want_mn)
                umn = umax64(umn, __shfl_xor_sync(0xffffffffu, umn, off));
            if (want_mb)
                umb = umax64(umb, __shfl_xor_sync(0xffffffffu, umb, off));
        }
        if (lane == 0) {
            sh_wh[warp] = hc;
            sh_wmv[warp] = umv;
            sh_wmn[warp] = umn;
            sh_wmb[warp] = umb;
        }
        __syncthreads();
        // ---- warp 0: the step rule of the previous step, then the stop
        // decision (the grid kernels' rules), while the others gather y
        if (warp == 0) {
            const int lp = __shfl_sync(0xffffffffu, last_par, 0);
            const bool step_stop = lp >= 0 && k > 0 && step_rule(lp);
            if (lane == 0) {
                if (step_stop) {
                    status = NSLI_OK;
                    done = 1;
                } else {
                    long long H = 0;
                    unsigned long long a = sh_wmv[0], b = sh_wmn[0], c = sh_wmb[0];
                    for (int q = 0; q < NW; ++q) {
                        H += sh_wh[q];
                        a = umax64(a, sh_wmv[q]);
                        b = umax64(b, sh_wmn[q]);
                        c = umax64(c, sh_wmb[q]);
                    }
                    h_last = H;
                    mv_last = sp_ord_dec(a);
                    mn_last = sp_ord_dec(b);
                    mb_last = sp_ord_dec(c);
                    const bool pass = !force && ((stop != NSLI_STOP_NONE && H == 0) ||
                                                 (stop == NSLI_STOP_EPSMEM && mn_last < eps) ||
                                                 (stop == NSLI_STOP_MAXVIOL_REL && mv_last <= eps * mb_last));
                    const bool at_max = !pass && it >= max_iter;
                    force = 0;
                    if (pass) {
                        status = ST_CANDIDATE;
                        done = 1;
                    } else if (at_max) {
                        status = NSLI_NOT_CONVERGED;
                        done = 1;
                    }
                    sh_scale = rtab[H];
                }
                sh_done = done;
            }
        }
        // y_j in CSC order over the violated rows (c_i = 0 adds nothing)
        if (tid < nt_c) {
            for (long long j = tid; j < n; j += nt_c) {
                const long long e0 = __ldg(p.cp + j), e1 = __ldg(p.cp + j + 1);
                if (e1 - e0 > kResLong)
                    continue;
                T y = T(0);
                bool first = true;
                for (long long e = e0; e < e1; ++e) {
                    const T c = cs[__ldg(p.ri + e)];
                    if (c != T(0)) {
                        y = first ? first_term(__ldg(vc + e), c) : fma(__ldg(vc + e), c, y);
                        first = false;
                    }
                }
                ys[j] = (double)y;
            }
        } else {
            for (int q = warp - (NW - lw_c); q < p.n_res_long_cols; q += lw_c) {
                const long long j = __ldg(p.res_long_cols + q);
                const long long e0 = __ldg(p.cp + j), e1 = __ldg(p.cp + j + 1);
                T y4[4] = {T(0), T(0), T(0), T(0)};
                for (long long c = e0 + lane; c < e1; c += 128) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const long long e = c + 32 * u;
                        if (e < e1) {
                            const T cf = cs[__ldg(p.ri + e)];
                            if (cf != T(0))
                                y4[u] = fma(__ldg(vc + e), cf, y4[u]);
                        }
                    }
                }
                T y = (y4[0] + y4[1]) + (y4[2] + y4[3]);
                y = warp_total(y);
                if (lane == 0)
                    ys[j] = (double)y;
            }
        }
        __syncthreads();
        if (sh_done)
            break;

        // ---- the step: x_j -= lambda y_j / h (relaxed) or lambda y_j / ||y||
        if (tid == 0) {
            it += 1;
            if (!hold)
                tick += 1;
            last_par = par;
        }
        if (modap) {
            double part = 0.0;
            for (long long j = tid; j < n; j += kResThreads)
                part += ys[j] * ys[j];
            sh_part[par][tid] = part;
            __syncthreads();
            if (warp == 0) {
                const double y2 = res_fold(sh_part[par], lane);
                if (lane == 0) {
                    yn = sqrt(y2);
                    sh_scale = yn > 0.0 ? lambda / yn : 0.0;
                }
            }
            __syncthreads();
        } else if (tid == 0) {
            yn = 0.0;
        }
        const double sc = sh_scale;
        for (long long j = tid; j < n; j += kResThreads) {
            const double yj = ys[j];
            const double xo = x64s[j];
            ys[j] = xo;
            if (yj != 0.0) {   // x_j - sc * 0 = x_j
                const double xn = xo - sc * yj;
                x64s[j] = xn;
                xs[j] = (T)xn;
            }
        }
        __syncthreads();
        // the terms of ||dx|| (this thread's columns), for the step rule
        // decided after the next Map's barrier
        {
            double part = 0.0;
            long long dmax = 0;
            for (long long j = tid; j < n; j += kResThreads) {
                const double d = x64s[j] - ys[j];
                part += d * d;
                dmax = max(dmax, abs_bits(d));
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
                dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, off));
            sh_part[par][tid] = part;
            if (lane == 0)
                sh_dmax[par][warp] = dmax;
        }
    }
    __syncthreads();
    for (long long j = tid; j < n; j += kResThreads) {
        p.x64[j] = x64s[j];
        xg[j] = xs[j];
    }
    // the last step: its step rule (if the loop ended right after it) and ||dx||^2
    double dx2 = dx2_0;
    if (warp == 0) {
        const int lp = __shfl_sync(0xffffffffu, last_par, 0);
        const int dn = __shfl_sync(0xffffffffu, done, 0);
        if (lp >= 0) {
            if (!dn && step_rule(lp) && lane == 0) {
                status = NSLI_OK;
                done = 1;
            }
            dx2 = res_fold(sh_part[lp], lane);
        }
    }
    if (tid == 0) {
        st->it = it;
        st->tick = tick;
        st->force_step = force;
        st->h = h_last;
        st->maxviol = mv_last;
        st->maxnorm = mn_last;
        st->maxb = mb_last;
        st->dx2 = dx2;
        st->y_norm = yn;
        st->status = status;
        st->done = done;
    }
}

template <typename T> int blocks_per_sm_row(int w)
{
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (w) {
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sparse_row_kernel<T, 1>, kThreads, 0); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sparse_row_kernel<T, 2>, kThreads, 0); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sparse_row_kernel<T, 4>, kThreads, 0); break;
    case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sparse_row_kernel<T, 8>, kThreads, 0); break;
    case 16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sparse_row_kernel<T, 16>, kThreads, 0); break;
    case 32: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sparse_row_kernel<T, 32>, kThreads, 0); break;
    default: break;
    }
    return e == cudaSuccess ? nb : 0;
}

template <typename T> int blocks_per_sm_col(int w)
{
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (w) {
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sparse_col_kernel<T, 1>, kThreads, 0); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sparse_col_kernel<T, 2>, kThreads, 0); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sparse_col_kernel<T, 4>, kThreads, 0); break;
    case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sparse_col_kernel<T, 8>, kThreads, 0); break;
    case 16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sparse_col_kernel<T, 16>, kThreads, 0); break;
    case 32: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sparse_col_kernel<T, 32>, kThreads, 0); break;
    default: break;
    }
    return e == cudaSuccess ? nb : 0;
}

template <typename T> cudaError_t row_launch(int w, unsigned grid, cudaStream_t s, const SparseArgs &a)
{
    switch (w) {
    case 1: sparse_row_kernel<T, 1><<<grid, kThreads, 0, s>>>(a); break;
    case 2: sparse_row_kernel<T, 2><<<grid, kThreads, 0, s>>>(a); break;
    case 4: sparse_row_kernel<T, 4><<<grid, kThreads, 0, s>>>(a); break;
    case 8: sparse_row_kernel<T, 8><<<grid, kThreads, 0, s>>>(a); break;
    case 16: sparse_row_kernel<T, 16><<<grid, kThreads, 0, s>>>(a); break;
    case 32: sparse_row_kernel<T, 32><<<grid, kThreads, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T> cudaError_t col_launch(int w, unsigned grid, cudaStream_t s, const SparseArgs &a)
{
    switch (w) {
    case 1: sparse_col_kernel<T, 1><<<grid, kThreads, 0, s>>>(a); break;
    case 2: sparse_col_kernel<T, 2><<<grid, kThreads, 0, s>>>(a); break;
    case 4: sparse_col_kernel<T, 4><<<grid, kThreads, 0, s>>>(a); break;
    case 8: sparse_col_kernel<T, 8><<<grid, kThreads, 0, s>>>(a); break;
    case 16: sparse_col_kernel<T, 16><<<grid, kThreads, 0, s>>>(a); break;
    case 32: sparse_col_kernel<T, 32><<<grid, kThreads, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

void sparse_blocks_per_sm(bool f64, int w_row, int w_col, int *row_bps, int *col_bps)
{
    *row_bps = f64 ? blocks_per_sm_row<double>(w_row) : blocks_per_sm_row<float>(w_row);
    *col_bps = f64 ? blocks_per_sm_col<double>(w_col) : blocks_per_sm_col<float>(w_col);
}

cudaError_t sparse_row_launch(bool f64, cudaStream_t s, const SparseArgs &a)
{
    const unsigned grid = (unsigned)(a.n_row_pieces + a.row_light_ctas);
    return f64 ? row_launch<double>(a.w_row, grid, s, a) : row_launch<float>(a.w_row, grid, s, a);
}

cudaError_t sparse_col_launch(bool f64, cudaStream_t s, const SparseArgs &a)
{
    const unsigned grid = (unsigned)(a.n_col_pieces + a.col_light_ctas);
    return f64 ? col_launch<double>(a.w_col, grid, s, a) : col_launch<float>(a.w_col, grid, s, a);
}

cudaError_t sparse_step_launch(bool f64, cudaStream_t s, const SparseArgs &a)
{
    const unsigned grid = (unsigned)a.step_ctas;
    if (f64)
        sparse_step_kernel<double><<<grid, kThreads, 0, s>>>(a);
    else
        sparse_step_kernel<float><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t sparse_norms_launch(bool f64, int grid, cudaStream_t s, const SparseArgs &a, double *n2, int *flags)
{
    if (f64)
        sparse_norms_kernel<double><<<grid, kThreads, 0, s>>>(a, n2, flags);
    else
        sparse_norms_kernel<float><<<grid, kThreads, 0, s>>>(a, n2, flags);
    return cudaGetLastError();
}

cudaError_t sparse_verify_launch(bool f64, int grid, cudaStream_t s, const SparseArgs &a, const VerifyArgs &v)
{
    if (f64)
        sparse_verify_kernel<double><<<grid, kThreads, 0, s>>>(a, v);
    else
        sparse_verify_kernel<float><<<grid, kThreads, 0, s>>>(a, v);
    return cudaGetLastError();
}


size_t sparse_resident_smem(bool f64, long long m, long long n)
{
    const size_t t = f64 ? 8 : 4;
    return (size_t)n * (16 + t) + (size_t)m * t + (size_t)(m + 1) * 8;
}

cudaError_t sparse_resident_prepare(bool f64, size_t smem)
{
    if (f64)
        return cudaFuncSetAttribute(sparse_resident_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
    return cudaFuncSetAttribute(sparse_resident_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
}

cudaError_t sparse_resident_launch(bool f64, cudaStream_t s, const SparseArgs &a, size_t smem, int iters)
{
    if (a.mode != 0 || smem > kResSmemMax)
        return cudaErrorInvalidValue;
    if (f64)
        sparse_resident_kernel<double><<<1, kResThreads, smem, s>>>(a, iters);
    else
        sparse_resident_kernel<float><<<1, kResThreads, smem, s>>>(a, iters);
    return cudaGetLastError();
}

cudaError_t sparse_rows_launch(bool f64, cudaStream_t s, const SparseArgs &a, long long row0, long long rows,
                               double *out)
{
    if (rows <= 0)
        return cudaSuccess;
    if (f64)
        sparse_rows_kernel<double><<<(unsigned)rows, 128, 0, s>>>(a, row0, rows, out);
    else
        sparse_rows_kernel<float><<<(unsigned)rows, 128, 0, s>>>(a, row0, rows, out);
    return cudaGetLastError();
}

}  // namespace nsli
