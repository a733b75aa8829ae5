// nsli_kernels.cu -- device code of the pseudo-projection solver (sm_103a).
//
// Kernels of one iteration (Sokolinsky & Sokolinskaya 2020):
//   map_kernel     Map of Eq. 13 fused with the CTA-level Reduce(+): streams
//                  the CTA's contiguous block of rows of A once through a
//                  shared-memory ring filled by the bulk-copy (TMA) engine,
//                  forms r_i = <a_i, x> - b_i(k) with b_i(k) = b0_i + k rho Av_i
//                  (Section 5 tick, never materialised), and while the row is
//                  still on chip adds the positive slice (Eq. 7)
//                  r_i / ||a_i||^2 * a_i into register-resident partial sums.
//   reduce_update  deterministic fixed-order sum of the per-CTA partials,
//                  the stopping test (Eq. 10 and the step rule), and the step
//                  x <- x - lambda y / h (Eq. 8) or x <- x - lambda y / ||y||
//                  (Eq. 12), with ||dx|| in binary64.
// Plus the set-up kernels (quantisation of A, binary64 row norms, per-row
// records) and the binary64 feasibility check (Eq. 10 on the stored A).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <cfloat>
#include <cmath>

#include "nsli.h"
#include "nsli_internal.h"
#include "nsli_async.cuh"
#include "nsli_sumsq.cuh"

namespace nsli {

// ---------------------------------------------------------------- traits ----

template <int S> struct Traits;
template <> struct Traits<NSLI_F64> {
    using acc = double;
    using meta = RowMeta64;
    static constexpr int EPV = 2;   // elements per 16-byte vector
    static constexpr int BYTES = 8;
};
template <> struct Traits<NSLI_F32> {
    using acc = float;
    using meta = RowMeta32;
    static constexpr int EPV = 4;
    static constexpr int BYTES = 4;
};
template <> struct Traits<NSLI_BF16> {
    using acc = float;
    using meta = RowMeta32;
    static constexpr int EPV = 8;
    static constexpr int BYTES = 2;
};
template <> struct Traits<NSLI_FP8E4M3> {
    using acc = float;
    using meta = RowMeta32;
    static constexpr int EPV = 16;
    static constexpr int BYTES = 1;
};

__device__ __forceinline__ float meta_scale(const RowMeta32 &m) { return m.scale; }
__device__ __forceinline__ double meta_scale(const RowMeta64 &) { return 1.0; }

__device__ __forceinline__ void fp8x2_to_float2(unsigned int pair, float &lo, float &hi)
{
    __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(pair & 0xffffu), __NV_E4M3);
    const float2 f = __half22float2(__half2(hr));
    lo = f.x;
    hi = f.y;
}

// Decode one 16-byte vector of stored elements into the accumulation type.
template <int S>
__device__ __forceinline__ void decode(const uint4 q, typename Traits<S>::acc (&a)[Traits<S>::EPV]);

template <> __device__ __forceinline__ void decode<NSLI_F64>(const uint4 q, double (&a)[2])
{
    a[0] = __hiloint2double((int)q.y, (int)q.x);
    a[1] = __hiloint2double((int)q.w, (int)q.z);
}
template <> __device__ __forceinline__ void decode<NSLI_F32>(const uint4 q, float (&a)[4])
{
    a[0] = __uint_as_float(q.x);
    a[1] = __uint_as_float(q.y);
    a[2] = __uint_as_float(q.z);
    a[3] = __uint_as_float(q.w);
}
template <> __device__ __forceinline__ void decode<NSLI_BF16>(const uint4 q, float (&a)[8])
{
    const unsigned int w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        a[2 * k] = __uint_as_float(w[k] << 16);
        a[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
    }
}
template <> __device__ __forceinline__ void decode<NSLI_FP8E4M3>(const uint4 q, float (&a)[16])
{
    const unsigned int w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        fp8x2_to_float2(w[k], a[4 * k], a[4 * k + 1]);
        fp8x2_to_float2(w[k] >> 16, a[4 * k + 2], a[4 * k + 3]);
    }
}

// barriers and bulk copies: nsli_async.cuh

template <typename T> __device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// d0 += a0 * b0 and d1 += a1 * b1 with one packed binary32x2 FMA
// (round to nearest; the same result as two scalar fmaf).
__device__ __forceinline__ void fma2(float &d0, float &d1, float a0, float a1, float b0, float b1)
{
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rd, {%0, %1};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rd;\n\t"
        "mov.b64 {%0, %1}, rd;\n\t}"
        : "+f"(d0), "+f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}
__device__ __forceinline__ void fma2(double &d0, double &d1, double a0, double a1, double b0, double b1)
{
    d0 = fma(a0, b0, d0);
    d1 = fma(a1, b1, d1);
}

template <typename T> __device__ __forceinline__ T neg_inf();
template <> __device__ __forceinline__ float neg_inf<float>() { return -INFINITY; }
template <> __device__ __forceinline__ double neg_inf<double>() { return -INFINITY; }

// ------------------------------------------------------------- Map kernel --
//
// Block = `nt` threads (a multiple of 32, at most 512).  Thread t owns the
// 16-byte vectors j = t + v * nt (v < VPT) of every row, i.e. fixed column
// slices, and keeps the matching slices of x and of the CTA's partial y in
// registers.  Thread 0 also issues the bulk copies: slots 0..nstage-1 up
// front, then, right after the first barrier of slot s, the refill of the
// stage that slot s-1 released (every warp released it before reaching that
// barrier, so the wait is immediate).
//
// Rows are handled in groups of RG (compile time; a slot holds a multiple of
// RG rows, rows past the CTA's end are masked).  Per group: per-thread
// partial dots (packed FMAs), a transposed warp reduction that folds the RG
// rows into one butterfly (lanes [q*32/RG, (q+1)*32/RG) end with row q), one
// barrier, a second transposed reduction of the per-warp totals that every
// warp performs in the same order (so all threads hold bit-identical r_i),
// then the violated rows are added into the y registers from the same
// shared-memory copy of the row.  GUARD = false when every thread's vectors
// lie inside the row (no per-vector bounds tests).

// Sum v[0..RG) over the warp with one folded butterfly; returns, in lane l,
// the warp total of row l / (32 / RG).
template <int RG, typename T> __device__ __forceinline__ T warp_fold_rows(const T (&v)[RG], int lane)
{
    if constexpr (RG == 1) {
        return warp_sum(v[0]);
    } else if constexpr (RG == 2) {
        const bool hi = (lane & 16) != 0;
        T keep = hi ? v[1] : v[0];
        const T send = hi ? v[0] : v[1];
        keep += __shfl_xor_sync(0xffffffffu, send, 16);
#pragma unroll
        for (int off = 8; off > 0; off >>= 1)
            keep += __shfl_xor_sync(0xffffffffu, keep, off);
        return keep;
    } else if constexpr (RG == 8) {
        // lanes [4q, 4q + 4) end with row q: three exchange levels, then a
        // butterfly over four lanes (the pairing of every level as in the
        // one-row butterfly)
        const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0, b2 = (lane & 4) != 0;
        T k[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const T keep = b4 ? v[q + 4] : v[q];
            const T send = b4 ? v[q] : v[q + 4];
            k[q] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
        T m0 = b3 ? k[2] : k[0], m1 = b3 ? k[3] : k[1];
        const T t0 = b3 ? k[0] : k[2], t1 = b3 ? k[1] : k[3];
        m0 += __shfl_xor_sync(0xffffffffu, t0, 8);
        m1 += __shfl_xor_sync(0xffffffffu, t1, 8);
        T keep = b2 ? m1 : m0;
        const T send = b2 ? m0 : m1;
        keep += __shfl_xor_sync(0xffffffffu, send, 4);
        keep += __shfl_xor_sync(0xffffffffu, keep, 2);
        keep += __shfl_xor_sync(0xffffffffu, keep, 1);
        return keep;
    } else {
        static_assert(RG == 4, "row groups of 1, 2, 4 or 8");
        const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0;
        T k0 = b4 ? v[2] : v[0], k1 = b4 ? v[3] : v[1];
        const T s0 = b4 ? v[0] : v[2], s1 = b4 ? v[1] : v[3];
        k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
        k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
        T keep = b3 ? k1 : k0;
        const T send = b3 ? k0 : k1;
        keep += __shfl_xor_sync(0xffffffffu, send, 8);
#pragma unroll
        for (int off = 4; off > 0; off >>= 1)
            keep += __shfl_xor_sync(0xffffffffu, keep, off);
        return keep;
    }
}

// The Map of rows [row_begin, row_end) of one problem by the calling CTA:
// the CTA-level sum of the positive slices goes to part_row (ld elements of
// the accumulation type), the CTA's counters to *stat_out.  Threads
// t < nt own vectors t + v * nt (v < vpt_used <= VPT); the others only take
// part in the barriers and reductions (with zero partial sums).  PARTIAL is
// false when every thread of the block owns VPT vectors (nt == blockDim.x,
// vpt_used == VPT), which keeps the guard-free instances free of tests.
template <int S, int VPT, bool GUARD, bool PARTIAL>
__device__ __forceinline__ void map_body(const MapArgs &p, const long long row_begin, const long long row_end,
                                         void *part_row, PartStat *stat_out, const int nt, const int vpt_used)
{
    using Tr = Traits<S>;
    using Acc = typename Tr::acc;
    using Meta = typename Tr::meta;
    constexpr int EPV = Tr::EPV;
    constexpr int RG = map_rows_per_group(VPT, (int)sizeof(Acc));
    static_assert(RG * 32 * sizeof(Acc) <= 1024, "a group's warp sums fit half the buffer");
    constexpr int W = 32 / RG;                 // lanes per row in the folded reductions
    constexpr int NCH = (VPT >= 4 && RG <= 2) ? 2 : 1;  // independent chains per row

    DevState *st = p.st;

    extern __shared__ __align__(128) unsigned char smem[];
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem);  // full[8], empty[8]
    Acc *red = reinterpret_cast<Acc *>(smem + 256);                          // two halves of 1024 bytes
    unsigned char *stages = smem + kSmemHeader;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int nwarps = (int)blockDim.x >> 5;

    const int R = p.rows_per_slot;
    const int nslots = (int)((row_end - row_begin + R - 1) / R);
    const unsigned char *Ab = static_cast<const unsigned char *>(p.A);
    const unsigned char *Mb = static_cast<const unsigned char *>(p.meta);

    // issue the copies of slot s into its stage (thread 0 only)
    const int skip = (blockIdx.x == 0) ? p.skip_slot : -1;
    auto issue = [&](int s) {
        if (s == skip)
            return;  // failure injection: a wait that nothing will complete
        const int stage = s % p.nstage;
        const long long r0 = row_begin + (long long)s * R;
        const long long left = row_end - r0;
        const int rows = (int)(left < R ? left : R);
        const unsigned int bytesA = (unsigned int)rows * (unsigned int)p.row_bytes;
        const unsigned int bytesM = (unsigned int)rows * 32u;
        unsigned char *dst = stages + (size_t)stage * p.stage_stride;
        const unsigned int fb = smem_u32(&bars[stage]);
        mbar_expect_tx(fb, bytesA + bytesM);
        bulk_g2s(smem_u32(dst), Ab + r0 * (long long)p.row_bytes, bytesA, fb);
        bulk_g2s(smem_u32(dst + (size_t)R * p.row_bytes), Mb + r0 * 32, bytesM, fb);
    };

    int issued = 0;
    if (tid == 0) {
        for (int s = 0; s < p.nstage; ++s) {
            mbar_init(smem_u32(&bars[s]), 1u);
            mbar_init(smem_u32(&bars[8 + s]), (unsigned int)nwarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const int first = nslots < p.nstage ? nslots : p.nstage;
        for (int s = 0; s < first; ++s)
            issue(s);
        issued = first;
    }
    __syncthreads();

    // shared-memory byte offsets of this thread's vectors within a row
    int voff[VPT];
    bool vok[VPT];
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        const int j = tid + v * nt;
        voff[v] = j * 16;
        vok[v] = (!PARTIAL || (v < vpt_used && tid < nt)) && (!GUARD || j < p.nv);
    }

    Acc xr[VPT][EPV];
    Acc yr[VPT][EPV];
    {
        const Acc *xg = static_cast<const Acc *>(p.x);
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const int j = tid + v * nt;
#pragma unroll
            for (int e = 0; e < EPV; ++e) {
                xr[v][e] = vok[v] ? xg[(long long)j * EPV + e] : Acc(0);
                yr[v][e] = Acc(0);
            }
        }
    }
    const Acc tk = (Acc)((double)st->tick * st->rho);

    long long h_loc = 0;
    Acc mv = neg_inf<Acc>(), mn = neg_inf<Acc>(), mb = Acc(0);
    int grp_counter = 0;
    int aborted = 0;
    int consumed = 0;

    for (int s = 0; s < nslots; ++s) {
        const int stage = s % p.nstage;
        const unsigned int ph = (unsigned int)((s / p.nstage) & 1);
        int timed_out = mbar_wait_bounded(smem_u32(&bars[stage]), ph) ? 0 : 1;
        const unsigned char *sbase = stages + (size_t)stage * p.stage_stride;
        const Meta *smeta = reinterpret_cast<const Meta *>(sbase + (size_t)R * p.row_bytes);
        const long long r0 = row_begin + (long long)s * R;
        const long long left = row_end - r0;
        const int rows = (int)(left < R ? left : R);

        for (int g0 = 0; g0 < rows; g0 += RG) {
            // ---- per-thread partial dots of the RG rows of this group
            Acc acc[RG];
#pragma unroll
            for (int rr = 0; rr < RG; ++rr) {
                const unsigned char *row = sbase + (size_t)(g0 + rr) * p.row_bytes;
                Acc pe[NCH], po[NCH];
#pragma unroll
                for (int q = 0; q < NCH; ++q) {
                    pe[q] = Acc(0);
                    po[q] = Acc(0);
                }
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    if (vok[v]) {
                        Acc a[EPV];
                        decode<S>(*reinterpret_cast<const uint4 *>(row + voff[v]), a);
#pragma unroll
                        for (int e = 0; e < EPV; e += 2)
                            fma2(pe[v % NCH], po[v % NCH], a[e], a[e + 1], xr[v][e], xr[v][e + 1]);
                    }
                }
                Acc t = pe[0] + po[0];
#pragma unroll
                for (int q = 1; q < NCH; ++q)
                    t += pe[q] + po[q];
                acc[rr] = t;
            }
            Acc *rb = red + (grp_counter & 1) * (1024 / (int)sizeof(Acc));
            const Acc wsum = warp_fold_rows<RG>(acc, lane);
            if ((lane & (W - 1)) == 0)
                rb[(lane / W) * 32 + warp] = wsum;
            aborted = bar_all_or((int)blockDim.x, timed_out);  // every thread of the block arrives
            if (aborted)
                break;
            if (tid == 0 && g0 == 0 && s >= 1 && issued < nslots) {
                // slot s-1 was released by every warp before this barrier
                const int sp = s - 1;
                if (mbar_wait_bounded(smem_u32(&bars[8 + sp % p.nstage]),
                                      (unsigned int)((sp / p.nstage) & 1))) {
                    issue(issued);
                    ++issued;
                } else {
                    timed_out = 1;  // reported below
                }
            }

            // ---- block totals: lane (q, i) adds the partials of warps
            // i, i + W, ... of row q; every warp runs the same tree
            Acc tsum = Acc(0);
            {
                const int q = lane / W, i = lane % W;
                for (int w = i; w < nwarps; w += W)
                    tsum += rb[q * 32 + w];
#pragma unroll
                for (int off = W / 2; off > 0; off >>= 1)
                    tsum += __shfl_xor_sync(0xffffffffu, tsum, off);
            }
            Acc c[RG];
#pragma unroll
            for (int rr = 0; rr < RG; ++rr) {
                const Acc dot = (RG == 1) ? tsum : __shfl_sync(0xffffffffu, tsum, rr * W);
                const bool valid = (g0 + rr) < rows;
                const Meta md = smeta[valid ? g0 + rr : 0];
                const Acc sc = (Acc)meta_scale(md);
                const Acc bi = fma(tk, (Acc)md.av, (Acc)md.b0);
                const Acc ri = (S == NSLI_FP8E4M3) ? dot * sc - bi : dot - bi;
                const bool viol = valid && ri > Acc(0);
                c[rr] = viol ? ((S == NSLI_FP8E4M3) ? ri * (Acc)md.inv_n2 * sc : ri * (Acc)md.inv_n2) : Acc(0);
                if (warp == 0 && valid) {  // warp-uniform; thread 0 writes them out
                    h_loc += viol ? 1 : 0;
                    mv = ri > mv ? ri : mv;
                    const Acc rn = ri * (Acc)md.inv_n;
                    mn = rn > mn ? rn : mn;
                    const Acc ab = bi < Acc(0) ? -bi : bi;
                    mb = ab > mb ? ab : mb;
                }
            }
            // ---- add the positive slices of the violated rows
#pragma unroll
            for (int rr = 0; rr < RG; ++rr) {
                if (c[rr] != Acc(0)) {
                    const unsigned char *row = sbase + (size_t)(g0 + rr) * p.row_bytes;
                    const Acc cr = c[rr];
#pragma unroll
                    for (int v = 0; v < VPT; ++v) {
                        if (vok[v]) {
                            Acc a[EPV];
                            decode<S>(*reinterpret_cast<const uint4 *>(row + voff[v]), a);
#pragma unroll
                            for (int e = 0; e < EPV; e += 2)
                                fma2(yr[v][e], yr[v][e + 1], cr, cr, a[e], a[e + 1]);
                        }
                    }
                }
            }
            ++grp_counter;
            if (timed_out && tid == 0)
                atomicOr(&st->error, ERRF_TIMEOUT);
        }
        if (aborted)
            break;
        __syncwarp();
        if (lane == 0)
            mbar_arrive(smem_u32(&bars[8 + stage]));
        consumed = s + 1;
    }

    if (aborted) {
        // Give up: record the error and wait (bounded) for every bulk copy
        // still in flight before the CTA exits.
        if (tid == 0) {
            atomicOr(&st->error, ERRF_TIMEOUT);
            for (int s = consumed; s < issued; ++s)
                mbar_wait_bounded(smem_u32(&bars[s % p.nstage]), (unsigned int)((s / p.nstage) & 1));
        }
        return;
    }

    Acc *py = static_cast<Acc *>(part_row);
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        if (vok[v]) {
            const long long j = tid + v * nt;
#pragma unroll
            for (int e = 0; e < EPV; ++e)
                py[j * EPV + e] = yr[v][e];
        }
    }
    if (tid == 0) {
        PartStat ps;
        ps.h = h_loc;
        ps.maxviol = (double)mv;
        ps.maxnorm = (double)mn;
        ps.maxb = (double)mb;
        *stat_out = ps;
    }
}

// One problem: CTA b maps its contiguous balanced block of rows.
template <int S, int VPT, bool GUARD>
__global__ void __launch_bounds__(kMapMaxConsumers, 1) map_kernel(const MapArgs p)
{
    using Acc = typename Traits<S>::acc;
    if (!p.ignore_done && *(volatile int *)&p.st->done)
        return;
    const long long b = blockIdx.x;
    const long long row_begin = b * p.rows_base + (b < p.rows_rem ? b : (long long)p.rows_rem);
    const long long row_end = row_begin + p.rows_base + (b < p.rows_rem ? 1 : 0);
    map_body<S, VPT, GUARD, false>(p, row_begin, row_end, static_cast<Acc *>(p.part_y) + b * p.ld,
                                   p.part_stat + b, (int)blockDim.x, VPT);
}

// Many problems in one launch: CTA b maps work item b (a block of rows of
// one problem) with that problem's own thread mapping, so a problem's
// partial sums do not depend on which other problems share the launch.
template <int S, int VPT>
__global__ void __launch_bounds__(kMapMaxConsumers, 1) map_group_kernel(const GroupProblem *probs,
                                                                        const GroupItem *items)
{
    using Acc = typename Traits<S>::acc;
    const GroupItem it = items[blockIdx.x];
    const GroupProblem &gp = probs[it.prob];
    if (*(volatile int *)&gp.map.st->done)
        return;
    map_body<S, VPT, true, true>(gp.map, it.row_begin, it.row_end,
                           static_cast<Acc *>(gp.map.part_y) + (long long)it.part * gp.map.ld,
                           gp.map.part_stat + it.part, gp.nt, gp.vpt);
}

// --------------------------------------------------- Map, long rows --------
//
// Rows longer than the register-resident limit (n > 16384 for 4-, 2- and
// 1-byte storage, n > 8192 for binary64).  The CTA takes its rows RG at a
// time and walks them in column chunks of 512 * 8 / RG 16-byte vectors:
// thread t owns vectors t, t + 512, ... of every chunk.  Pass 1 streams the chunk of
// the RG rows from HBM with 16-byte loads and accumulates the dots against
// the chunk of x (loaded once per group, 16 bytes at a time); one block
// reduction gives the RG residuals.  A thread owns 8 / RG vectors per chunk,
// so every thread has 8 row vectors in flight whatever RG is.  Pass 2 re-reads the chunks of the violated rows and adds
// r_i / ||a_i||^2 * a_i into the CTA's row of partial sums, each thread its
// own columns (no atomics, a fixed order).  The host picks RG (4, 2 or 1) so
// that the rows of a group, over all CTAs, stay within a budget of L2 until
// pass 2 re-reads them, and keeps the partial sums in shared memory (SY)
// when a row of them fits there; otherwise they live in global memory.
constexpr int kLongThreads = 512;

// x entries of one 16-byte vector of A, loaded 16 bytes at a time
template <typename Acc, int EPV> __device__ __forceinline__ void load_x_vec(const Acc *xg, long long j, Acc (&xv)[EPV])
{
    const uint4 *src = reinterpret_cast<const uint4 *>(xg + j * EPV);
    constexpr int NQ = EPV * (int)sizeof(Acc) / 16;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const uint4 w = __ldg(src + q);
        const Acc *a = reinterpret_cast<const Acc *>(&w);
#pragma unroll
        for (int e = 0; e < 16 / (int)sizeof(Acc); ++e)
            xv[q * (16 / (int)sizeof(Acc)) + e] = a[e];
    }
}

template <int S, int RG, bool SY>
__global__ void __launch_bounds__(kLongThreads, 1) map_long_kernel(const MapArgs p)
{
    using Tr = Traits<S>;
    using Acc = typename Tr::acc;
    using Meta = typename Tr::meta;
    constexpr int EPV = Tr::EPV;
    constexpr int W = 32 / RG;
    // vectors per thread per chunk: 8 row vectors in flight per thread
    // whatever the group size
    constexpr int kLongVPT = 8 / RG;

    DevState *st = p.st;
    if (!p.ignore_done && *(volatile int *)&st->done)
        return;
    __shared__ Acc red[2][RG][32];
    extern __shared__ __align__(16) unsigned char long_smem[];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nwarps = kLongThreads / 32;
    const long long b = blockIdx.x;
    const long long row_begin = b * p.rows_base + (b < p.rows_rem ? b : (long long)p.rows_rem);
    const long long row_end = row_begin + p.rows_base + (b < p.rows_rem ? 1 : 0);
    const long long nv = p.nv;
    const long long chunk = (long long)kLongThreads * kLongVPT;
    const int nchunks = (int)((nv + chunk - 1) / chunk);
    const unsigned char *Ab = static_cast<const unsigned char *>(p.A);
    const Meta *meta = static_cast<const Meta *>(p.meta);
    const Acc *xg = static_cast<const Acc *>(p.x);
    Acc *py_g = static_cast<Acc *>(p.part_y) + b * p.ld;
    Acc *py = SY ? reinterpret_cast<Acc *>(long_smem) : py_g;
    for (long long e = tid; e < p.ld; e += kLongThreads)
        py[e] = Acc(0);
    const Acc tk = (Acc)((double)st->tick * st->rho);

    long long h_loc = 0;
    Acc mv = neg_inf<Acc>(), mn = neg_inf<Acc>(), mb = Acc(0);
    int grp_counter = 0;
    for (long long r0 = row_begin; r0 < row_end; r0 += RG) {
        const int gr = (int)((row_end - r0) < RG ? (row_end - r0) : RG);
        Acc pe[RG], po[RG];
#pragma unroll
        for (int rr = 0; rr < RG; ++rr) {
            pe[rr] = Acc(0);
            po[rr] = Acc(0);
        }
        // ---- pass 1: dots of the group's rows, chunk by chunk
        for (int c = 0; c < nchunks; ++c) {
            long long j[kLongVPT];
            bool ok[kLongVPT];
            Acc xv[kLongVPT][EPV];
            uint4 q[RG][kLongVPT];
#pragma unroll
            for (int v = 0; v < kLongVPT; ++v) {
                j[v] = (long long)c * chunk + tid + v * kLongThreads;
                ok[v] = j[v] < nv;
#pragma unroll
                for (int rr = 0; rr < RG; ++rr)
                    q[rr][v] = (ok[v] && rr < gr)
                                   ? __ldg(reinterpret_cast<const uint4 *>(Ab + (r0 + rr) * (long long)p.row_bytes) + j[v])
                                   : make_uint4(0u, 0u, 0u, 0u);
                if (ok[v]) {
                    load_x_vec<Acc, EPV>(xg, j[v], xv[v]);
                } else {
#pragma unroll
                    for (int e = 0; e < EPV; ++e)
                        xv[v][e] = Acc(0);
                }
            }
#pragma unroll
            for (int rr = 0; rr < RG; ++rr) {
#pragma unroll
                for (int v = 0; v < kLongVPT; ++v) {
                    Acc a[EPV];
                    decode<S>(q[rr][v], a);
#pragma unroll
                    for (int e = 0; e < EPV; e += 2)
                        fma2(pe[rr], po[rr], a[e], a[e + 1], xv[v][e], xv[v][e + 1]);
                }
            }
        }
        Acc acc[RG];
#pragma unroll
        for (int rr = 0; rr < RG; ++rr)
            acc[rr] = pe[rr] + po[rr];
        Acc *rb = &red[grp_counter & 1][0][0];
        const Acc wsum = warp_fold_rows<RG>(acc, lane);
        if ((lane & (W - 1)) == 0)
            rb[(lane / W) * 32 + warp] = wsum;
        __syncthreads();
        Acc tsum = Acc(0);
        {
            const int qq = lane / W, i = lane % W;
            for (int w = i; w < nwarps; w += W)
                tsum += rb[qq * 32 + w];
#pragma unroll
            for (int off = W / 2; off > 0; off >>= 1)
                tsum += __shfl_xor_sync(0xffffffffu, tsum, off);
        }
        Acc cr[RG];
        bool any = false;
#pragma unroll
        for (int rr = 0; rr < RG; ++rr) {
            const Acc dot = __shfl_sync(0xffffffffu, tsum, rr * W);
            const bool valid = rr < gr;
            const Meta md = meta[r0 + (valid ? rr : 0)];
            const Acc sc = (Acc)meta_scale(md);
            const Acc bi = fma(tk, (Acc)md.av, (Acc)md.b0);
            const Acc ri = (S == NSLI_FP8E4M3) ? dot * sc - bi : dot - bi;
            const bool viol = valid && ri > Acc(0);
            cr[rr] = viol ? ((S == NSLI_FP8E4M3) ? ri * (Acc)md.inv_n2 * sc : ri * (Acc)md.inv_n2) : Acc(0);
            any = any || viol;
            if (warp == 0 && valid) {
                h_loc += viol ? 1 : 0;
                mv = ri > mv ? ri : mv;
                const Acc rn = ri * (Acc)md.inv_n;
                mn = rn > mn ? rn : mn;
                const Acc ab = bi < Acc(0) ? -bi : bi;
                mb = ab > mb ? ab : mb;
            }
        }
        // ---- pass 2: add the violated rows' slices (rows re-read from L2)
        if (any) {
            for (int c = 0; c < nchunks; ++c) {
#pragma unroll
                for (int v = 0; v < kLongVPT; ++v) {
                    const long long jj = (long long)c * chunk + tid + v * kLongThreads;
                    if (jj >= nv)
                        continue;
                    Acc y[EPV];
#pragma unroll
                    for (int e = 0; e < EPV; ++e)
                        y[e] = py[jj * EPV + e];
#pragma unroll
                    for (int rr = 0; rr < RG; ++rr) {
                        if (cr[rr] != Acc(0)) {
                            Acc a[EPV];
                            decode<S>(__ldg(reinterpret_cast<const uint4 *>(Ab + (r0 + rr) * (long long)p.row_bytes) + jj), a);
#pragma unroll
                            for (int e = 0; e < EPV; e += 2)
                                fma2(y[e], y[e + 1], cr[rr], cr[rr], a[e], a[e + 1]);
                        }
                    }
#pragma unroll
                    for (int e = 0; e < EPV; ++e)
                        py[jj * EPV + e] = y[e];
                }
            }
        }
        ++grp_counter;
    }
    if (SY) {
        // each thread wrote only its own columns; the copy-out mixes them
        __syncthreads();
        for (long long e = tid; e < p.ld; e += kLongThreads)
            py_g[e] = py[e];
    }
    if (tid == 0) {
        PartStat ps;
        ps.h = h_loc;
        ps.maxviol = (double)mv;
        ps.maxnorm = (double)mn;
        ps.maxb = (double)mb;
        p.part_stat[b] = ps;
    }
}

// ------------------------------------------ Map, long rows on a cluster ----
//
// A thread-block cluster of C CTAs (C = 2, 4 or 8, one per SM) maps a block
// of rows whose columns it splits: CTA q of the cluster owns the vectors
// [q S, (q + 1) S) of every row (S = slice_nv), keeps the matching slices of
// x and of the cluster's partial y in registers, and streams its slice of
// each row through its own ring of bulk copies (one row slice and the row's
// record per stage).  Per row every CTA forms its partial dot (thread
// chains, warp butterfly, the warps' sums in order), writes it into slot q
// of the row's exchange buffer in EVERY CTA of the cluster (distributed
// shared memory) and arrives on that CTA's exchange barrier; each CTA then
// adds the C partials in rank order, so all of them hold the same r_i, and
// adds the violated row's slice from its own shared-memory copy.  A is read
// from HBM once, with no second pass.  The exchange of row k is waited for
// D rows later (D = cluster_lag, 1..3), while the dots of rows k+1 .. k+D
// run, so the exchange latency is not on the critical path.  Eight exchange
// buffers suffice: a CTA sends row k only after every CTA sent row k - D,
// i.e. after every CTA finished reading rows up to k - 2D - 1, and
// 8 >= 2D + 1.  A row's stage is refilled as soon as every mapping warp has
// finished the row (an "empty" barrier per stage that the warps arrive on
// and the exchange warp waits for), so the ring holds the D + 1 rows in use
// and the rest of its stages are in flight.  Every wait is bounded; all CTAs
// of a cluster meet at a cluster barrier before they exit, so no CTA's
// shared memory is written after it has gone.
__device__ __forceinline__ unsigned int cluster_rank()
{
    unsigned int r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned int map_to_rank(unsigned int addr, unsigned int rank)
{
    unsigned int r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void st_remote(unsigned int raddr, float v)
{
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(raddr), "f"(v) : "memory");
}
__device__ __forceinline__ void st_remote(unsigned int raddr, double v)
{
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(raddr), "d"(v) : "memory");
}
__device__ __forceinline__ void arrive_remote(unsigned int rbar)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(rbar) : "memory");
}
__device__ __forceinline__ bool mbar_test_cluster(unsigned int bar, unsigned int parity)
{
    unsigned int ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cluster_bounded(unsigned int bar, unsigned int parity)
{
    const long long t0 = clock64();
    for (unsigned int it = 0;; ++it) {
        if (mbar_test_cluster(bar, parity))
            return true;
        if ((it & 255u) == 255u && clock64() - t0 > kWaitLimitCycles)
            return false;
    }
}

// shared-memory header of the cluster Map (within kSmemHeader)
constexpr int kClXB = 8;          // exchange buffers (group k uses k % 8)
constexpr int kClMaxStages = 16;  // ring stages (one row slice each)
constexpr int kClFull = 0;        // 16 full barriers (stages)
constexpr int kClXbar = 128;      // 8 exchange barriers
constexpr int kClEmpty = 192;     // 16 empty barriers (stages)
constexpr int kClRed = 512;       // [2][RG][16] warp sums (at most 512 bytes)
constexpr int kClXch = 1024;      // [8][RG][8] exchanged partial dots (at most 1024 bytes)
static_assert(kClEmpty + kClMaxStages * 8 <= kClRed, "cluster Map barriers fit");
static_assert(kClXch + 1024 <= kSmemHeader, "cluster Map header fits");

// 512 threads map; a 17th warp (the exchange warp) issues the bulk copies,
// waits for the exchanges, adds the warps' sums and sends the partial dots,
// so the latency of the remote stores and releases is off the mapping
// warps' path (they only meet it at the per-group block barrier).
constexpr int kClusterCompute = 512;
constexpr int kClusterThreads = kClusterCompute + 32;

// RG = rows per group (1, 2 or 4): the rows of a group share one block
// barrier and one exchange message, and their dependent chains interleave.  The
// arithmetic of every row is the same for both (the warp fold of two rows
// adds the same operands in the same tree as one warp butterfly per row,
// and rows enter y in row order).
template <int S, int VPT, int RG>
__global__ void __launch_bounds__(kClusterThreads, 1) map_cluster_kernel(const MapArgs p)
{
    static_assert(RG == 1 || RG == 2 || RG == 4, "one, two or four rows per group");
    static_assert(2 * RG * 16 * sizeof(typename Traits<S>::acc) <= kClXch - kClRed, "warp sums fit");
    static_assert(kClXB * RG * 8 * sizeof(typename Traits<S>::acc) <= 1024, "exchange buffers fit");
    using Tr = Traits<S>;
    using Acc = typename Tr::acc;
    using Meta = typename Tr::meta;
    constexpr int EPV = Tr::EPV;
    constexpr int NCW = kClusterCompute / 32;   // mapping warps

    DevState *st = p.st;
    if (!p.ignore_done && *(volatile int *)&st->done)
        return;   // the same for every CTA of the grid
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned long long *full = reinterpret_cast<unsigned long long *>(smem + kClFull);
    unsigned long long *xbar = reinterpret_cast<unsigned long long *>(smem + kClXbar);
    unsigned long long *empty = reinterpret_cast<unsigned long long *>(smem + kClEmpty);
    Acc *xch = reinterpret_cast<Acc *>(smem + kClXch);   // [group % 8][row][rank]
    Acc *red = reinterpret_cast<Acc *>(smem + kClRed);   // [group & 1][row][warp]
    unsigned char *stages = smem + kSmemHeader;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool xw = warp == NCW;                 // the exchange warp
    const bool leader = xw && lane == 0;
    const int C = p.cluster;
    const unsigned int rank = cluster_rank();
    const long long cl = blockIdx.x / C;
    const long long row_begin = cl * p.rows_base + (cl < p.rows_rem ? cl : (long long)p.rows_rem);
    const long long row_end = row_begin + p.rows_base + (cl < p.rows_rem ? 1 : 0);
    const int nrows = (int)(row_end - row_begin);
    const int ngroups = (nrows + RG - 1) / RG;
    const long long v0 = (long long)rank * p.slice_nv;
    const int my_nv = (int)max(0ll, min((long long)p.slice_nv, (long long)p.nv - v0));
    const unsigned int slice_bytes = (unsigned int)my_nv * 16u;
    const unsigned int meta_off = (unsigned int)p.slice_nv * 16u;   // record after the largest slice
    const unsigned char *Ab = static_cast<const unsigned char *>(p.A);
    const unsigned char *Mb = static_cast<const unsigned char *>(p.meta);

    auto issue = [&](int s) {   // row s of the block into its stage
        const int stage = s % p.nstage;
        const long long row = row_begin + s;
        unsigned char *dst = stages + (size_t)stage * p.stage_stride;
        const unsigned int fb = smem_u32(&full[stage]);
        mbar_expect_tx(fb, slice_bytes + 32u);
        if (slice_bytes)
            bulk_g2s(smem_u32(dst), Ab + row * (long long)p.row_bytes + v0 * 16, slice_bytes, fb);
        bulk_g2s(smem_u32(dst + meta_off), Mb + row * 32, 32u, fb);
    };

    if (tid == 0) {
        for (int q = 0; q < p.nstage; ++q) {
            mbar_init(smem_u32(&full[q]), 1u);
            mbar_init(smem_u32(&empty[q]), (unsigned int)NCW);
        }
        for (int q = 0; q < kClXB; ++q)
            mbar_init(smem_u32(&xbar[q]), (unsigned int)C);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    cluster_sync_all();   // every exchange barrier of the cluster is initialised
    int issued = 0;
    if (leader) {
        const int first = nrows < p.nstage ? nrows : p.nstage;
        for (int q = 0; q < first; ++q)
            issue(q);
        issued = first;
    }

    int voff[VPT];
    bool vok[VPT];
    Acc xr[VPT][EPV], yr[VPT][EPV];
    {
        const Acc *xg = static_cast<const Acc *>(p.x);
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const int j = tid + v * kClusterCompute;
            voff[v] = j * 16;
            vok[v] = !xw && j < my_nv;
#pragma unroll
            for (int e = 0; e < EPV; ++e) {
                xr[v][e] = vok[v] ? xg[(v0 + j) * EPV + e] : Acc(0);
                yr[v][e] = Acc(0);
            }
        }
    }
    const Acc tk = (Acc)((double)st->tick * st->rho);
    long long h_loc = 0;
    Acc mv = neg_inf<Acc>(), mn = neg_inf<Acc>(), mb = Acc(0);
    int aborted = 0, at = 0, stalled = 0;

    const int D = p.cluster_lag;
    for (int g = 0; g < ngroups + D; ++g) {
        int flag = 0;
        if (g < ngroups && !xw) {
            // partial dots of the group's rows (a missing second row adds 0)
            Acc acc[RG];
#pragma unroll
            for (int rr = 0; rr < RG; ++rr) {
                const int s = g * RG + rr;
                Acc pe = Acc(0), po = Acc(0);
                if (s < nrows) {
                    const int stage = s % p.nstage;
                    if (!mbar_wait_bounded(smem_u32(&full[stage]), (unsigned int)((s / p.nstage) & 1)))
                        flag = 1;
                    const unsigned char *row = stages + (size_t)stage * p.stage_stride;
#pragma unroll
                    for (int v = 0; v < VPT; ++v) {
                        if (vok[v] && !flag) {
                            Acc a[EPV];
                            decode<S>(*reinterpret_cast<const uint4 *>(row + voff[v]), a);
#pragma unroll
                            for (int e = 0; e < EPV; e += 2)
                                fma2(pe, po, a[e], a[e + 1], xr[v][e], xr[v][e + 1]);
                        }
                    }
                }
                acc[rr] = pe + po;
            }
            const Acc ws = warp_fold_rows<RG>(acc, lane);   // lanes [16q, 16q + 16) end with row q
            if ((lane & (32 / RG - 1)) == 0)
                red[(g & 1) * (RG * 16) + (lane / (32 / RG)) * 16 + warp] = ws;
        }
        if (leader && g >= D) {
            const int t = g - D;
            if (stalled || !mbar_wait_cluster_bounded(smem_u32(&xbar[t % kClXB]), (unsigned int)((t / kClXB) & 1)))
                flag = 1;
        }
        aborted = bar_all_or((int)blockDim.x, flag);
        at = g;
        if (aborted)
            break;
        if (xw) {
            if (g < ngroups) {
                // the mapping warps' sums in a fixed butterfly, 32 at a time
                // (rows 2h and 2h + 1 in lanes [0, 16) and [16, 32) of
                // chunk h); lane q sends this CTA's partial dots of the
                // group to CTA q
                constexpr int NCHK = RG >= 2 ? RG / 2 : 1;
                Acc rowv[RG];
#pragma unroll
                for (int h = 0; h < NCHK; ++h) {
                    Acc tot = (RG >= 2 || lane < NCW) ? red[(g & 1) * (RG * 16) + h * 32 + lane] : Acc(0);
#pragma unroll
                    for (int off = 8; off > 0; off >>= 1)
                        tot += __shfl_xor_sync(0xffffffffu, tot, off);
                    rowv[(2 * h) % RG] = __shfl_sync(0xffffffffu, tot, 0);
                    if constexpr (RG >= 2)
                        rowv[2 * h + 1] = __shfl_sync(0xffffffffu, tot, 16);
                }
                if (lane < C) {
                    const unsigned int la = smem_u32(&xch[(g % kClXB) * (RG * 8) + rank]);
                    const unsigned int lb = smem_u32(&xbar[g % kClXB]);
#pragma unroll
                    for (int r = 0; r < RG; ++r)
                        st_remote(map_to_rank(la + (unsigned int)(r * 8 * sizeof(Acc)), (unsigned int)lane), rowv[r]);
                    arrive_remote(map_to_rank(lb, (unsigned int)lane));
                }
            }
            if (lane == 0 && g >= D) {
                // refill the stages of group g - D once every mapping warp
                // has finished it (in this iteration, below)
                const int t = g - D;
                for (int rr = 0; rr < RG && !stalled; ++rr) {
                    const int r = t * RG + rr;
                    if (r >= nrows || issued >= nrows)
                        break;
                    if (mbar_wait_bounded(smem_u32(&empty[r % p.nstage]), (unsigned int)((r / p.nstage) & 1))) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        issue(issued);
                        ++issued;
                    } else {
                        atomicOr(&st->error, ERRF_TIMEOUT);   // the next barrier ends the loop
                        stalled = 1;
                    }
                }
            }
        } else if (g >= D) {
            const int t = g - D;
#pragma unroll
            for (int rr = 0; rr < RG; ++rr) {
                const int r = t * RG + rr;
                if (r >= nrows)
                    break;
                Acc dot = Acc(0);
                for (int q = 0; q < C; ++q)
                    dot += xch[(t % kClXB) * (RG * 8) + rr * 8 + q];
                const unsigned char *row = stages + (size_t)(r % p.nstage) * p.stage_stride;
                const Meta md = *reinterpret_cast<const Meta *>(row + meta_off);
                const Acc sc = (Acc)meta_scale(md);
                const Acc bi = fma(tk, (Acc)md.av, (Acc)md.b0);
                const Acc ri = (S == NSLI_FP8E4M3) ? dot * sc - bi : dot - bi;
                const bool viol = ri > Acc(0);
                const Acc c = viol ? ((S == NSLI_FP8E4M3) ? ri * (Acc)md.inv_n2 * sc : ri * (Acc)md.inv_n2)
                                   : Acc(0);
                if (warp == 0) {
                    h_loc += viol ? 1 : 0;
                    mv = ri > mv ? ri : mv;
                    const Acc rn = ri * (Acc)md.inv_n;
                    mn = rn > mn ? rn : mn;
                    const Acc ab = bi < Acc(0) ? -bi : bi;
                    mb = ab > mb ? ab : mb;
                }
                if (c != Acc(0)) {
#pragma unroll
                    for (int v = 0; v < VPT; ++v) {
                        if (vok[v]) {
                            Acc a[EPV];
                            decode<S>(*reinterpret_cast<const uint4 *>(row + voff[v]), a);
#pragma unroll
                            for (int e = 0; e < EPV; e += 2)
                                fma2(yr[v][e], yr[v][e + 1], c, c, a[e], a[e + 1]);
                        }
                    }
                }
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(smem_u32(&empty[r % p.nstage]));   // row r's stage is free
            }
        }
    }

    if (aborted) {
        // record the error; wait (bounded) for this CTA's copies in flight
        // (rows before the aborted group were waited for already)
        if (leader) {
            atomicOr(&st->error, ERRF_TIMEOUT);
            const int first = at * RG < nrows ? at * RG : nrows;
            for (int q = first; q < issued; ++q)
                mbar_wait_bounded(smem_u32(&full[q % p.nstage]), (unsigned int)((q / p.nstage) & 1));
        }
    } else {
        Acc *py = static_cast<Acc *>(p.part_y) + cl * p.ld + v0 * EPV;
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            if (vok[v]) {
                const long long j = tid + v * (long long)kClusterCompute;
#pragma unroll
                for (int e = 0; e < EPV; ++e)
                    py[j * EPV + e] = yr[v][e];
            }
        }
        if (tid == 0 && rank == 0) {
            PartStat ps;
            ps.h = h_loc;
            ps.maxviol = (double)mv;
            ps.maxnorm = (double)mn;
            ps.maxb = (double)mb;
            p.part_stat[cl] = ps;
        }
    }
    __syncthreads();
    cluster_sync_all();   // no CTA leaves while a peer may still write to it
}

// instances up to the register-resident limit of the storage type (8, 8,
// 4, 2 vectors per thread for binary64, binary32, bf16, fp8)
template <int S> constexpr int cluster_vpt_max() { return S == NSLI_BF16 ? 4 : (S == NSLI_FP8E4M3 ? 2 : 8); }
// rows per group: up to four for FP8 and two for bf16 (short row slices,
// whose fixed cost per group would otherwise dominate); binary64 and
// binary32 take one
template <int S> constexpr int cluster_rg_max() { return S == NSLI_FP8E4M3 ? 4 : (S == NSLI_BF16 ? 2 : 1); }
template <int S, int RG> const void *cluster_fn_v(int vpt)
{
    if (vpt == 1)
        return (const void *)map_cluster_kernel<S, 1, RG>;
    if (vpt == 2)
        return (const void *)map_cluster_kernel<S, 2, RG>;
    if constexpr (cluster_vpt_max<S>() >= 4) {
        if (vpt == 4)
            return (const void *)map_cluster_kernel<S, 4, RG>;
    }
    if constexpr (cluster_vpt_max<S>() >= 8) {
        if (vpt == 8)
            return (const void *)map_cluster_kernel<S, 8, RG>;
    }
    return nullptr;
}
template <int S> const void *cluster_fn_s(int vpt, int rg)
{
    if (rg == 1)
        return cluster_fn_v<S, 1>(vpt);
    if constexpr (cluster_rg_max<S>() >= 4) {
        if (rg == 4)
            return cluster_fn_v<S, 4>(vpt);
    }
    if constexpr (cluster_rg_max<S>() >= 2) {
        if (rg == 2)
            return cluster_fn_v<S, 2>(vpt);
    }
    return nullptr;
}
const void *cluster_fn(int storage, int vpt, int rg)
{
    if (vpt > map_vpt_limit(storage))
        return nullptr;
    switch (storage) {
    case NSLI_F64: return cluster_fn_s<NSLI_F64>(vpt, rg);
    case NSLI_F32: return cluster_fn_s<NSLI_F32>(vpt, rg);
    case NSLI_BF16: return cluster_fn_s<NSLI_BF16>(vpt, rg);
    case NSLI_FP8E4M3: return cluster_fn_s<NSLI_FP8E4M3>(vpt, rg);
    default: return nullptr;
    }
}

template <int S, int RG, bool SY> const void *long_fn_rg() { return (const void *)map_long_kernel<S, RG, SY>; }
template <int S> const void *long_fn_s(int rg, bool sy)
{
    if (sy)
        return rg == 4 ? long_fn_rg<S, 4, true>() : (rg == 2 ? long_fn_rg<S, 2, true>() : long_fn_rg<S, 1, true>());
    return rg == 4 ? long_fn_rg<S, 4, false>() : (rg == 2 ? long_fn_rg<S, 2, false>() : long_fn_rg<S, 1, false>());
}
// the long-row instance for a storage type, rows per group and y placement
const void *long_fn(int storage, int rg, bool sy)
{
    if (rg != 1 && rg != 2 && rg != 4)
        return nullptr;
    switch (storage) {
    case NSLI_F64: return long_fn_s<NSLI_F64>(rg, sy);
    case NSLI_F32: return long_fn_s<NSLI_F32>(rg, sy);
    case NSLI_BF16: return long_fn_s<NSLI_BF16>(rg, sy);
    case NSLI_FP8E4M3: return long_fn_s<NSLI_FP8E4M3>(rg, sy);
    default: return nullptr;
    }
}

// ---------------------------------------------------- reduce and update ----
//
// Block = 256 threads = 8 groups x 32 columns.  Group q sums partial rows
// g = q, q + 8, ... of its column in the accumulation type, and the 8 group
// sums are added in binary64: in order 0..7 for binary32 storage; for
// binary64 storage, whose dependent operations are slow on GB300, as four
// running sums per group and trees.  Every block recomputes h and the maxima
// from the per-CTA records (exact integer sum / exact maxima), so all blocks
// take the same decision.  The last block to finish (ticket) completes the
// step.
template <int NGRP> struct ReduceSharedT {
    double part[NGRP][32];
    double red[NGRP];
    long long h;
    double mv, mn, mb;
    int last;
};
using ReduceShared = ReduceSharedT<8>;

__device__ __forceinline__ unsigned long long red_ord_enc(double d)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double red_ord_dec(unsigned long long u)
{
    const unsigned long long bits = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
    return __longlong_as_double((long long)bits);
}

// Barrier of the threads that run one reduce item: the whole block
// (bar_id < 0) or the named barrier bar_id of nthr threads.
__device__ __forceinline__ void sub_sync(int bar_id, int nthr)
{
    if (bar_id < 0)
        __syncthreads();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(nthr) : "memory");
}

template <typename SH>
__device__ __forceinline__ void reduce_stats(const PartStat *ps, int G, SH &sh, int tid = threadIdx.x)
{
    const int lane = tid & 31;
    // maxima as order-preserving integers: exact, and no binary64 compare
    // (a long dependency chain on GB300) on the way
    if (tid < 32) {
        long long h = 0;
        unsigned long long mv = red_ord_enc(-INFINITY), mn = mv, mb = red_ord_enc(0.0);
#pragma unroll 4
        for (int g = lane; g < G; g += 32) {
            const PartStat q = ps[g];
            h += q.h;
            mv = max(mv, red_ord_enc(q.maxviol));
            mn = max(mn, red_ord_enc(q.maxnorm));
            mb = max(mb, red_ord_enc(q.maxb));
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            h += __shfl_xor_sync(0xffffffffu, h, off);
            mv = max(mv, __shfl_xor_sync(0xffffffffu, mv, off));
            mn = max(mn, __shfl_xor_sync(0xffffffffu, mn, off));
            mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, off));
        }
        if (lane == 0) {
            sh.h = h;
            sh.mv = red_ord_dec(mv);
            sh.mn = red_ord_dec(mn);
            sh.mb = red_ord_dec(mb);
        }
    }
}

// Column block `blk` of `nblk` of one problem's reduce-and-step, by a block
// of NGRP warps (NGRP groups of partial rows per column: 8 in the
// reduce kernels, 16 in the persistent serving kernel).
template <typename Acc, int NGRP = 8>
__device__ __forceinline__ void reduce_body(const ReduceArgs &p, const int blk, const int nblk,
                                            ReduceSharedT<NGRP> &sh, const int tid, const int bar_id)
{
    // tid / bar_id: the thread's index within the NGRP warps that run this
    // item and their barrier (-1: the whole block; else the named barrier
    // bar_id of NGRP * 32 threads)
    const int nthr = NGRP * 32;
    DevState *st = p.st;
    if (*(volatile int *)&st->done)
        return;
    const int lane = tid & 31, grp = tid >> 5;
    reduce_stats(p.part_stat, p.G, sh, tid);
    sub_sync(bar_id, nthr);
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
    const long long j = (long long)blk * kReduceCols + lane;

    if (step) {
        double yj = 0.0;
        if (j < p.ld) {
            const Acc *py = static_cast<const Acc *>(p.part_y);
            // the partial rows g = grp, grp + NGRP, ... added in that order
            // in the accumulation type (binary64 is slow on this part), the
            // NGRP group sums then in binary64
            if constexpr (sizeof(Acc) == 8) {
                // binary64: four running sums (g = grp + NGRP (4c + u)),
                // added in a tree; a dependent binary64 add costs ~435
                // cycles here
                double a[4] = {0.0, 0.0, 0.0, 0.0};
                for (int g = grp; g < p.G; g += 4 * NGRP) {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (g + NGRP * u < p.G)
                            a[u] += py[(long long)(g + NGRP * u) * p.ld + j];
                }
                yj = (a[0] + a[1]) + (a[2] + a[3]);
            } else {
                Acc t = Acc(0);
#pragma unroll 8
                for (int g = grp; g < p.G; g += NGRP)
                    t += py[(long long)g * p.ld + j];
                yj = (double)t;
            }
        }
        sh.part[grp][lane] = yj;
    }
    sub_sync(bar_id, nthr);
    if (step && grp == 0) {
        // the NGRP group sums added pairwise (adjacent pairs, log2 NGRP
        // levels): a chain of dependent binary64 adds costs ~435 cycles a
        // link on this part
        static_assert((NGRP & (NGRP - 1)) == 0, "a power-of-two number of groups");
        double v[NGRP];
#pragma unroll
        for (int q = 0; q < NGRP; ++q)
            v[q] = sh.part[q][lane];
#pragma unroll
        for (int w = NGRP / 2; w >= 1; w /= 2) {
#pragma unroll
            for (int q = 0; q < w; ++q)
                v[q] = v[2 * q] + v[2 * q + 1];
        }
        const double y = v[0];
        double val = 0.0;
        if (j < p.ld) {
            if (rule == NSLI_RULE_MODAP) {
                p.ybuf[j] = y;
                val = y * y;
            } else {
                const double s = h > 0 ? (p.rtab ? __ldg(p.rtab + h) : lambda / (double)h) : 0.0;
                const double xo = p.x64[j];
                const double xn = xo - s * y;
                p.x64[j] = xn;
                static_cast<Acc *>(p.x)[j] = (Acc)xn;
                const double d = xn - xo;
                val = d * d;
            }
        }
        val = warp_sum(val);
        if (lane == 0)
            p.part_dx[blk] = val;
    }
    __threadfence();
    sub_sync(bar_id, nthr);
    if (tid == 0) {
        const unsigned int t = atomicAdd(&st->ticket, 1u);
        sh.last = (t == (unsigned int)nblk - 1) ? 1 : 0;
    }
    sub_sync(bar_id, nthr);
    if (!sh.last)
        return;
    __threadfence();

    double dx2 = 0.0, ynorm = 0.0;
    if (step) {
        if (grp == 0) {
            // four running sums per lane (blocks q = lane + 32 (4c + u)),
            // added pairwise: a quarter of the dependent binary64 adds
            double v4[4] = {0.0, 0.0, 0.0, 0.0};
            for (int q = lane; q < nblk; q += 128) {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (q + 32 * u < nblk)
                        v4[u] += __ldcg(p.part_dx + q + 32 * u);
            }
            double v = (v4[0] + v4[1]) + (v4[2] + v4[3]);
            v = warp_sum(v);
            if (lane == 0)
                sh.red[0] = v;
        }
        sub_sync(bar_id, nthr);
        const double tot = sh.red[0];
        if (rule == NSLI_RULE_MODAP) {
            ynorm = sqrt(tot);
            const double s = ynorm > 0.0 ? lambda / ynorm : 0.0;
            Acc *x = static_cast<Acc *>(p.x);
            double v = 0.0;
            for (long long q = tid; q < p.ld; q += nthr) {
                const double xo = p.x64[q];
                const double xn = xo - s * __ldcg(p.ybuf + q);
                p.x64[q] = xn;
                x[q] = (Acc)xn;
                const double d = xn - xo;
                v += d * d;
            }
            v = warp_sum(v);
            sub_sync(bar_id, nthr);
            if (lane == 0)
                sh.red[grp] = v;
            sub_sync(bar_id, nthr);
            double t = 0.0;
            for (int q = 0; q < NGRP; ++q)
                t += sh.red[q];
            dx2 = t;
        } else {
            dx2 = tot;
        }
    }
    if (tid == 0) {
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

template <typename Acc>
__global__ void __launch_bounds__(256) reduce_update_kernel(const ReduceArgs p)
{
    __shared__ ReduceShared sh;
    reduce_body<Acc>(p, blockIdx.x, gridDim.x, sh, threadIdx.x, -1);
}

// Many problems in one launch: block b serves (problem, column block) tab[b].
template <typename Acc>
__global__ void __launch_bounds__(256) reduce_group_kernel(const GroupProblem *probs, const GroupRed *tab)
{
    __shared__ ReduceShared sh;
    const GroupRed t = tab[blockIdx.x];
    const GroupProblem &gp = probs[t.prob];
    reduce_body<Acc>(gp.red, t.blk, gp.red_blocks, sh, threadIdx.x, -1);
}

// Map + Reduce without a step (diagnostics and parity): y in binary64.
template <typename Acc>
__global__ void __launch_bounds__(256) reduce_only_kernel(const ReduceArgs p, double *y_out)
{
    __shared__ ReduceShared sh;
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const long long j = (long long)blockIdx.x * kReduceCols + lane;
    double yj = 0.0;
    if (j < p.ld) {
        const Acc *py = static_cast<const Acc *>(p.part_y);
        Acc t = Acc(0);
#pragma unroll 8
        for (int g = grp; g < p.G; g += 8)
            t += py[(long long)g * p.ld + j];
        yj = (double)t;
    }
    sh.part[grp][lane] = yj;
    __syncthreads();
    if (grp == 0 && j < p.ld) {
        double y = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            y += sh.part[q][lane];
        y_out[j] = y;
    }
    if (blockIdx.x == 0) {
        reduce_stats(p.part_stat, p.G, sh);
        __syncthreads();
        if (threadIdx.x == 0) {
            p.st->h = sh.h;
            p.st->maxviol = sh.mv;
            p.st->maxnorm = sh.mn;
            p.st->maxb = sh.mb;
        }
    }
}

// ------------------------------------------------- persistent serving ----
//
// One cooperative launch (every CTA resident, one per SM) iterates all live
// problems of a pool round after round:
//   control   CTA 0: wall-clock ticks, problems that stopped in the last
//             round go to the host-mapped completion list, the stop decision
//             (host yield, nothing left running, round or time bound);
//   Map       CTAs take the work items (a block of rows of one problem)
//             i = blockIdx.x, blockIdx.x + grid, ...;
//   Reduce    the same for the (problem, column block) items;
// with a grid barrier after each phase.  A problem's items and their
// arithmetic are those of the grouped launches, so its iterates do not
// depend on the other problems or on which CTA ran which item.  Every
// barrier wait is bounded: on expiry the CTA records the error and returns
// (the others then expire too).

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The serving kernel keeps its few shared words in the tail of the Map
// ring's header (free for a binary32 accumulator: the barriers and warp sums
// end at byte 1280), and the reduce's shared block in the ring's stages
// (idle during the Reduce phase), so it needs no shared memory beyond the
// largest ring of its problems.
constexpr int kServeRedGrp = 2;   // warps per serving reduce item
constexpr int kServeRedSub = 8;   // reduce items in flight per CTA
struct ServeShared {
    unsigned long long t_start;
    int ok, running;
    int item;    // the work item the CTA took
};
constexpr int kServeSharedOffset = 2304;
static_assert(kServeSharedOffset + sizeof(ServeShared) <= kSmemHeader, "serving words fit the ring header");
static_assert(256 + 2 * 1024 <= kServeSharedOffset, "ring header layout: barriers, warp sums, serving words");
__device__ __forceinline__ ServeShared &serve_shared()
{
    extern __shared__ __align__(128) unsigned char smem[];
    return *reinterpret_cast<ServeShared *>(smem + kServeSharedOffset);
}

// Grid barrier over nblocks resident CTAs: sense by generation count.
__device__ __forceinline__ bool serve_grid_sync(ServeSync *sy, unsigned int nblocks)
{
    int &ok = serve_shared().ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *gen = &sy->bar_gen;
        const unsigned int g = *gen;          // before arriving
        __threadfence();
        const unsigned int arrived = atomicAdd(&sy->bar_count, 1u) + 1u;
        int good = 1;
        if (arrived == nblocks) {
            atomicExch(&sy->bar_count, 0u);   // reset before the release
            __threadfence();
            atomicAdd(&sy->bar_gen, 1u);
        } else {
            const long long t0 = clock64();
            for (unsigned int it = 0; *gen == g; ++it) {
                if ((it & 63u) == 63u && clock64() - t0 > kWaitLimitCycles) {
                    good = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// Control phase (CTA 0).
__device__ __forceinline__ void serve_control(const ServeArgs &a, long long round, unsigned long long t_start)
{
    int &running = serve_shared().running;
    if (threadIdx.x == 0)
        running = 0;
    __syncthreads();
    const unsigned long long now = global_ns();
    int mine = 0;
    for (int q = threadIdx.x; q < a.nprob; q += blockDim.x) {
        DevState *st = a.probs[q].red.st;
        if (round == 0) {
            a.tick0[q] = st->tick;
            a.reported[q] = *(volatile int *)&st->done;   // stopped before this launch
        }
        const int done = *(volatile int *)&st->done;
        if (done && !a.reported[q]) {
            a.reported[q] = 1;
            const unsigned int k = atomicAdd(&a.sync->ndone, 1u);
            if (k < (unsigned int)kServeMaxProblems) {
                ServeDone d;
                d.prob = q;
                d.status = st->status;
                d.it = st->it;
                a.ctrl->done[k] = d;
            }
        }
        if (!done) {
            ++mine;
            if (a.tick_ns > 0)
                st->tick = a.tick0[q] + (long long)((now - t_start) / a.tick_ns);
        }
    }
    if (mine)
        atomicAdd(&running, mine);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence_system();
        *(volatile unsigned int *)&a.ctrl->done_count = a.sync->ndone;
        *(volatile unsigned long long *)&a.ctrl->rounds = (unsigned long long)round;
        const int yield = *(volatile int *)&a.ctrl->yield;
        a.sync->stop = (yield || running == 0 || round >= a.max_rounds || now - t_start > a.max_ns) ? 1 : 0;
        a.sync->map_next = 0u;   // every CTA has left the previous round's phases
        a.sync->red_next = 0u;
        __threadfence_system();
    }
}

template <int S, int V>
__device__ __forceinline__ void serve_map_item(const GroupProblem &gp, const GroupItem &it,
                                               typename Traits<S>::acc *prow, PartStat *pst)
{
    if (gp.nt == (int)blockDim.x && gp.nt * gp.vpt == gp.map.nv && gp.vpt == V)
        map_body<S, V, false, false>(gp.map, it.row_begin, it.row_end, prow, pst, gp.nt, V);
    else
        map_body<S, V, true, true>(gp.map, it.row_begin, it.row_end, prow, pst, gp.nt, gp.vpt);
}

template <int S, int VPT>
__global__ void __launch_bounds__(kMapMaxConsumers, 1) serve_kernel(const ServeArgs a)
{
    using Acc = typename Traits<S>::acc;
    static_assert(sizeof(Acc) == 4, "the serving kernel keeps its words in a binary32 ring header");
    // Reduce items run kServeRedSub at a time per CTA, each on its own
    // kServeRedGrp warps (their own named barrier and shared block, placed
    // in the ring's stages, free in that phase): an item is a chain of
    // dependent global-memory round trips, and several in flight overlap
    constexpr int NGRP = kServeRedGrp;
    constexpr int NSUB = kMapMaxConsumers / (32 * NGRP);
    static_assert(NSUB == kServeRedSub, "reduce sub-blocks tile the CTA");
    extern __shared__ __align__(128) unsigned char smem[];
    const int sub = threadIdx.x / (32 * NGRP), stid = threadIdx.x % (32 * NGRP);
    ReduceSharedT<NGRP> &rsh = reinterpret_cast<ReduceSharedT<NGRP> *>(smem + kSmemHeader)[sub];
    int *sub_item = reinterpret_cast<int *>(smem + kSmemHeader + NSUB * sizeof(ReduceSharedT<NGRP>));
    ServeShared &ss = serve_shared();
    if (threadIdx.x == 0)
        ss.t_start = global_ns();
    __syncthreads();
    const unsigned long long t_start = ss.t_start;
    const unsigned int G = gridDim.x;
    for (long long round = 0;; ++round) {
        if (blockIdx.x == 0)
            serve_control(a, round, t_start);
        if (!serve_grid_sync(a.sync, G))
            break;
        if (*(volatile int *)&a.sync->stop)
            break;
        // items are taken one at a time from a shared counter (an item's
        // arithmetic does not depend on the CTA that runs it)
        for (;;) {
            if (threadIdx.x == 0)
                ss.item = (int)atomicAdd(&a.sync->map_next, 1u);
            __syncthreads();
            const int i = ss.item;
            if (i >= a.nitems)
                break;
            const GroupItem it = a.items[i];
            const GroupProblem &gp = a.probs[it.prob];
            if (!*(volatile int *)&gp.map.st->done) {
                Acc *prow = static_cast<Acc *>(gp.map.part_y) + (long long)it.part * gp.map.ld;
                PartStat *pst = gp.map.part_stat + it.part;
                // the instance of the problem's own vectors per thread (its
                // rows per block barrier), guard-free when the block covers
                // the row exactly
                if (gp.vpt == 1)
                    serve_map_item<S, 1>(gp, it, prow, pst);
                else if (gp.vpt == 2)
                    serve_map_item<S, 2>(gp, it, prow, pst);
                else if (gp.vpt == 4 || VPT < 8)
                    serve_map_item<S, (VPT < 4 ? VPT : 4)>(gp, it, prow, pst);
                else
                    serve_map_item<S, VPT>(gp, it, prow, pst);
            }
            __syncthreads();   // every warp has left the ring before it is armed again
        }
        if (!serve_grid_sync(a.sync, G))
            break;
        for (;;) {
            if (stid == 0)
                sub_item[sub] = (int)atomicAdd(&a.sync->red_next, 1u);
            sub_sync(1 + sub, 32 * NGRP);
            const int i = sub_item[sub];
            if (i >= a.nreds)
                break;
            const GroupRed t = a.reds[i];
            const GroupProblem &gp = a.probs[t.prob];
            reduce_body<Acc, NGRP>(gp.red, t.blk, gp.red_blocks, rsh, stid, 1 + sub);
            sub_sync(1 + sub, 32 * NGRP);   // the item's shared words are free again
        }
        __syncthreads();
        if (!serve_grid_sync(a.sync, G))
            break;
    }
    if (threadIdx.x == 0 && *(volatile int *)&a.sync->stop == 0) {
        // left on an expired barrier wait
        atomicOr(&a.ctrl->error, 1);
        __threadfence_system();
    }
}

// ------------------------------------------------------- binary64 check ----

__device__ __forceinline__ unsigned long long ord_enc(double d)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// One warp per row: r_i = sum_j a_ij x_j - (b0_i + (k rho) Av_i) with binary64
// products and sums on the stored entries; maxima by order-preserving
// integer atomics (exact, so the result does not depend on the schedule).
template <int S>
__global__ void __launch_bounds__(256) verify_kernel(const VerifyArgs p)
{
    using Tr = Traits<S>;
    using Acc = typename Tr::acc;
    constexpr int EPV = Tr::EPV;
    const int lane = threadIdx.x & 31;
    const long long wg = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const double kr = __dmul_rn((double)p.st->tick, p.st->rho);
    const double *x = p.x64;
    const long long row_bytes = (long long)p.nv * 16;
    double mv = -INFINITY, mn = -INFINITY, mb = 0.0;
    unsigned long long h = 0;
    for (long long i = wg; i < p.m; i += nw) {
        const uint4 *row = reinterpret_cast<const uint4 *>(static_cast<const unsigned char *>(p.A) + i * row_bytes);
        double s = 0.0;
        for (int j = lane; j < p.nv; j += 32) {
            Acc a[EPV];
            decode<S>(__ldg(row + j), a);
#pragma unroll
            for (int e = 0; e < EPV; ++e)
                s = fma((double)a[e], x[(long long)j * EPV + e], s);
        }
        s = warp_sum(s);
        if (S == NSLI_FP8E4M3)
            s = s * (double)p.scale[i];
        const double bi = __dadd_rn(p.b0_64[i], __dmul_rn(kr, p.av_64[i]));
        const double ri = s - bi;
        mv = fmax(mv, ri);
        mn = fmax(mn, ri / sqrt(p.n2_64[i]));
        mb = fmax(mb, fabs(bi));
        h += (ri > 0.0) ? 1ull : 0ull;
    }
    if (lane == 0) {
        atomicMax(&p.out->maxviol, ord_enc(mv));
        atomicMax(&p.out->maxnorm, ord_enc(mn));
        atomicMax(&p.out->maxb, ord_enc(mb));
        atomicAdd(&p.out->h, h);
    }
}

// ---------------------------------------------------------------- set-up ----

// One block per row: optional FP8 row scale, store the row in the storage
// type (zero padding up to ld), binary64 ||a_i||^2 of the STORED values in a
// fixed order, finiteness and zero-row flags.
template <int S>
__global__ void __launch_bounds__(256) prep_kernel(const PrepArgs p)
{
    const long long r = blockIdx.x;
    if (r >= p.rows)
        return;
    const long long gi = p.row0 + r;
    __shared__ double sred[8];
    __shared__ float samax[8];
    __shared__ int sbad;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0)
        sbad = 0;
    __syncthreads();
    const float *s32 = static_cast<const float *>(p.src) + r * p.lda;
    const double *s64 = static_cast<const double *>(p.src) + r * p.lda;
    int bad = 0;

    float scale = 1.0f, inv_scale = 1.0f;
    if (S == NSLI_FP8E4M3) {
        float amax = 0.0f;
        for (long long j = threadIdx.x; j < p.n; j += blockDim.x) {
            const float a = s32[j];
            if (!isfinite(a))
                bad = 1;
            amax = fmaxf(amax, fabsf(a));
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
        if (lane == 0)
            samax[wid] = amax;
        __syncthreads();
        amax = 0.0f;
        for (int q = 0; q < 8; ++q)
            amax = fmaxf(amax, samax[q]);
        int e = 0;
        if (amax > 0.0f && isfinite(amax)) {
            int e2;
            const float f = frexpf(amax, &e2);  // amax = f 2^e2, f in [0.5, 1)
            e = (f <= 0.875f) ? e2 - 9 : e2 - 8;  // smallest 2^e with amax / 2^e <= 448
        }
        scale = ldexpf(1.0f, e);
        inv_scale = ldexpf(1.0f, -e);
        if (threadIdx.x == 0)
            p.scale[gi] = scale;
    }

    // ||a_i||^2 of the stored values: binary64 for binary64 storage, else the
    // double-float accumulation of nsli_sumsq.cuh, folded into binary64 every
    // 8 entries (fast = 0: the binary64 norms) or not at all (fast = 1: the
    // norm behind the row records, as in the row-update kernel), and the
    // block total of sumsq_block_total
    double n2 = 0.0;
    SumSq sq = sumsq_init();
    for (long long j = threadIdx.x; j < p.ld; j += blockDim.x) {
        const bool in = j < p.n;
        if (S == NSLI_F64) {
            const double v = in ? (p.src_f64 ? s64[j] : (double)s32[j]) : 0.0;
            if (in && !isfinite(v))
                bad = 1;
            static_cast<double *>(p.A)[gi * p.ld + j] = v;
            n2 += v * v;
        } else if (S == NSLI_F32) {
            const float v = in ? (p.src_f64 ? __double2float_rn(s64[j]) : s32[j]) : 0.0f;
            if (in && !(p.src_f64 ? isfinite(s64[j]) : isfinite(v)))
                bad = 1;
            static_cast<float *>(p.A)[gi * p.ld + j] = v;
            if (in && isfinite(v))
                p.fast ? sumsq_add<0>(sq, v) : sumsq_add<8>(sq, v);
        } else if (S == NSLI_BF16) {
            const float a = in ? s32[j] : 0.0f;
            if (in && !isfinite(a))
                bad = 1;
            // (a value that rounds to infinity makes the norm infinite and
            // the row invalid, as in the row-update kernel)
            const __nv_bfloat16 q = __float2bfloat16_rn(a);
            static_cast<__nv_bfloat16 *>(p.A)[gi * p.ld + j] = q;
            const float v = __bfloat162float(q);
            if (in)
                p.fast ? sumsq_add<0>(sq, v) : sumsq_add<8>(sq, v);
        } else {
            const float a = in ? s32[j] : 0.0f;
            const __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(a * inv_scale, __NV_SATFINITE, __NV_E4M3);
            static_cast<unsigned char *>(p.A)[gi * p.ld + j] = (unsigned char)q;
            const __half_raw hr = __nv_cvt_fp8_to_halfraw(q, __NV_E4M3);
            const float v = __fmul_rn(__half2float(__half(hr)), scale);   // exact: scale is a power of two
            if (in)
                p.fast ? sumsq_add<0>(sq, v) : sumsq_add<8>(sq, v);
        }
    }
    if (bad)
        sbad = 1;
    double t = 0.0;   // the row total, in thread 0
    if constexpr (S != NSLI_F64) {
        __shared__ float2 spair[8];
        __shared__ double sacc[8];
        t = sumsq_block_total<8>(sq, spair, sacc);   // (synchronises the block)
    } else {
        n2 = warp_sum(n2);
        if (lane == 0)
            sred[wid] = n2;
        __syncthreads();
        if (threadIdx.x == 0)
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q)
                t += sred[q];
    }
    if (threadIdx.x == 0) {
        if (p.norms_in != nullptr)
            t = p.norms_in[gi];
        p.n2_64[gi] = t;
        int f = 0;
        if (sbad || !isfinite(t))
            f |= PREPF_NONFINITE;
        if (t == 0.0)
            f |= PREPF_ZERO_ROW;
        if (f)
            atomicOr(p.flags, f);
    }
}

template <bool F64>
__global__ void __launch_bounds__(256) meta_kernel(const MetaArgs p)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= p.m)
        return;
    const long long i = p.row0 + k;
    const double b0 = p.b0_64[i];
    const double av = p.av_64[i];
    const double n2 = p.n2_64[i];
    if (!isfinite(b0) || !isfinite(av))
        atomicOr(p.flags, PREPF_NONFINITE);
    const double inv_n2 = 1.0 / n2;
    const double inv_n = 1.0 / sqrt(n2);
    if (F64) {
        RowMeta64 m{b0, av, inv_n2, inv_n};
        static_cast<RowMeta64 *>(p.meta)[i] = m;
    } else {
        RowMeta32 m{(float)b0, (float)av, (float)inv_n2, (float)inv_n,
                    p.scale ? p.scale[i] : 1.0f, 0.0f, 0.0f, 0.0f};
        static_cast<RowMeta32 *>(p.meta)[i] = m;
    }
}

// Only the b0 field of rows [row0, row0 + m): a new right-hand side leaves
// the norms, Av and the FP8 scale as they are, and the field gets the value
// meta_kernel would give it (no binary64 divide or root per row).
template <bool F64> __global__ void __launch_bounds__(256) meta_b0_kernel(const MetaArgs p)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= p.m)
        return;
    const long long i = p.row0 + k;
    const double b0 = p.b0_64[i];
    if (!isfinite(b0))
        atomicOr(p.flags, PREPF_NONFINITE);
    if (F64)
        static_cast<RowMeta64 *>(p.meta)[i].b0 = b0;
    else
        static_cast<RowMeta32 *>(p.meta)[i].b0 = (float)b0;
}

template <typename Acc>
__global__ void x_from_f64_kernel(const double *src, double *x64, Acc *x, long long n, long long ld, int *flags)
{
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ld)
        return;
    double v = 0.0;
    if (j < n) {
        v = src[j];
        if (!isfinite(v))
            atomicOr(flags, PREPF_NONFINITE);
    }
    x64[j] = v;
    x[j] = (Acc)v;
}

__global__ void check_finite_kernel(const double *v, long long n, int *flags)
{
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n && !isfinite(v[j]))
        atomicOr(flags, PREPF_NONFINITE);
}

// Run parameters into the state (block 0, thread 0) and, when the step size
// changed, the table lambda / h that the step reads instead of dividing (a
// binary64 division is a long dependency chain on GB300).
__global__ void state_begin_kernel(DevState *st, const StateBegin b)
{
    if (b.rtab) {
        for (long long h = (long long)blockIdx.x * blockDim.x + threadIdx.x; h <= b.rtab_m;
             h += (long long)gridDim.x * blockDim.x)
            b.rtab[h] = h > 0 ? b.lambda / (double)h : 0.0;
    }
    if (blockIdx.x != 0 || threadIdx.x != 0)
        return;
    st->lambda = b.lambda;
    st->eps = b.eps;
    st->rho = b.rho;
    st->max_iter = b.max_iter;
    st->rule = b.rule;
    st->stop = b.stop;
    st->force_step = b.force_step;
    if (b.reset_it)
        st->it = 0;
    if (b.tick >= 0)
        st->tick = b.tick;
    st->done = 0;
    st->status = ST_RUNNING;
    st->error = 0;
    st->ticket = 0u;
}

__global__ void set_ticks_kernel(DevState *const *sts, const long long *ticks, int count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) {
        sts[i]->tick = ticks[i];
        sts[i]->hold_tick = 1;
    }
}

__global__ void state_resume_kernel(DevState *st)
{
    st->done = 0;
    st->status = ST_RUNNING;
    st->force_step = 1;
}

// Exact values of stored rows as binary64 (diagnostics).
template <int S>
__global__ void stored_rows_kernel(const void *A, const float *scale, long long ld, long long n, long long row0,
                                   long long rows, double *out)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * n)
        return;
    const long long r = t / n, j = t % n;
    const long long i = row0 + r;
    double v;
    if (S == NSLI_F64) {
        v = static_cast<const double *>(A)[i * ld + j];
    } else if (S == NSLI_F32) {
        v = (double)static_cast<const float *>(A)[i * ld + j];
    } else if (S == NSLI_BF16) {
        v = (double)__bfloat162float(static_cast<const __nv_bfloat16 *>(A)[i * ld + j]);
    } else {
        const __nv_fp8_storage_t q = static_cast<const unsigned char *>(A)[i * ld + j];
        const __half_raw hr = __nv_cvt_fp8_to_halfraw(q, __NV_E4M3);
        v = (double)__half2float(__half(hr)) * (double)scale[i];
    }
    out[t] = v;
}

// ------------------------------------------------------------- launchers ----

int map_vpt_limit(int storage)
{
    switch (storage) {
    case NSLI_F64: return 8;
    case NSLI_F32: return 8;
    case NSLI_BF16: return 4;
    case NSLI_FP8E4M3: return 2;
    default: return 0;
    }
}

template <int S, bool G> static const void *map_fn(int vpt)
{
    switch (vpt) {
    case 1: return (const void *)map_kernel<S, 1, G>;
    case 2: return (const void *)map_kernel<S, 2, G>;
    case 4:
        if constexpr (S != NSLI_FP8E4M3)
            return (const void *)map_kernel<S, 4, G>;
        return nullptr;
    case 8:
        if constexpr (S == NSLI_F64 || S == NSLI_F32)
            return (const void *)map_kernel<S, 8, G>;
        return nullptr;
    default: return nullptr;
    }
}

static const void *map_fn_any(int storage, int vpt, bool guard)
{
    switch (storage) {
    case NSLI_F64: return guard ? map_fn<NSLI_F64, true>(vpt) : map_fn<NSLI_F64, false>(vpt);
    case NSLI_F32: return guard ? map_fn<NSLI_F32, true>(vpt) : map_fn<NSLI_F32, false>(vpt);
    case NSLI_BF16: return guard ? map_fn<NSLI_BF16, true>(vpt) : map_fn<NSLI_BF16, false>(vpt);
    case NSLI_FP8E4M3: return guard ? map_fn<NSLI_FP8E4M3, true>(vpt) : map_fn<NSLI_FP8E4M3, false>(vpt);
    default: return nullptr;
    }
}

cudaError_t map_prepare(int storage, int vpt, bool guard, size_t smem)
{
    if (vpt == 0) {
        // long rows: partial sums in shared memory for every group size
        if (smem == 0)
            return cudaSuccess;
        for (int rg = 1; rg <= 4; rg *= 2) {
            const void *fn = long_fn(storage, rg, true);
            if (!fn)
                return cudaErrorInvalidValue;
            cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess)
                return e;
        }
        return cudaSuccess;
    }
    const void *fn = map_fn_any(storage, vpt, guard);
    if (!fn)
        return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t cluster_prepare(int storage, int vpt, int rg, int C, size_t smem, int *clusters)
{
    *clusters = 0;
    const void *fn = cluster_fn(storage, vpt, rg);
    if (!fn || C < 2 || C > 8)
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(clusters, fn, &cfg);
}

cudaError_t map_launch(int storage, int vpt, bool guard, int grid, int consumers, size_t smem, cudaStream_t s,
                       const MapArgs &a)
{
    if (vpt == 0 && a.cluster > 1) {
        // long rows on clusters: `grid` clusters of a.cluster CTAs
        const void *fn = cluster_fn(storage, a.cluster_vpt, a.cluster_rg);
        if (!fn)
            return cudaErrorInvalidValue;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(grid * a.cluster));
        cfg.blockDim = dim3(kClusterThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)a.cluster;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        void *args[] = {const_cast<MapArgs *>(&a)};
        return cudaLaunchKernelExC(&cfg, fn, args);
    }
    if (vpt == 0) {
        // long rows: rows_per_slot carries the group size, smem the
        // partial-sum row in shared memory (0: in global memory)
        const void *fn = long_fn(storage, a.rows_per_slot, smem > 0);
        if (!fn)
            return cudaErrorInvalidValue;
        void *args[] = {const_cast<MapArgs *>(&a)};
        return cudaLaunchKernel(fn, dim3(grid), dim3(kLongThreads), args, smem, s);
    }
    const void *fn = map_fn_any(storage, vpt, guard);
    if (!fn)
        return cudaErrorInvalidValue;
    void *args[] = {const_cast<MapArgs *>(&a)};
    return cudaLaunchKernel(fn, dim3(grid), dim3(consumers), args, smem, s);
}

cudaError_t map_group_prepare(int storage, size_t smem)
{
    const void *fn = nullptr;
    if (storage == NSLI_BF16)
        fn = (const void *)map_group_kernel<NSLI_BF16, 4>;
    else if (storage == NSLI_F32)
        fn = (const void *)map_group_kernel<NSLI_F32, 8>;
    if (!fn)
        return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t map_group_launch(int storage, int items, size_t smem, cudaStream_t s, const GroupProblem *probs,
                             const GroupItem *it)
{
    if (storage == NSLI_BF16)
        map_group_kernel<NSLI_BF16, 4><<<items, kMapMaxConsumers, smem, s>>>(probs, it);
    else if (storage == NSLI_F32)
        map_group_kernel<NSLI_F32, 8><<<items, kMapMaxConsumers, smem, s>>>(probs, it);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

static const void *serve_fn(int storage)
{
    if (storage == NSLI_BF16)
        return (const void *)serve_kernel<NSLI_BF16, 4>;
    if (storage == NSLI_F32)
        return (const void *)serve_kernel<NSLI_F32, 8>;
    return nullptr;
}

cudaError_t serve_prepare(int storage, size_t smem, int *blocks_per_sm)
{
    const void *fn = serve_fn(storage);
    if (!fn)
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kMapMaxConsumers, smem);
}

cudaError_t serve_launch(int storage, int grid, size_t smem, cudaStream_t s, const ServeArgs &a)
{
    const void *fn = serve_fn(storage);
    if (!fn)
        return cudaErrorInvalidValue;
    void *args[] = {(void *)&a};
    return cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(kMapMaxConsumers), args, smem, s);
}

cudaError_t reduce_group_launch(bool f64, int blocks, cudaStream_t s, const GroupProblem *probs,
                                const GroupRed *tab)
{
    if (f64)
        reduce_group_kernel<double><<<blocks, 256, 0, s>>>(probs, tab);
    else
        reduce_group_kernel<float><<<blocks, 256, 0, s>>>(probs, tab);
    return cudaGetLastError();
}

cudaError_t reduce_launch(bool f64, int grid, cudaStream_t s, const ReduceArgs &a)
{
    if (f64)
        reduce_update_kernel<double><<<grid, 256, 0, s>>>(a);
    else
        reduce_update_kernel<float><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t reduce_only_launch(bool f64, int grid, cudaStream_t s, const ReduceArgs &a, double *y_out)
{
    if (f64)
        reduce_only_kernel<double><<<grid, 256, 0, s>>>(a, y_out);
    else
        reduce_only_kernel<float><<<grid, 256, 0, s>>>(a, y_out);
    return cudaGetLastError();
}

cudaError_t verify_launch(int storage, int grid, cudaStream_t s, const VerifyArgs &a)
{
    switch (storage) {
    case NSLI_F64: verify_kernel<NSLI_F64><<<grid, 256, 0, s>>>(a); break;
    case NSLI_F32: verify_kernel<NSLI_F32><<<grid, 256, 0, s>>>(a); break;
    case NSLI_BF16: verify_kernel<NSLI_BF16><<<grid, 256, 0, s>>>(a); break;
    case NSLI_FP8E4M3: verify_kernel<NSLI_FP8E4M3><<<grid, 256, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t prep_launch(int storage, cudaStream_t s, const PrepArgs &a)
{
    const unsigned int grid = (unsigned int)a.rows;
    switch (storage) {
    case NSLI_F64: prep_kernel<NSLI_F64><<<grid, 256, 0, s>>>(a); break;
    case NSLI_F32: prep_kernel<NSLI_F32><<<grid, 256, 0, s>>>(a); break;
    case NSLI_BF16: prep_kernel<NSLI_BF16><<<grid, 256, 0, s>>>(a); break;
    case NSLI_FP8E4M3: prep_kernel<NSLI_FP8E4M3><<<grid, 256, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t meta_b0_launch(bool f64, cudaStream_t s, const MetaArgs &a)
{
    if (a.m <= 0)
        return cudaSuccess;
    const unsigned int grid = (unsigned int)((a.m + 255) / 256);
    if (f64)
        meta_b0_kernel<true><<<grid, 256, 0, s>>>(a);
    else
        meta_b0_kernel<false><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t meta_launch(bool f64, cudaStream_t s, const MetaArgs &a)
{
    if (a.m <= 0)
        return cudaSuccess;
    const unsigned int grid = (unsigned int)((a.m + 255) / 256);
    if (f64)
        meta_kernel<true><<<grid, 256, 0, s>>>(a);
    else
        meta_kernel<false><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t x_from_f64_launch(bool f64, cudaStream_t s, const double *src, double *x64, void *x, long long n,
                              long long ld, int *flags)
{
    const unsigned int grid = (unsigned int)((ld + 255) / 256);
    if (f64)
        x_from_f64_kernel<double><<<grid, 256, 0, s>>>(src, x64, static_cast<double *>(x), n, ld, flags);
    else
        x_from_f64_kernel<float><<<grid, 256, 0, s>>>(src, x64, static_cast<float *>(x), n, ld, flags);
    return cudaGetLastError();
}

cudaError_t check_finite_launch(cudaStream_t s, const double *v, long long n, int *flags)
{
    const unsigned int grid = (unsigned int)((n + 255) / 256);
    check_finite_kernel<<<grid, 256, 0, s>>>(v, n, flags);
    return cudaGetLastError();
}

cudaError_t state_begin_launch(cudaStream_t s, DevState *st, const StateBegin &b)
{
    long long blocks = b.rtab ? (b.rtab_m + 256) / 256 : 1;
    if (blocks > 1024)
        blocks = 1024;
    state_begin_kernel<<<(unsigned)blocks, b.rtab ? 256 : 1, 0, s>>>(st, b);
    return cudaGetLastError();
}

cudaError_t set_ticks_launch(cudaStream_t s, DevState *const *sts, const long long *ticks, int count)
{
    set_ticks_kernel<<<(count + 127) / 128, 128, 0, s>>>(sts, ticks, count);
    return cudaGetLastError();
}

cudaError_t state_resume_launch(cudaStream_t s, DevState *st)
{
    state_resume_kernel<<<1, 1, 0, s>>>(st);
    return cudaGetLastError();
}

cudaError_t stored_rows_launch(int storage, cudaStream_t s, const void *A, const float *scale, long long ld,
                               long long n, long long row0, long long rows, double *out)
{
    const long long total = rows * n;
    const unsigned int grid = (unsigned int)((total + 255) / 256);
    switch (storage) {
    case NSLI_F64: stored_rows_kernel<NSLI_F64><<<grid, 256, 0, s>>>(A, scale, ld, n, row0, rows, out); break;
    case NSLI_F32: stored_rows_kernel<NSLI_F32><<<grid, 256, 0, s>>>(A, scale, ld, n, row0, rows, out); break;
    case NSLI_BF16: stored_rows_kernel<NSLI_BF16><<<grid, 256, 0, s>>>(A, scale, ld, n, row0, rows, out); break;
    case NSLI_FP8E4M3:
        stored_rows_kernel<NSLI_FP8E4M3><<<grid, 256, 0, s>>>(A, scale, ld, n, row0, rows, out);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace nsli
