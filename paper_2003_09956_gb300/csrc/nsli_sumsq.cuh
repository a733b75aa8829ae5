// nsli_sumsq.cuh -- ||a_i||^2 of stored rows with little binary64 work.
//
// GB300 executes binary64 at a small fraction of its binary32 rate, and a
// plain binary64 sum of squares (one conversion and one binary64 FMA per
// entry) bounds the set-up and row-update kernels.  Every stored value of a
// binary32 / bf16 / FP8 row is a binary32 number, so each thread instead
// keeps an unevaluated pair s + c of binary32 numbers ("double-float"):
//   v^2 = p + e exactly (p = fl(v v), e = fma(v, v, -p)),
//   s + p = t + err exactly (two-sum),
//   c += err + e, then (s, c) = fast-two-sum(t, c), so |c| <= ulp(s) / 2.
// Every 8 entries the pair is added to a binary64 accumulator (two binary64
// additions for 8 entries instead of 16 operations).  The pair carries about
// 48 significant bits, so each group of 8 is summed to within a few units of
// 2^-48 relative and the result agrees with a binary64 sum to about 1e-14.
// Without the periodic fold (FOLD = 0) the pair carries the whole per-thread
// sum: no binary64 work per entry, and sumsq_block_total adds the pairs of a
// block as double-floats and converts the row total once.
// Values whose square could leave the binary32 normal range (|v| outside
// [2^-60, 2^60]) are squared and added in binary64 directly.  The order is
// fixed per thread, so the set-up kernel and the row-update kernel, which
// both use this, give identical norms for identical rows.  Every operation is
// an explicit round-to-nearest intrinsic so no multiply-add is contracted.
#pragma once

#include <cuda_runtime.h>

namespace nsli {

struct SumSq {
    double acc;
    float s, c;
    int k;
};

__device__ __forceinline__ SumSq sumsq_init()
{
    SumSq q;
    q.acc = 0.0;
    q.s = 0.0f;
    q.c = 0.0f;
    q.k = 0;
    return q;
}

__device__ __forceinline__ void sumsq_flush(SumSq &q)
{
    q.acc = __dadd_rn(q.acc, (double)q.s);
    q.acc = __dadd_rn(q.acc, (double)q.c);
    q.s = 0.0f;
    q.c = 0.0f;
    q.k = 0;
}

// FOLD = 8: fold into binary64 every 8 entries (accurate to ~1e-14: the
// binary64 norms); FOLD = 0: never until the end (no binary64 work per
// entry; accurate to ~1e-12 for a few hundred entries per thread, which is
// ample for the binary32 row records).
template <int FOLD = 8> __device__ __forceinline__ void sumsq_add(SumSq &q, float v)
{
    const float a = fabsf(v);
    if (a == 0.0f)
        return;
    if (a < 0x1p-60f || a > 0x1p60f) {
        q.acc = __fma_rn((double)v, (double)v, q.acc);
        return;
    }
    const float p = __fmul_rn(v, v);
    const float e = __fmaf_rn(v, v, -p);          // p + e = v^2 exactly
    const float t = __fadd_rn(q.s, p);            // two-sum: s + p = t + err
    const float bp = __fsub_rn(t, q.s);
    const float err = __fadd_rn(__fsub_rn(q.s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    const float c = __fadd_rn(q.c, __fadd_rn(err, e));
    const float s2 = __fadd_rn(t, c);             // fast-two-sum (|t| >= |c|)
    q.c = __fsub_rn(c, __fsub_rn(s2, t));
    q.s = s2;
    if (FOLD > 0 && ++q.k == FOLD)
        sumsq_flush(q);
}

__device__ __forceinline__ double sumsq_value(SumSq &q)
{
    sumsq_flush(q);
    return q.acc;
}

// (s, c) += (s2, c2) for two double-float pairs of non-negative sums:
// two-sum of the heads (its error is exact, so the result does not depend
// on the order of the operands), the tails and that error added, and a
// fast-two-sum to renormalise (the head dominates: all terms are >= 0).
__device__ __forceinline__ void sumsq_pair_add(float &s, float &c, float s2, float c2)
{
    const float t = __fadd_rn(s, s2);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2, bp));
    const float cc = __fadd_rn(__fadd_rn(c, c2), err);
    const float s3 = __fadd_rn(t, cc);
    c = __fsub_rn(cc, __fsub_rn(s3, t));
    s = s3;
}

// The block total of the per-thread sums of squares taken without the
// periodic fold (FOLD = 0), for blocks of NW warps: the pairs are added as
// double-floats in an xor tree within each warp and then in warp order by
// thread 0, and converted to binary64 once; the binary64 parts (squares
// outside the binary32 range) are added in binary64 only when some thread
// has one.  Binary32 work instead of a binary64 tree: GB300's binary64 pipe
// takes a whole warp instruction for each binary64 operation.  Every thread
// of the block calls it; the result is valid in thread 0.  spair and sacc
// are shared arrays of NW entries.
template <int NW>
__device__ __forceinline__ double sumsq_block_total(const SumSq &q, float2 *spair, double *sacc)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float s = q.s, c = q.c;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, off);
        const float c2 = __shfl_xor_sync(0xffffffffu, c, off);
        sumsq_pair_add(s, c, s2, c2);
    }
    const bool wide = __syncthreads_or(q.acc != 0.0) != 0;   // block-uniform
    double acc = 0.0;
    if (wide) {
        acc = q.acc;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            acc += __shfl_xor_sync(0xffffffffu, acc, off);
    }
    if (lane == 0) {
        spair[wid] = make_float2(s, c);
        sacc[wid] = acc;
    }
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        float S = spair[0].x, Cc = spair[0].y;
        for (int w = 1; w < NW; ++w)
            sumsq_pair_add(S, Cc, spair[w].x, spair[w].y);
        t = __dadd_rn((double)S, (double)Cc);
        if (wide) {
            double a = 0.0;
            for (int w = 0; w < NW; ++w)
                a = __dadd_rn(a, sacc[w]);
            t = __dadd_rn(t, a);
        }
    }
    return t;
}

}  // namespace nsli
