// nsli_batch.cu -- batched form: many problems sharing one bf16 A on the
// 5th-generation tensor cores (tcgen05, sm_103a).
//
// P problems share the matrix A (m x n, stored as bf16) and differ in x_p
// and in the tick offset s_p of their right-hand side
// b_p(k) = b0 + (s_p + k) rho Av.  One batch iteration is, for every p, the
// iteration of Algorithm 1 (Section 2, Eq. 7 and Eq. 8, relaxed step):
//
//   R = A X            (m x P)         GEMM 1, contraction over n
//   W = max(R - B, 0) / ||a_i||^2      epilogue of GEMM 1 (Eq. 7 weights)
//   h_p = #{i : R_ip > B_ip}           epilogue of GEMM 1
//   Y = A^T W          (n x P)         GEMM 2, contraction over m
//   x_p <- x_p - lambda y_p / h_p      epilogue of GEMM 2
//
// Both GEMMs read both operands K-major (GEMM 2 reads a transposed bf16
// copy of A), so one tcgen05 kernel serves both; only the epilogues differ.
// The binary32 values of X and W enter the bf16 tensor cores as three bf16
// terms hi + mid + lo, which reproduce each binary32 value exactly, so every
// product is exact and the accumulation is binary32 (in TMEM): the
// operand's N dimension holds the 3 * P split columns and the epilogue adds
// the three partial dots of each problem.
//
// Kernel layout: 6 warps.  Warp 0 issues the TMA tile loads (128B swizzle)
// into a 5-stage shared-memory ring; warp 1 allocates 512 TMEM columns (two
// 128 x 256 binary32 accumulators) and one of its threads issues
// tcgen05.mma; warps 2-5 drain an accumulator with tcgen05.ld while the
// other one is being filled.  Every wait is bounded.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>

#include "nsli.h"
#include "nsli_internal.h"

namespace nsli {
namespace batch {

constexpr int BM = 128;        // rows of the A operand per tile (TMEM lanes)
constexpr int BK = 64;         // K per stage: 64 bf16 = one 128-byte swizzle row
#ifndef NSLI_BATCH_STAGES
#define NSLI_BATCH_STAGES 5
#endif
constexpr int NSTAGE = NSLI_BATCH_STAGES;   // shared-memory ring depth (5 x 40 KB fits in 227 KB)
// mbarrier slots after the ring: full[s], empty[s], accumulator full[2], accumulator empty[2]
constexpr int kBarFull = 0, kBarEmpty = NSTAGE, kBarTFull = 2 * NSTAGE, kBarTEmpty = 2 * NSTAGE + 2;
constexpr int kBarCount = 2 * NSTAGE + 4;
constexpr int kThreads = 192;  // 6 warps
constexpr int kAccCols = 256;  // TMEM columns per accumulator
constexpr int kTmemCols = 512;
constexpr int kMaxBN = 192;    // 3 split columns x 64 problems
constexpr int kStageA = BM * BK * 2;          // 16 KB
constexpr int kStageB = kMaxBN * BK * 2;      // 24 KB
constexpr int kStageBytes = kStageA + kStageB;
constexpr int kSmemBytes = 1024 + NSTAGE * kStageBytes + 256;
static_assert(kBarCount * 8 + 16 <= 256, "barriers fit behind the ring");
constexpr long long kWaitCycles = 4000000000ll;

struct State {
    long long k;       // batch iteration counter (tick)
    double lambda, rho;
    int error;
    int pad;
};

struct EpiArgs {
    int mode;          // 0: GEMM 1 epilogue, 3: GEMM 2 partial sums of one K split
    int Pp, nprob, BN;
    long long Mdim;    // rows of the A operand (m, or n for GEMM 2)
    int ktiles;        // 64-wide K chunks per K split
    int ktiles_total;  // 64-wide K chunks of the whole contraction
    int mtiles;        // 128-row tiles of the A operand
    int nwork;         // mtiles * K splits
    // GEMM 1
    const float *b0f, *avf, *invn2f;
    const long long *s_off;
    __nv_bfloat16 *Ws;
    long long ldw;
    int *cnt;                 // [2][Pp] violated rows
    unsigned long long *maxv; // [2][Pp] order-preserving max residual
    // GEMM 2
    double *X64;              // [Pp][ldx]
    __nv_bfloat16 *Xs;        // [3 Pp][ldx]
    long long ldx;
    float *Ypart;             // [splits][Pp][ldx] (mode 3)
    State *st;
};

// ---------------------------------------------------------------- PTX ----

__device__ __forceinline__ unsigned int smem_u32(const void *p)
{
    return (unsigned int)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned int bar, unsigned int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned int bar, unsigned int bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned int bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned int bar, unsigned int parity)
{
    unsigned int ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait; gives up at the cycle limit or when *abort is set (and then
// sets *abort so that every role leaves its loop).
__device__ __forceinline__ bool wait_bar(unsigned int bar, unsigned int parity, volatile int *abort)
{
    const long long t0 = clock64();
    for (unsigned int it = 0;; ++it) {
        if (mbar_test(bar, parity))
            return true;
        if ((it & 63u) == 63u) {
            if (*abort)
                return false;
            if (clock64() - t0 > kWaitCycles) {
                *abort = 1;
                return false;
            }
        }
    }
}
__device__ __forceinline__ void tma_load_2d(unsigned int dst, const CUtensorMap *tm, int x, int y, unsigned int bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((unsigned long long)tm), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
// K-major operand tile in shared memory with 128-byte swizzle: rows of 128
// bytes (64 bf16 of K), 8-row atoms of 1024 bytes (stride byte offset 1024).
__device__ __forceinline__ unsigned long long sdesc(unsigned int saddr)
{
    unsigned long long d = 0;
    d |= (unsigned long long)((saddr & 0x3FFFFu) >> 4);
    d |= (unsigned long long)1 << 16;              // leading byte offset (unused with swizzle)
    d |= (unsigned long long)(1024 >> 4) << 32;    // stride byte offset
    d |= (unsigned long long)1 << 46;              // descriptor version
    d |= (unsigned long long)2 << 61;              // 128-byte swizzle
    return d;
}
// kind::f16 instruction descriptor: D binary32, A and B bf16, both K-major.
__host__ __device__ constexpr unsigned int idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned int)(N >> 3) << 17) | ((unsigned int)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(unsigned int tmem_d, unsigned long long a, unsigned long long b,
                                         unsigned int idesc, unsigned int accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(unsigned int bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld16(unsigned int taddr, float (&v)[16])
{
    unsigned int r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i)
        v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ unsigned long long ord_enc(double d)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// binary32 -> hi + mid + lo, each bf16, with hi + mid + lo == v exactly
__device__ __forceinline__ void split3(float v, __nv_bfloat16 &h, __nv_bfloat16 &m, __nv_bfloat16 &l)
{
    h = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(h);
    m = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(m);
    l = __float2bfloat16_rn(r2);
}

// --------------------------------------------------------------- kernel ----

__global__ void __launch_bounds__(kThreads, 1)
    gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const EpiArgs e)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const unsigned int raw = smem_u32(smem_raw);
    const unsigned int base = (raw + 1023u) & ~1023u;
    unsigned char *sbase = smem_raw + (base - raw);
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(sbase + NSTAGE * kStageBytes);
    unsigned int *tmem_holder = reinterpret_cast<unsigned int *>(bars + kBarCount);
    volatile int *abort = reinterpret_cast<volatile int *>(bars + kBarCount + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int BN = e.BN;
    const unsigned int idesc = idesc_bf16(BM, BN);
    const unsigned int stage_tx = (unsigned int)(kStageA + BN * BK * 2);

    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(smem_u32(&bars[kBarFull + s]), 1);
            mbar_init(smem_u32(&bars[kBarEmpty + s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&bars[kBarTFull + a]), 1);
            mbar_init(smem_u32(&bars[kBarTEmpty + a]), 4);
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned int tmem_base = *tmem_holder;

    if (warp == 0) {
        // ---- TMA producer
        if (lane == 0) {
            int s = 0;
            unsigned int ph = 0;
            bool ok = true;
            for (int w = blockIdx.x; w < e.nwork && ok; w += gridDim.x) {
                const int tile = w % e.mtiles, ks = w / e.mtiles;
                const int kbeg = ks * e.ktiles;
                const int kend = min(kbeg + e.ktiles, e.ktiles_total);
                for (int kc = kbeg; kc < kend; ++kc) {
                    if (!wait_bar(smem_u32(&bars[kBarEmpty + s]), ph ^ 1u, abort)) {
                        ok = false;
                        break;
                    }
                    const unsigned int fb = smem_u32(&bars[kBarFull + s]);
                    mbar_expect_tx(fb, stage_tx);
                    const unsigned int sa = base + s * kStageBytes;
                    tma_load_2d(sa, &tmA, kc * BK, tile * BM, fb);
                    tma_load_2d(sa + kStageA, &tmB, kc * BK, 0, fb);
                    if (++s == NSTAGE) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            // wait (bounded) until the MMA side has consumed every issued stage
            if (ok) {
                for (int q = 0; q < NSTAGE; ++q) {
                    if (!wait_bar(smem_u32(&bars[kBarEmpty + s]), ph ^ 1u, abort))
                        break;
                    if (++s == NSTAGE) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            int s = 0;
            unsigned int ph = 0;
            int acc = 0;
            unsigned int aph = 0;
            bool ok = true;
            for (int w = blockIdx.x; w < e.nwork && ok; w += gridDim.x) {
                const int ks = w / e.mtiles;
                const int kbeg = ks * e.ktiles;
                const int kend = min(kbeg + e.ktiles, e.ktiles_total);
                if (!wait_bar(smem_u32(&bars[kBarTEmpty + acc]), aph ^ 1u, abort))
                    break;
                tc_fence_after();
                const unsigned int dcol = tmem_base + (unsigned int)(acc * kAccCols);
                for (int kc = kbeg; kc < kend; ++kc) {
                    if (!wait_bar(smem_u32(&bars[kBarFull + s]), ph, abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const unsigned int sa = base + s * kStageBytes;
#pragma unroll
                    for (int k16 = 0; k16 < BK / 16; ++k16) {
                        const unsigned long long ad = sdesc(sa + k16 * 32);
                        const unsigned long long bd = sdesc(sa + kStageA + k16 * 32);
                        mma_bf16(dcol, ad, bd, idesc, (kc > kbeg || k16 > 0) ? 1u : 0u);
                    }
                    mma_commit(smem_u32(&bars[kBarEmpty + s]));  // frees the stage once these MMAs have read it
                    if (++s == NSTAGE) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (!ok)
                    break;
                mma_commit(smem_u32(&bars[kBarTFull + acc]));    // accumulator ready
                if (++acc == 2) {
                    acc = 0;
                    aph ^= 1u;
                }
            }
        }
    } else {
        // ---- epilogue warps 2..5: TMEM lanes 32 * (warp % 4) ...
        const int lg = warp & 3;
        const unsigned int lane_off = (unsigned int)(32 * lg) << 16;
        int acc = 0;
        unsigned int aph = 0;
        const long long k = e.st->k;
        const int cur = (int)(k & 1);
        const float rho = (float)e.st->rho;
        for (int w = blockIdx.x; w < e.nwork; w += gridDim.x) {
            const int tile = w % e.mtiles, ks = w / e.mtiles;
            if (!wait_bar(smem_u32(&bars[kBarTFull + acc]), aph, abort))
                break;
            tc_fence_after();
            const long long row = (long long)tile * BM + 32 * lg + lane;
            const bool valid = row < e.Mdim;
            const unsigned int tbase = tmem_base + lane_off + (unsigned int)(acc * kAccCols);
            if (e.mode == 0) {
                float b0 = 0.f, av = 0.f, in2 = 0.f;
                if (valid) {
                    b0 = e.b0f[row];
                    av = e.avf[row];
                    in2 = e.invn2f[row];
                }
                for (int pc = 0; pc < e.Pp; pc += 16) {
                    float v0[16], v1[16], v2[16];
                    tmem_ld16(tbase + pc, v0);
                    tmem_ld16(tbase + e.Pp + pc, v1);
                    tmem_ld16(tbase + 2 * e.Pp + pc, v2);
                    tmem_wait_ld();
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int p = pc + q;
                        const bool live = p < e.nprob;
                        const float tk = live ? (float)((double)(e.s_off[p] + k) * (double)rho) : 0.f;
                        const float bi = fmaf(tk, av, b0);
                        const float r = (v0[q] + v1[q]) + v2[q] - bi;
                        const bool viol = valid && live && r > 0.f;
                        const float w = viol ? r * in2 : 0.f;
                        if (valid) {
                            __nv_bfloat16 h, m, l;
                            split3(w, h, m, l);
                            e.Ws[(long long)p * e.ldw + row] = h;
                            e.Ws[(long long)(e.Pp + p) * e.ldw + row] = m;
                            e.Ws[(long long)(2 * e.Pp + p) * e.ldw + row] = l;
                        }
                        const unsigned int bal = __ballot_sync(0xffffffffu, viol);
                        float mr = (valid && live) ? r : -INFINITY;
#pragma unroll
                        for (int off = 16; off > 0; off >>= 1)
                            mr = fmaxf(mr, __shfl_xor_sync(0xffffffffu, mr, off));
                        if (lane == 0 && live) {
                            if (bal)
                                atomicAdd(&e.cnt[cur * e.Pp + p], __popc(bal));
                            if (mr > -INFINITY)
                                atomicMax(&e.maxv[cur * e.Pp + p], ord_enc((double)mr));
                        }
                    }
                }
            } else {
                // GEMM 2: the three split columns of each problem, summed, are
                // this K split's partial y; the finish kernel adds the splits
                for (int pc = 0; pc < e.Pp; pc += 16) {
                    float v0[16], v1[16], v2[16];
                    tmem_ld16(tbase + pc, v0);
                    tmem_ld16(tbase + e.Pp + pc, v1);
                    tmem_ld16(tbase + 2 * e.Pp + pc, v2);
                    tmem_wait_ld();
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int p = pc + q;
                        if (valid && p < e.nprob)
                            e.Ypart[((long long)ks * e.Pp + p) * e.ldx + row] = (v0[q] + v1[q]) + v2[q];
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(smem_u32(&bars[kBarTEmpty + acc]));
            if (++acc == 2) {
                acc = 0;
                aph ^= 1u;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort)
        atomicOr(&e.st->error, ERRF_TIMEOUT);
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols)
                     : "memory");
    }
}

// ------------------------------------------------------ helper kernels ----

// y_p[j] = sum over K splits (in order) of the partials; then either the
// relaxed step of problem p (mode 1) or y written out (mode 2).
__global__ void finish_kernel(const float *Ypart, int splits, int Pp, int nprob, long long n, long long ldx,
                              const int *cnt, const State *st, double *X64, __nv_bfloat16 *Xs, double *Yout,
                              int mode)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)nprob * ldx)
        return;
    const long long p = t / ldx, j = t % ldx;
    if (j >= n)
        return;
    double y = 0.0;
    for (int ks = 0; ks < splits; ++ks)
        y += (double)Ypart[((long long)ks * Pp + p) * ldx + j];
    const long long ix = p * ldx + j;
    if (mode == 2) {
        Yout[ix] = y;
        return;
    }
    const int cur = (int)(st->k & 1);
    const int hc = cnt[cur * Pp + p];
    const double s = hc > 0 ? st->lambda / (double)hc : 0.0;
    const double xn = X64[ix] - s * y;
    X64[ix] = xn;
    __nv_bfloat16 h, m, l;
    split3((float)xn, h, m, l);
    Xs[ix] = h;
    Xs[(long long)Pp * ldx + ix] = m;
    Xs[(long long)(2 * Pp) * ldx + ix] = l;
}

// AT[j][i] = A[i][j] (bf16), 32 x 32 tiles through shared memory.
__global__ void transpose_kernel(const __nv_bfloat16 *A, long long lda, __nv_bfloat16 *AT, long long ldt, long long m,
                                 long long n)
{
    __shared__ __nv_bfloat16 t[32][33];
    const long long i0 = (long long)blockIdx.y * 32, j0 = (long long)blockIdx.x * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const long long i = i0 + r, j = j0 + threadIdx.x;
        t[r][threadIdx.x] = (i < m && j < n) ? A[i * lda + j] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const long long j = j0 + r, i = i0 + threadIdx.x;
        if (j < n && i < ldt)
            AT[j * ldt + i] = (i < m) ? t[threadIdx.x][r] : __float2bfloat16_rn(0.f);
    }
}

// X64[p][j] (p < nprob, j < n) from X0 (nprob x n doubles); zero elsewhere;
// Xs = three-term bf16 split of the binary32 rounding.
__global__ void x_init_kernel(const double *X0, double *X64, __nv_bfloat16 *Xs, int nprob, int Pp, long long n,
                              long long ldx, int *flags)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)Pp * ldx)
        return;
    const long long p = t / ldx, j = t % ldx;
    double v = 0.0;
    if (p < nprob && j < n) {
        v = X0[p * n + j];
        if (!isfinite(v))
            atomicOr(flags, PREPF_NONFINITE);
    }
    X64[t] = v;
    __nv_bfloat16 h, m, l;
    split3((float)v, h, m, l);
    Xs[p * ldx + j] = h;
    Xs[(Pp + p) * ldx + j] = m;
    Xs[(2 * Pp + p) * ldx + j] = l;
}

__global__ void rows_init_kernel(const double *b0, const double *av, const double *n2, float *b0f, float *avf,
                                 float *invn2f, long long m, int *flags)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m)
        return;
    if (!isfinite(b0[i]) || !isfinite(av[i]))
        atomicOr(flags, PREPF_NONFINITE);
    b0f[i] = (float)b0[i];
    avf[i] = (float)av[i];
    invn2f[i] = (float)(1.0 / n2[i]);
}

// End of a batch iteration: k += 1 and clear the counters the next GEMM 1 uses.
__global__ void tick_kernel(State *st, int *cnt, unsigned long long *maxv, int Pp, int advance)
{
    const long long k = st->k + (advance ? 1 : 0);
    const int nxt = (int)(k & 1);
    for (int p = threadIdx.x; p < Pp; p += blockDim.x) {
        cnt[nxt * Pp + p] = 0;
        maxv[nxt * Pp + p] = 0ull;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        st->k = k;
}

// Per-problem state for the binary64 check (verify_kernel reads tick and rho).
__global__ void vstate_kernel(DevState *vs, const long long *s_off, const State *st, int nprob)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < nprob) {
        vs[p].tick = s_off[p] + st->k;
        vs[p].rho = st->rho;
    }
}

}  // namespace batch
}  // namespace nsli

// ====================================================================== host

using namespace nsli;
using namespace nsli::batch;

struct nsli_batch_solver {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    long long m = 0, n = 0, ldn = 0, ldm = 0;
    int nprob = 0, Pp = 0, BN = 0, num_sms = 1;
    __nv_bfloat16 *A = nullptr, *AT = nullptr, *Xs = nullptr, *Ws = nullptr;
    double *b0_64 = nullptr, *av_64 = nullptr, *n2_64 = nullptr, *X64 = nullptr, *Y = nullptr;
    float *Ypart = nullptr;
    int splits = 1, split_tiles = 1;
    float *b0f = nullptr, *avf = nullptr, *invn2f = nullptr;
    long long *s_off = nullptr;
    int *cnt = nullptr, *flags = nullptr;
    unsigned long long *maxv = nullptr;
    State *st = nullptr;
    DevState *vst = nullptr;
    VerOut *ver = nullptr;
    CUtensorMap tmA, tmX, tmAT, tmW;
    cudaGraphExec_t graph = nullptr;
    int graph_iters = 0;
    long long launches = 0;
    std::string last_error;
};
namespace {

int berr(nsli_batch h, int code, const std::string &msg)
{
    if (h)
        h->last_error = msg;
    return code;
}
int bcuda(nsli_batch h, cudaError_t e, const char *what)
{
    const std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    return berr(h, e == cudaErrorMemoryAllocation ? NSLI_ERR_OOM : NSLI_ERR_CUDA, msg);
}
#define BCK(call, what)                                                                                      \
    do {                                                                                                     \
        cudaError_t e_ = (call);                                                                             \
        if (e_ != cudaSuccess)                                                                               \
            return bcuda(h, e_, what);                                                                       \
    } while (0)

PFN_cuTensorMapEncodeTiled_v12000 get_encode()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D bf16 tensor [rows][cols] with row pitch `ld` elements; box 64 x box_rows.
bool make_map(CUtensorMap *tm, void *ptr, long long cols, long long rows, long long ld, int box_rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
    if (!enc)
        return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void bfree(nsli_batch h)
{
    if (h->graph)
        cudaGraphExecDestroy(h->graph);
    void *p[] = {h->A, h->AT, h->Xs, h->Ws, h->b0_64, h->av_64, h->n2_64, h->X64, h->Y, h->Ypart, h->b0f, h->avf,
                 h->invn2f, h->s_off, h->cnt, h->flags, h->maxv, h->st, h->vst, h->ver};
    for (void *q : p)
        if (q)
            cudaFree(q);
    if (h->own_stream && h->stream)
        cudaStreamDestroy(h->stream);
}

EpiArgs epi_args(nsli_batch h, int mode)
{
    EpiArgs e;
    std::memset(&e, 0, sizeof e);
    e.mode = mode;
    e.Pp = h->Pp;
    e.nprob = h->nprob;
    e.BN = h->BN;
    e.b0f = h->b0f;
    e.avf = h->avf;
    e.invn2f = h->invn2f;
    e.s_off = h->s_off;
    e.Ws = h->Ws;
    e.ldw = h->ldm;
    e.cnt = h->cnt;
    e.maxv = h->maxv;
    e.X64 = h->X64;
    e.Xs = h->Xs;
    e.ldx = h->ldn;
    e.Ypart = h->Ypart;
    e.st = h->st;
    if (mode == 0) {
        e.Mdim = h->m;
        e.ktiles_total = (int)((h->n + BK - 1) / BK);
        e.ktiles = e.ktiles_total;
        e.mtiles = (int)((h->m + BM - 1) / BM);
        e.nwork = e.mtiles;
    } else {
        e.Mdim = h->n;
        e.ktiles_total = (int)((h->m + BK - 1) / BK);
        e.ktiles = h->split_tiles;
        e.mtiles = (int)((h->n + BM - 1) / BM);
        e.nwork = e.mtiles * h->splits;
    }
    return e;
}

// mode 0: GEMM 1 with its epilogue; mode 1 / 2: GEMM 2 partial sums, then
// the finish kernel (1: relaxed step, 2: y written out)
cudaError_t launch_gemm(nsli_batch h, int mode)
{
    const EpiArgs e = epi_args(h, mode == 0 ? 0 : 3);
    // the fewest CTAs that take the work items in as many rounds as one CTA
    // per SM would (512 row tiles on 152 SMs: 128 CTAs of 4 tiles each, the
    // same rounds with less contention); NSLI_BATCH_GRID=sms keeps one per SM
    const int rounds = (e.nwork + h->num_sms - 1) / h->num_sms;
    int grid = (e.nwork + rounds - 1) / rounds;
    if (const char *env = std::getenv("NSLI_BATCH_GRID"))
        if (std::strcmp(env, "sms") == 0)
            grid = std::min(h->num_sms, e.nwork);
    if (mode == 0) {
        gemm_kernel<<<grid, kThreads, kSmemBytes, h->stream>>>(h->tmA, h->tmX, e);
        return cudaGetLastError();
    }
    gemm_kernel<<<grid, kThreads, kSmemBytes, h->stream>>>(h->tmAT, h->tmW, e);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess)
        return err;
    const long long tot = (long long)h->nprob * h->ldn;
    finish_kernel<<<(unsigned int)((tot + 255) / 256), 256, 0, h->stream>>>(
        h->Ypart, h->splits, h->Pp, h->nprob, h->n, h->ldn, h->cnt, h->st, h->X64, h->Xs, h->Y, mode);
    return cudaGetLastError();
}

cudaError_t launch_batch_iteration(nsli_batch h)
{
    cudaError_t err = launch_gemm(h, 0);
    if (err == cudaSuccess)
        err = launch_gemm(h, 1);
    if (err == cudaSuccess) {
        tick_kernel<<<1, 64, 0, h->stream>>>(h->st, h->cnt, h->maxv, h->Pp, 1);
        err = cudaGetLastError();
    }
    return err;
}

int read_error(nsli_batch h)
{
    State s;
    BCK(cudaMemcpyAsync(&s, h->st, sizeof s, cudaMemcpyDeviceToHost, h->stream), "read state");
    BCK(cudaStreamSynchronize(h->stream), "synchronize");
    if (s.error & ERRF_TIMEOUT)
        return berr(h, NSLI_ERR_TIMEOUT, "a bounded device wait expired");
    return NSLI_OK;
}

}  // namespace

extern "C" {

int nsli_batch_create(nsli_batch *out, int64_t m, int64_t n, int32_t nprob, const float *A, int64_t lda,
                      const double *b0, const double *Av, const int64_t *tick_offsets, const double *X0,
                      void *stream)
{
    if (!out)
        return NSLI_ERR_ARG;
    *out = nullptr;
    if (m < 1 || n < 1 || lda < n || nprob < 1 || !A || !b0 || !X0)
        return NSLI_ERR_ARG;
    if (nprob > 64 || m > (1ll << 31) || n > (1ll << 31))
        return NSLI_ERR_UNSUPPORTED;
    nsli_batch h = new nsli_batch_solver();
    auto fail = [&](int code) {
        bfree(h);
        delete h;
        return code;
    };
#define BCKC(call, what)                                                                                     \
    do {                                                                                                     \
        cudaError_t e_ = (call);                                                                             \
        if (e_ != cudaSuccess)                                                                               \
            return fail(bcuda(h, e_, what));                                                                 \
    } while (0)
    h->m = m;
    h->n = n;
    h->nprob = nprob;
    h->Pp = (nprob + 15) / 16 * 16;
    h->BN = 3 * h->Pp;
    h->ldn = (n + 7) / 8 * 8;
    h->ldm = (m + 7) / 8 * 8;
    BCKC(cudaGetDevice(&h->device), "get device");
    BCKC(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device), "SM count");
    if (!get_encode())
        return fail(berr(h, NSLI_ERR_CUDA, "cuTensorMapEncodeTiled unavailable"));
    if (stream) {
        h->stream = static_cast<cudaStream_t>(stream);
    } else {
        BCKC(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking), "create stream");
        h->own_stream = true;
    }
    cudaStream_t s = h->stream;
    BCKC(cudaMalloc((void **)&h->A, (size_t)m * h->ldn * 2), "allocate A");
    BCKC(cudaMalloc((void **)&h->AT, (size_t)n * h->ldm * 2), "allocate A^T");
    BCKC(cudaMalloc((void **)&h->Xs, (size_t)3 * h->Pp * h->ldn * 2), "allocate X splits");
    BCKC(cudaMalloc((void **)&h->Ws, (size_t)3 * h->Pp * h->ldm * 2), "allocate W splits");
    BCKC(cudaMalloc((void **)&h->X64, (size_t)h->Pp * h->ldn * 8), "allocate X");
    BCKC(cudaMalloc((void **)&h->Y, (size_t)h->Pp * h->ldn * 8), "allocate Y");
    {
        // K splits of GEMM 2 so that its (n / 128) x splits work items fill the SMs
        const long long jt = (n + BM - 1) / BM;
        const long long kt = (m + BK - 1) / BK;
        h->splits = (int)std::max<long long>(1, std::min<long long>(h->num_sms / std::max<long long>(1, jt), kt));
        if (const char *env = std::getenv("NSLI_BATCH_SPLITS")) {
            const int v = std::atoi(env);
            if (v >= 1 && v <= 64)
                h->splits = (int)std::min<long long>(v, kt);
        }
        // equal chunk counts per split and no empty split
        const long long per = (kt + h->splits - 1) / h->splits;
        h->splits = (int)((kt + per - 1) / per);
        h->split_tiles = (int)per;
    }
    BCKC(cudaMalloc((void **)&h->Ypart, (size_t)h->splits * h->Pp * h->ldn * 4), "allocate partial y");
    BCKC(cudaMalloc((void **)&h->b0_64, (size_t)m * 8), "allocate b0");
    BCKC(cudaMalloc((void **)&h->av_64, (size_t)m * 8), "allocate Av");
    BCKC(cudaMalloc((void **)&h->n2_64, (size_t)m * 8), "allocate norms");
    BCKC(cudaMalloc((void **)&h->b0f, (size_t)m * 4), "allocate b0f");
    BCKC(cudaMalloc((void **)&h->avf, (size_t)m * 4), "allocate Avf");
    BCKC(cudaMalloc((void **)&h->invn2f, (size_t)m * 4), "allocate 1/norms");
    BCKC(cudaMalloc((void **)&h->s_off, (size_t)h->Pp * 8), "allocate tick offsets");
    BCKC(cudaMalloc((void **)&h->cnt, (size_t)2 * h->Pp * 4), "allocate counters");
    BCKC(cudaMalloc((void **)&h->maxv, (size_t)2 * h->Pp * 8), "allocate maxima");
    BCKC(cudaMalloc((void **)&h->flags, 4), "allocate flags");
    BCKC(cudaMalloc((void **)&h->st, sizeof(State)), "allocate state");
    BCKC(cudaMalloc((void **)&h->vst, (size_t)h->Pp * sizeof(DevState)), "allocate check state");
    BCKC(cudaMalloc((void **)&h->ver, (size_t)h->Pp * sizeof(VerOut)), "allocate check output");

    BCKC(cudaMemsetAsync(h->flags, 0, 4, s), "clear flags");
    BCKC(cudaMemsetAsync(h->st, 0, sizeof(State), s), "clear state");
    BCKC(cudaMemsetAsync(h->cnt, 0, (size_t)2 * h->Pp * 4, s), "clear counters");
    BCKC(cudaMemsetAsync(h->maxv, 0, (size_t)2 * h->Pp * 8, s), "clear maxima");
    BCKC(cudaMemsetAsync(h->vst, 0, (size_t)h->Pp * sizeof(DevState), s), "clear check state");
    BCKC(cudaMemsetAsync(h->s_off, 0, (size_t)h->Pp * 8, s), "clear tick offsets");
    if (tick_offsets)
        BCKC(cudaMemcpyAsync(h->s_off, tick_offsets, (size_t)nprob * 8, cudaMemcpyDefault, s), "copy tick offsets");
    BCKC(cudaMemcpyAsync(h->b0_64, b0, (size_t)m * 8, cudaMemcpyDefault, s), "copy b0");
    if (Av)
        BCKC(cudaMemcpyAsync(h->av_64, Av, (size_t)m * 8, cudaMemcpyDefault, s), "copy Av");
    else
        BCKC(cudaMemsetAsync(h->av_64, 0, (size_t)m * 8, s), "clear Av");

    // A -> bf16 rows (shared set-up kernel of the single-problem path) and norms
    {
        void *stage = nullptr;
        const long long chunk = std::min<long long>(m, std::max<long long>(1, (256ll << 20) / (lda * 4)));
        BCKC(cudaMalloc(&stage, (size_t)chunk * lda * 4), "allocate staging");
        cudaError_t err = cudaSuccess;
        for (long long r0 = 0; r0 < m && err == cudaSuccess; r0 += chunk) {
            const long long rows = std::min(chunk, m - r0);
            err = cudaMemcpy2DAsync(stage, (size_t)lda * 4, A + r0 * lda, (size_t)lda * 4, (size_t)n * 4, (size_t)rows,
                                    cudaMemcpyDefault, s);
            if (err != cudaSuccess)
                break;
            PrepArgs pa;
            pa.src = stage;
            pa.lda = lda;
            pa.src_f64 = 0;
            pa.A = h->A;
            pa.ld = h->ldn;
            pa.n = n;
            pa.row0 = r0;
            pa.rows = rows;
            pa.norms_in = nullptr;
            pa.n2_64 = h->n2_64;
            pa.scale = nullptr;
            pa.flags = h->flags;
            pa.fast = 0;   // the binary64 norms: the batched check uses them
            err = prep_launch(NSLI_BF16, s, pa);
            if (err == cudaSuccess)
                err = cudaStreamSynchronize(s);
        }
        cudaFree(stage);
        if (err != cudaSuccess)
            return fail(bcuda(h, err, "prepare A"));
    }
    {
        dim3 tb(32, 8), tg((unsigned int)((h->ldn + 31) / 32), (unsigned int)((h->ldm + 31) / 32));
        transpose_kernel<<<tg, tb, 0, s>>>(h->A, h->ldn, h->AT, h->ldm, m, n);
        BCKC(cudaGetLastError(), "transpose A");
        rows_init_kernel<<<(unsigned int)((m + 255) / 256), 256, 0, s>>>(h->b0_64, h->av_64, h->n2_64, h->b0f,
                                                                          h->avf, h->invn2f, m, h->flags);
        BCKC(cudaGetLastError(), "row records");
        double *x0d = nullptr;
        BCKC(cudaMalloc((void **)&x0d, (size_t)nprob * n * 8), "allocate x0");
        cudaError_t err = cudaMemcpyAsync(x0d, X0, (size_t)nprob * n * 8, cudaMemcpyDefault, s);
        if (err == cudaSuccess) {
            const long long tot = (long long)h->Pp * h->ldn;
            x_init_kernel<<<(unsigned int)((tot + 255) / 256), 256, 0, s>>>(x0d, h->X64, h->Xs, nprob, h->Pp, n,
                                                                             h->ldn, h->flags);
            err = cudaGetLastError();
        }
        if (err == cudaSuccess)
            err = cudaStreamSynchronize(s);
        cudaFree(x0d);
        if (err != cudaSuccess)
            return fail(bcuda(h, err, "initial x"));
        BCKC(cudaMemsetAsync(h->Ws, 0, (size_t)3 * h->Pp * h->ldm * 2, s), "clear W");
        int f = 0;
        BCKC(cudaMemcpyAsync(&f, h->flags, 4, cudaMemcpyDeviceToHost, s), "read flags");
        BCKC(cudaStreamSynchronize(s), "synchronize");
        if (f & PREPF_NONFINITE)
            return fail(berr(h, NSLI_ERR_NONFINITE, "NaN or Inf in the input"));
        if (f & PREPF_ZERO_ROW)
            return fail(berr(h, NSLI_ERR_ZERO_ROW, "A has a zero row"));
    }
    if (!make_map(&h->tmA, h->A, n, m, h->ldn, BM) || !make_map(&h->tmX, h->Xs, n, h->BN, h->ldn, h->BN) ||
        !make_map(&h->tmAT, h->AT, m, n, h->ldm, BM) || !make_map(&h->tmW, h->Ws, m, h->BN, h->ldm, h->BN))
        return fail(berr(h, NSLI_ERR_CUDA, "tensor map encoding failed"));
    BCKC(cudaFuncSetAttribute(gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes),
         "configure GEMM kernel");
#undef BCKC
    *out = h;
    return NSLI_OK;
}

void nsli_batch_destroy(nsli_batch h)
{
    if (!h)
        return;
    if (h->stream)
        cudaStreamSynchronize(h->stream);
    bfree(h);
    delete h;
}

int nsli_batch_iterate(nsli_batch h, const nsli_params *p, int64_t n_iter)
{
    if (!h || !p || n_iter < 0)
        return NSLI_ERR_ARG;
    if (!(p->lambda > 0.0) || !std::isfinite(p->lambda) || !std::isfinite(p->rho))
        return berr(h, NSLI_ERR_ARG, "bad lambda or rho");
    if (p->rule != NSLI_RULE_RELAXED)
        return berr(h, NSLI_ERR_UNSUPPORTED, "the batched form implements the relaxed rule");
    BCK(cudaMemcpyAsync(&h->st->lambda, &p->lambda, 8, cudaMemcpyHostToDevice, h->stream), "set lambda");
    BCK(cudaMemcpyAsync(&h->st->rho, &p->rho, 8, cudaMemcpyHostToDevice, h->stream), "set rho");
    const int B = p->block_iters > 0 ? p->block_iters : 16;
    const long long full = n_iter / B, rem = n_iter % B;
    if (full > 0 && !(h->graph && h->graph_iters == B)) {
        if (h->graph) {
            cudaGraphExecDestroy(h->graph);
            h->graph = nullptr;
        }
        BCK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t err = cudaSuccess;
        for (int i = 0; i < B && err == cudaSuccess; ++i)
            err = launch_batch_iteration(h);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
        if (err != cudaSuccess || e2 != cudaSuccess) {
            if (g)
                cudaGraphDestroy(g);
            return bcuda(h, err != cudaSuccess ? err : e2, "capture batch iterations");
        }
        cudaError_t e3 = cudaGraphInstantiate(&h->graph, g, 0);
        cudaGraphDestroy(g);
        BCK(e3, "instantiate batch graph");
        h->graph_iters = B;
    }
    for (long long i = 0; i < full; ++i) {
        BCK(cudaGraphLaunch(h->graph, h->stream), "launch batch graph");
        h->launches += 4ll * B;
    }
    for (long long i = 0; i < rem; ++i) {
        BCK(launch_batch_iteration(h), "launch batch iteration");
        h->launches += 4;
    }
    return NSLI_OK;
}

int nsli_batch_map_reduce(nsli_batch h, double rho, double *Y, int64_t *violated, double *max_viol)
{
    if (!h || !std::isfinite(rho))
        return NSLI_ERR_ARG;
    BCK(cudaMemcpyAsync(&h->st->rho, &rho, 8, cudaMemcpyHostToDevice, h->stream), "set rho");
    BCK(launch_gemm(h, 0), "launch GEMM 1");
    BCK(launch_gemm(h, 2), "launch GEMM 2");
    h->launches += 3;
    int rc = read_error(h);
    if (rc != NSLI_OK)
        return rc;
    State s;
    BCK(cudaMemcpyAsync(&s, h->st, sizeof s, cudaMemcpyDeviceToHost, h->stream), "read state");
    BCK(cudaStreamSynchronize(h->stream), "synchronize");
    const int cur = (int)(s.k & 1);
    if (Y) {
        BCK(cudaMemcpy2DAsync(Y, (size_t)h->n * 8, h->Y, (size_t)h->ldn * 8, (size_t)h->n * 8, (size_t)h->nprob,
                              cudaMemcpyDefault, h->stream),
            "copy Y");
    }
    int cnt[64];
    unsigned long long mv[64];
    BCK(cudaMemcpyAsync(cnt, h->cnt + cur * h->Pp, (size_t)h->nprob * 4, cudaMemcpyDeviceToHost, h->stream),
        "copy counts");
    BCK(cudaMemcpyAsync(mv, h->maxv + cur * h->Pp, (size_t)h->nprob * 8, cudaMemcpyDeviceToHost, h->stream),
        "copy maxima");
    BCK(cudaStreamSynchronize(h->stream), "synchronize");
    for (int p = 0; p < h->nprob; ++p) {
        if (violated)
            violated[p] = cnt[p];
        if (max_viol) {
            const unsigned long long u = mv[p];
            unsigned long long bits = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
            double d;
            std::memcpy(&d, &bits, 8);
            max_viol[p] = d;
        }
    }
    // leave the counters of this tick clear for the next iteration
    tick_kernel<<<1, 64, 0, h->stream>>>(h->st, h->cnt, h->maxv, h->Pp, 0);
    BCK(cudaGetLastError(), "clear counters");
    h->launches += 1;
    return NSLI_OK;
}

int nsli_batch_get_x(nsli_batch h, double *X)
{
    if (!h || !X)
        return NSLI_ERR_ARG;
    BCK(cudaMemcpy2DAsync(X, (size_t)h->n * 8, h->X64, (size_t)h->ldn * 8, (size_t)h->n * 8, (size_t)h->nprob,
                          cudaMemcpyDefault, h->stream),
        "copy X");
    BCK(cudaStreamSynchronize(h->stream), "synchronize");
    return read_error(h);
}

int nsli_batch_residual_max(nsli_batch h, double *max_viol)
{
    if (!h || !max_viol)
        return NSLI_ERR_ARG;
    vstate_kernel<<<1, 64, 0, h->stream>>>(h->vst, h->s_off, h->st, h->nprob);
    BCK(cudaGetLastError(), "check state");
    BCK(cudaMemsetAsync(h->ver, 0, (size_t)h->Pp * sizeof(VerOut), h->stream), "clear check");
    for (int p = 0; p < h->nprob; ++p) {
        VerifyArgs a;
        a.A = h->A;
        a.x64 = h->X64 + (long long)p * h->ldn;
        a.b0_64 = h->b0_64;
        a.av_64 = h->av_64;
        a.n2_64 = h->n2_64;
        a.scale = nullptr;
        a.st = h->vst + p;
        a.out = h->ver + p;
        a.ld = h->ldn;
        a.m = h->m;
        a.nv = (int)(h->ldn * 2 / 16);
        BCK(verify_launch(NSLI_BF16, std::max(1, std::min<int>(h->num_sms * 8, (int)((h->m + 7) / 8))), h->stream, a),
            "binary64 check");
    }
    h->launches += 1 + h->nprob;
    VerOut v[64];
    BCK(cudaMemcpyAsync(v, h->ver, (size_t)h->nprob * sizeof(VerOut), cudaMemcpyDeviceToHost, h->stream),
        "read check");
    BCK(cudaStreamSynchronize(h->stream), "synchronize");
    for (int p = 0; p < h->nprob; ++p) {
        const unsigned long long u = v[p].maxviol;
        unsigned long long bits = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
        std::memcpy(&max_viol[p], &bits, 8);
    }
    return NSLI_OK;
}

int64_t nsli_batch_launch_count(nsli_batch h) { return h ? (int64_t)h->launches : 0; }

int nsli_batch_sync(nsli_batch h)
{
    if (!h)
        return NSLI_ERR_ARG;
    BCK(cudaStreamSynchronize(h->stream), "synchronize");
    return read_error(h);
}

const char *nsli_batch_last_error(nsli_batch h) { return h ? h->last_error.c_str() : ""; }

}  // extern "C"
