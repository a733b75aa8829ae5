// nsli_async.cuh -- mbarriers, bulk copies and the voting block barrier
// shared by the kernels that stage rows in shared memory.
//
// Every wait is bounded: a kernel that gives up records an error, waits
// (again bounded) for its own copies in flight and returns.
#pragma once

#include <cuda_runtime.h>

namespace nsli {

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
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
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
// Wait for the phase of the given parity to complete by polling (a
// non-suspending test: the waiting warps resume as soon as the phase
// completes).  Gives up after kWaitLimitCycles SM cycles (about two seconds
// at the maximum clock), checked every 256 polls.  Returns true on success.
constexpr long long kWaitLimitCycles = 4000000000ll;
__device__ __forceinline__ bool mbar_wait_bounded(unsigned int bar, unsigned int parity)
{
    const long long t0 = clock64();
    for (unsigned int it = 0;; ++it) {
        if (mbar_test(bar, parity))
            return true;
        if ((it & 255u) == 255u && clock64() - t0 > kWaitLimitCycles)
            return false;
    }
}
__device__ __forceinline__ void bulk_g2s(unsigned int dst, const void *src, unsigned int bytes,
                                         unsigned int bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
// Block barrier (id 1) with an OR-vote, so that every thread leaves the
// loop together when any of them gave up waiting.
__device__ __forceinline__ int bar_all_or(int nthreads, int pred)
{
    unsigned int out;
    asm volatile(
        "{\n\t.reg .pred q, p;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, 1, %2, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(out)
        : "r"(pred), "r"(nthreads)
        : "memory");
    return (int)out;
}

}  // namespace nsli
