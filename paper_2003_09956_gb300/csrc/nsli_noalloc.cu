// nsli_noalloc.cu -- a Map + Reduce entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc: code that runs under a fixed
// device-memory budget, and code inside a host framework that owns all
// device memory through its own allocator and does not let libraries take
// memory of their own (a cudaMalloc there can fail, or push the framework
// past its budget; cudaFree also waits for the whole device).
// nsli_map_reduce_noalloc serves them: the caller passes every input and
// output, and the kernels' scratch (one row of partial sums per CTA, and
// per-CTA counters) lives in the file-scope array below, which every GPU
// that loads this library holds until the process exits.
//
// The array is shared by every call: calls that overlap on the GPU (for
// example on two streams at once) race on it and must not be issued.  Each
// call clears the part it accumulates into before using it.
#include <mutex>

#include "nsli.h"
#include "nsli_internal.h"

namespace {

constexpr long long kScratchFloats = 1ll << 20;   // 4 MiB of partial sums
constexpr int kMaxCtas = 1024;                     // per-CTA counter records
constexpr int kThreads = 256;

struct CtaStat {
    int h;
    float maxviol;
    int pad0, pad1;
};

// scratch: [kScratchFloats floats of partial sums][kMaxCtas CtaStat]
static __device__ __align__(256) unsigned char nsli_noalloc_scratch[kScratchFloats * 4 + kMaxCtas * sizeof(CtaStat)];

// One CTA per contiguous block of rows.  Per row: a block-wide dot in a
// fixed order, r_i = <a_i, x> - b_i, and for r_i > 0 the positive slice
// r_i / ||a_i||^2 * a_i (Eq. 7) is added into the CTA's row of partial sums
// (thread t owns columns t, t + 256, ...; no two threads share an element).
__global__ void __launch_bounds__(kThreads) noalloc_map_kernel(const float *A, long long lda, long long m,
                                                               long long n, const float *b, const float *norms2,
                                                               const float *x, float *part, CtaStat *stat,
                                                               long long rows_base, int rows_rem)
{
    __shared__ float red[kThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long cta = blockIdx.x;
    const long long r0 = cta * rows_base + (cta < rows_rem ? cta : (long long)rows_rem);
    const long long r1 = r0 + rows_base + (cta < rows_rem ? 1 : 0);
    float *py = part + cta * n;
    for (long long j = tid; j < n; j += kThreads)
        py[j] = 0.0f;  // the array keeps the previous call's contents
    int h = 0;
    float mv = -INFINITY;
    for (long long i = r0; i < r1; ++i) {
        const float *a = A + i * lda;
        float s = 0.0f;
        for (long long j = tid; j < n; j += kThreads)
            s = fmaf(a[j], x[j], s);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            s += __shfl_xor_sync(0xffffffffu, s, off);
        __syncthreads();  // the previous row's reads of red are done
        if (lane == 0)
            red[warp] = s;
        __syncthreads();
        float dot = 0.0f;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w)
            dot += red[w];
        const float ri = dot - b[i];
        h += ri > 0.0f ? 1 : 0;
        mv = fmaxf(mv, ri);
        if (ri > 0.0f) {
            const float c = ri / norms2[i];
            for (long long j = tid; j < n; j += kThreads)
                py[j] = fmaf(c, a[j], py[j]);
        }
    }
    if (tid == 0) {
        CtaStat cs;
        cs.h = h;
        cs.maxviol = mv;
        cs.pad0 = 0;
        cs.pad1 = 0;
        stat[cta] = cs;
    }
}

// y_j = sum over CTAs g = 0..G-1 (in that order) of part[g][j], in binary64;
// block 0 also totals the per-CTA counters.
__global__ void __launch_bounds__(kThreads) noalloc_reduce_kernel(const float *part, const CtaStat *stat, int G,
                                                                  long long n, double *y, long long *violated,
                                                                  double *max_viol)
{
    const long long j = (long long)blockIdx.x * kThreads + threadIdx.x;
    if (j < n) {
        double s = 0.0;
        for (int g = 0; g < G; ++g)
            s += (double)part[(long long)g * n + j];
        y[j] = s;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        long long h = 0;
        float mv = -INFINITY;
        for (int g = 0; g < G; ++g) {
            h += stat[g].h;
            mv = fmaxf(mv, stat[g].maxviol);
        }
        *violated = h;
        *max_viol = (double)mv;
    }
}

struct DeviceScratch {
    bool ready = false;
    unsigned char *ptr = nullptr;
    int sms = 0;
};
constexpr int kMaxDevices = 64;
DeviceScratch g_dev[kMaxDevices];
std::mutex g_mutex;

}  // namespace

extern "C" int nsli_map_reduce_noalloc(int64_t m, int64_t n, const float *A, int64_t lda, const float *b,
                                       const float *norms2, const float *x, double *y, int64_t *violated,
                                       double *max_viol, void *stream)
{
    if (m < 1 || n < 1 || lda < n || !A || !b || !norms2 || !x || !y || !violated || !max_viol)
        return NSLI_ERR_ARG;
    if (n > kScratchFloats)
        return NSLI_ERR_UNSUPPORTED;  // not even one row of partial sums fits the scratch array
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return NSLI_ERR_CUDA;
    DeviceScratch *ds = &g_dev[dev];
    {
        // once per device, with that device current: the device address of
        // the scratch array (its host-side name is not a device address)
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!ds->ready) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, nsli_noalloc_scratch) != cudaSuccess)
                return NSLI_ERR_CUDA;
            int sms = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                return NSLI_ERR_CUDA;
            ds->ptr = static_cast<unsigned char *>(p);
            ds->sms = sms;
            ds->ready = true;
        }
    }
    long long G = ds->sms;
    if (G > m)
        G = m;
    if (G > kScratchFloats / n)
        G = kScratchFloats / n;
    if (G > kMaxCtas)
        G = kMaxCtas;
    float *part = reinterpret_cast<float *>(ds->ptr);
    CtaStat *stat = reinterpret_cast<CtaStat *>(ds->ptr + kScratchFloats * 4);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // an error left pending by the caller's own work is not ours to report
    // or to clear: leave it in place and launch nothing
    if (cudaPeekAtLastError() != cudaSuccess)
        return NSLI_ERR_CUDA;
    noalloc_map_kernel<<<(unsigned int)G, kThreads, 0, s>>>(A, lda, m, n, b, norms2, x, part, stat, m / G,
                                                            (int)(m % G));
    if (cudaGetLastError() != cudaSuccess)
        return NSLI_ERR_CUDA;
    const unsigned int rgrid = (unsigned int)((n + kThreads - 1) / kThreads);
    noalloc_reduce_kernel<<<rgrid, kThreads, 0, s>>>(part, stat, (int)G, n, y, reinterpret_cast<long long *>(violated),
                                                     max_viol);
    if (cudaGetLastError() != cudaSuccess)
        return NSLI_ERR_CUDA;
    return NSLI_OK;
}
