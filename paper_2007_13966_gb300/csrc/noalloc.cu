// ||x||_2 without any allocation: a variant of the deterministic norm
// reduction used by residual_eval (and the Krylov / Newton norms) whose
// partial-sum scratch lives in a static device array compiled into the
// library instead of a buffer the library allocates.
//
// Who needs it: code that must not allocate device memory at call time, for
// example a caller that owns all device memory through its own pool (a
// framework caching allocator, where raw cudaMalloc/cudaFree behind its back
// fragments memory or fails under its budget), or a latency-critical loop
// that cannot afford an allocation, its implicit synchronisation or its
// failure.
#include "common.cuh"

#include <cuda.h>

#include <mutex>

namespace ras {

// one partial sum per block of the reduction grid; every call overwrites all
// NA_BLOCKS entries before reading them, so nothing has to start at zero
constexpr int NA_BLOCKS = 608;
constexpr int NA_THREADS = 256;
// the element range of the library's other vectors (int32 sizes); the loop
// index below is 64-bit, so no stride step can overflow at this limit
constexpr long long NA_MAX_N = 2147483647LL;

static __device__ __align__(256) double g_na_partials[NA_BLOCKS];

__device__ __forceinline__ double na_block_sum(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < NA_THREADS / 32; ++i) s += sh[i];
    return s;
}

__global__ void __launch_bounds__(NA_THREADS) k_na_partial(const double *__restrict__ x, long long n,
                                                           double *__restrict__ partials) {
    __shared__ double sh[NA_THREADS / 32];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)NA_THREADS + threadIdx.x; i < n;
         i += (long long)NA_BLOCKS * NA_THREADS)
        acc = fma(x[i], x[i], acc);
    const double s = na_block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(NA_THREADS) k_na_final(const double *__restrict__ partials,
                                                         double *__restrict__ out) {
    __shared__ double sh[NA_THREADS / 32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < NA_BLOCKS; i += NA_THREADS) acc += partials[i];
    const double s = na_block_sum(acc, sh);
    if (threadIdx.x == 0) *out = sqrt(s);
}

// Device address of g_na_partials for each device, looked up with that device
// current the first time a context of that device calls (the host-side symbol
// is only a stand-in). The cache is keyed on the context's unique id, so a
// context created after cudaDeviceReset looks the address up again.
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);
static std::mutex g_na_mu;
static double *g_na_ptr[64] = {};
static unsigned long long g_na_ctx[64] = {};
static CtxGetCurrentFn g_ctx_current = nullptr;
static CtxGetIdFn g_ctx_id = nullptr;

static int na_scratch(double **out) {
    int dev = 0;
    RAS_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return RAS_EINVAL;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_ctx_current || !g_ctx_id) {
        cudaDriverEntryPointQueryResult q1, q2;
        RAS_CK(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void **)&g_ctx_current, 12000, cudaEnableDefault, &q1));
        RAS_CK(cudaGetDriverEntryPointByVersion("cuCtxGetId", (void **)&g_ctx_id, 12000, cudaEnableDefault, &q2));
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess) {
            g_ctx_current = nullptr;
            g_ctx_id = nullptr;
            return RAS_ECUDA;
        }
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    const bool known = g_ctx_current(&ctx) == CUDA_SUCCESS && ctx && g_ctx_id(ctx, &id) == CUDA_SUCCESS;
    if (!known || !g_na_ptr[dev] || g_na_ctx[dev] != id) {
        // cudaGetSymbolAddress also makes the device's primary context current
        void *p = nullptr;
        RAS_CK(cudaGetSymbolAddress(&p, g_na_partials));
        if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx || g_ctx_id(ctx, &id) != CUDA_SUCCESS) return RAS_ECUDA;
        g_na_ptr[dev] = static_cast<double *>(p);
        g_na_ctx[dev] = id;
    }
    *out = g_na_ptr[dev];
    return RAS_OK;
}

}  // namespace ras

using namespace ras;

extern "C" int ras_norm2_noalloc(const double *x, long long n, double *result, void *stream) {
    if (!result || n < 0 || (n > 0 && !x)) return RAS_EINVAL;
    if (n > NA_MAX_N) return RAS_EINVAL;
    double *scratch = nullptr;
    RAS_TRY(na_scratch(&scratch));
    cudaStream_t st = S(stream);
    k_na_partial<<<NA_BLOCKS, NA_THREADS, 0, st>>>(x, n, scratch);
    RAS_LAUNCHED();
    k_na_final<<<1, NA_THREADS, 0, st>>>(scratch, result);
    RAS_LAUNCHED();
    return RAS_OK;
}
