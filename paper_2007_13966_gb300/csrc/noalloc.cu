// ||x||_2 without any allocation: a variant of the deterministic norm
// reduction used by residual_eval (and the Krylov / Newton norms) whose
// partial-sum scratch lives in a static device array compiled into the
// library instead of a buffer the library allocates.
//
// Who needs it: code that must not allocate device memory at call time, for
// example a caller that owns all device memory through its own pool (a
// framework caching allocator, where raw cudaMalloc/cudaFree behind its back
// fragments memory or fails under its budget), a caller that records work
// into a CUDA stream capture (cudaMalloc is not a capturable operation), or a
// latency-critical loop that cannot afford an allocation or its failure.
#include "common.cuh"

#include <mutex>

namespace ras {

// one partial sum per block of the reduction grid; every call overwrites all
// NA_BLOCKS entries before reading them, so nothing has to start at zero
constexpr int NA_BLOCKS = 608;
constexpr int NA_THREADS = 256;
constexpr long long NA_MAX_N = 2147483647LL;   // int32 element index range

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

__global__ void __launch_bounds__(NA_THREADS) k_na_partial(const double *__restrict__ x, int n,
                                                           double *__restrict__ partials) {
    __shared__ double sh[NA_THREADS / 32];
    double acc = 0.0;
    for (int i = blockIdx.x * NA_THREADS + threadIdx.x; i < n; i += NA_BLOCKS * NA_THREADS)
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

// Device address of g_na_partials for each device, looked up once per device
// with that device current (the host-side symbol is only a stand-in).
static std::mutex g_na_mu;
static double *g_na_ptr[64] = {};

static int na_scratch(double **out) {
    int dev = 0;
    RAS_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return RAS_EINVAL;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        RAS_CK(cudaGetSymbolAddress(&p, g_na_partials));
        g_na_ptr[dev] = static_cast<double *>(p);
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
    k_na_partial<<<NA_BLOCKS, NA_THREADS, 0, st>>>(x, (int)n, scratch);
    RAS_LAUNCHED();
    k_na_final<<<1, NA_THREADS, 0, st>>>(scratch, result);
    RAS_LAUNCHED();
    return RAS_OK;
}
