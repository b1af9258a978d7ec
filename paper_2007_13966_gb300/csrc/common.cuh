// Shared definitions of the GB300 RAS Newton-Krylov library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "ras.h"

namespace ras {

extern std::atomic<long long> g_launches;

void record_error(cudaError_t e, const char *what, const char *file, int line);

inline void counted() { g_launches.fetch_add(1, std::memory_order_relaxed); }

#define RAS_CK(x)                                                                  \
    do {                                                                           \
        cudaError_t e_ = (x);                                                      \
        if (e_ != cudaSuccess) {                                                   \
            ::ras::record_error(e_, #x, __FILE__, __LINE__);                       \
            return e_ == cudaErrorMemoryAllocation ? RAS_ENOMEM : RAS_ECUDA;       \
        }                                                                          \
    } while (0)

// after a kernel launch: count it and surface launch-configuration errors
#define RAS_LAUNCHED()                                                             \
    do {                                                                           \
        ::ras::counted();                                                          \
        RAS_CK(cudaGetLastError());                                                \
    } while (0)

#define RAS_TRY(...)                                                               \
    do {                                                                           \
        int s_ = (__VA_ARGS__);                                                    \
        if (s_ < 0) return s_;                                                     \
    } while (0)

template <typename T>
inline int dalloc(T **p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void **)p, n * sizeof(T) + 64);
    if (e != cudaSuccess) {
        record_error(e, "cudaMalloc", __FILE__, __LINE__);
        *p = nullptr;
        return RAS_ENOMEM;
    }
    return RAS_OK;
}

template <typename T>
inline void dfree(T *&p) {
    if (p) cudaFree((void *)p);
    p = nullptr;
}

inline cudaStream_t S(void *s) { return (cudaStream_t)s; }

// Deterministic reductions: a fixed grid of RED_BLOCKS blocks writes partial
// sums, a single block adds them in a fixed order.
constexpr int RED_BLOCKS = 608;   // 4 x 152 SMs
constexpr int RED_THREADS = 256;
constexpr int MAX_MDOT = 33;      // Krylov vectors per multi-dot (restart <= 32)

struct ReduceWs {
    double *partials = nullptr;   // [MAX_MDOT+1][RED_BLOCKS]
    double *out = nullptr;        // [2*MAX_MDOT+8] device results
    double *host = nullptr;       // pinned mirror of out
};

int reduce_ws_init(ReduceWs &ws);
void reduce_ws_free(ReduceWs &ws);

// y . x over n entries -> ws.out[slot] (device); no synchronisation
int dot_async(ReduceWs &ws, const double *x, const double *y, int n, int slot, cudaStream_t st);
// ||x||_2 returned on the host (synchronises)
int norm2_sync(ReduceWs &ws, const double *x, int n, double *out, cudaStream_t st);
int dot_sync(ReduceWs &ws, const double *x, const double *y, int n, double *out, cudaStream_t st);

// vector kernels
int vec_axpby(double *y, double a, const double *x, double b, int n, cudaStream_t st);  // y = a x + b y
int vec_copy(double *y, const double *x, int n, cudaStream_t st);
int vec_scale_dev(double *y, const double *x, const double *dev_scalar, int n, cudaStream_t st); // y = x / *s
int vec_set(double *y, double v, int n, cudaStream_t st);

// 7-point operator helpers
struct Stencil7 {
    const double *c[7];
};

int stencil_apply(const Stencil7 &A, int nx, int ny, int nz, const double *x, double *y,
                  cudaStream_t st);
// y = b - A x
int stencil_residual(const Stencil7 &A, int nx, int ny, int nz, const double *b, const double *x,
                     double *y, cudaStream_t st);

}  // namespace ras

// Full problem handle (declared here so that the Krylov / Newton drivers and the
// preconditioner can share workspaces).
struct ras_problem {
    int nx, ny, nz, N;
    double hx, hy, hz, V;
    double a, b, R, T, mu, inv_mu;
    int upwind = 0;       // face mobility of the upstream cell instead of the mean
    int conservative = 0; // accumulation V phi D_t(p/Z) instead of V phi c(p) D_t p
    double *rateQ = nullptr;  // fixed injection rates per cell (m^3/s), or null
    double ghz = 0.0;     // g hz W mu / (R T): rho g hz across a z face = ghz * mbar (rho = that / (g hz) * m)
    double *Tx = nullptr, *Ty = nullptr, *Tz = nullptr, *phi = nullptr;
    double *kx = nullptr, *ky = nullptr, *kz = nullptr;   // permeabilities (sensitivities)
    int nconn = 0;
    int *conn_ptr = nullptr;       // [N+1] CSR of connections per cell
    double *conn_p = nullptr, *conn_T = nullptr, *conn_m = nullptr;
    double *eos_m = nullptr, *eos_dm = nullptr;  // per-cell scratch of the residual
    // set by the EOS kernels when a cell (or a fixed connection pressure) has no
    // admissible root; mapped pinned host memory, read after a synchronisation
    int *noroot_h = nullptr, *noroot_d = nullptr;
    ras::ReduceWs red;
    // Krylov workspace (allocated on first use for the largest restart seen)
    int kr_m = 0;
    double *kV = nullptr, *kZ = nullptr, *kw = nullptr, *kr = nullptr;
    // Newton workspace
    bool nw_ready = false;
    double *nX[2] = {nullptr, nullptr}, *nF[2] = {nullptr, nullptr};
    double *nJ[2][7] = {};
    double *ns = nullptr, *nrhs = nullptr, *ntmp = nullptr;
};
