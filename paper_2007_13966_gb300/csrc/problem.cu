// Discrete problem: Peng-Robinson EOS per cell, two-point-flux residual and
// exact Jacobian with BDF1/BDF2 (Section 2), 7-point operator products and
// deterministic reductions.
#include "common.cuh"

#include <cstring>
#include <mutex>
#include <string>

namespace ras {

std::atomic<long long> g_launches{0};
static std::mutex g_err_mu;
static std::string g_last_error;

void record_error(cudaError_t e, const char *what, const char *file, int line) {
    std::lock_guard<std::mutex> lk(g_err_mu);
    char buf[512];
    snprintf(buf, sizeof buf, "%s failed at %s:%d: %s", what, file, line, cudaGetErrorString(e));
    g_last_error = buf;
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// block-wide sum in a fixed order; result valid in thread 0
__device__ __forceinline__ double block_sum(double v, double *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = 0; i < nw; ++i) s += sh[i];
    }
    __syncthreads();
    return s;
}

__global__ void k_dot_partial(const double *__restrict__ x, const double *__restrict__ y, int n,
                              double *__restrict__ partials) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        acc = fma(x[i], y[i], acc);
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// sums `nvec` rows of partials (row stride RED_BLOCKS) into out[slot0 + v]
__global__ void k_finalize(const double *__restrict__ partials, int nvec, double *__restrict__ out,
                           int slot0, int sqrt_last) {
    __shared__ double sh[32];
    for (int v = 0; v < nvec; ++v) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < RED_BLOCKS; i += blockDim.x) acc += partials[v * RED_BLOCKS + i];
        double s = block_sum(acc, sh);
        if (threadIdx.x == 0) out[slot0 + v] = (sqrt_last && v == nvec - 1) ? sqrt(s) : s;
    }
}

int reduce_ws_init(ReduceWs &ws) {
    RAS_TRY(dalloc(&ws.partials, (size_t)(MAX_MDOT + 2) * RED_BLOCKS));
    RAS_TRY(dalloc(&ws.out, 2 * MAX_MDOT + 8));
    RAS_CK(cudaMallocHost((void **)&ws.host, (2 * MAX_MDOT + 8) * sizeof(double)));
    return RAS_OK;
}

void reduce_ws_free(ReduceWs &ws) {
    dfree(ws.partials);
    dfree(ws.out);
    if (ws.host) cudaFreeHost(ws.host);
    ws.host = nullptr;
}

int dot_async(ReduceWs &ws, const double *x, const double *y, int n, int slot, cudaStream_t st) {
    k_dot_partial<<<RED_BLOCKS, RED_THREADS, 0, st>>>(x, y, n, ws.partials);
    RAS_LAUNCHED();
    k_finalize<<<1, RED_THREADS, 0, st>>>(ws.partials, 1, ws.out, slot, 0);
    RAS_LAUNCHED();
    return RAS_OK;
}

int dot_sync(ReduceWs &ws, const double *x, const double *y, int n, double *out, cudaStream_t st) {
    RAS_TRY(dot_async(ws, x, y, n, 0, st));
    RAS_CK(cudaMemcpyAsync(ws.host, ws.out, sizeof(double), cudaMemcpyDeviceToHost, st));
    RAS_CK(cudaStreamSynchronize(st));
    *out = ws.host[0];
    return RAS_OK;
}

int norm2_sync(ReduceWs &ws, const double *x, int n, double *out, cudaStream_t st) {
    double d;
    RAS_TRY(dot_sync(ws, x, x, n, &d, st));
    *out = std::sqrt(d);
    return RAS_OK;
}

// ---------------------------------------------------------------------------
// vector kernels
// ---------------------------------------------------------------------------

__global__ void k_axpby(double *__restrict__ y, double a, const double *__restrict__ x, double b,
                        int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        y[i] = (b == 0.0) ? a * x[i] : fma(a, x[i], b * y[i]);
}

__global__ void k_copy(double *__restrict__ y, const double *__restrict__ x, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = x[i];
}

__global__ void k_scale_dev(double *__restrict__ y, const double *__restrict__ x,
                            const double *__restrict__ s, int n) {
    const double inv = 1.0 / *s;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        y[i] = x[i] * inv;
}

__global__ void k_set(double *__restrict__ y, double v, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = v;
}

static inline int grid_for(int n, int threads = 256) {
    int g = (n + threads - 1) / threads;
    const int cap = 152 * 8;
    return g < 1 ? 1 : (g > cap ? cap : g);
}

int vec_axpby(double *y, double a, const double *x, double b, int n, cudaStream_t st) {
    k_axpby<<<grid_for(n), 256, 0, st>>>(y, a, x, b, n);
    RAS_LAUNCHED();
    return RAS_OK;
}
int vec_copy(double *y, const double *x, int n, cudaStream_t st) {
    k_copy<<<grid_for(n), 256, 0, st>>>(y, x, n);
    RAS_LAUNCHED();
    return RAS_OK;
}
int vec_scale_dev(double *y, const double *x, const double *s, int n, cudaStream_t st) {
    k_scale_dev<<<grid_for(n), 256, 0, st>>>(y, x, s, n);
    RAS_LAUNCHED();
    return RAS_OK;
}
int vec_set(double *y, double v, int n, cudaStream_t st) {
    k_set<<<grid_for(n), 256, 0, st>>>(y, v, n);
    RAS_LAUNCHED();
    return RAS_OK;
}

// ---------------------------------------------------------------------------
// 7-point operator: y = A x  /  y = b - A x
// ---------------------------------------------------------------------------

template <bool RESID>
__global__ void __launch_bounds__(256) k_stencil(Stencil7 A, int nx, int ny, int nz,
                                                 const double *__restrict__ b,
                                                 const double *__restrict__ x,
                                                 double *__restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    const int nxy = nx * ny;
    const int n = i + nx * (j + ny * k);
    double s = A.c[0][n] * x[n];
    if (i > 0) s = fma(A.c[1][n], x[n - 1], s);
    if (i < nx - 1) s = fma(A.c[2][n], x[n + 1], s);
    if (j > 0) s = fma(A.c[3][n], x[n - nx], s);
    if (j < ny - 1) s = fma(A.c[4][n], x[n + nx], s);
    if (k > 0) s = fma(A.c[5][n], x[n - nxy], s);
    if (k < nz - 1) s = fma(A.c[6][n], x[n + nxy], s);
    y[n] = RESID ? b[n] - s : s;
}

static inline dim3 stencil_grid(int nx, int ny, int nz, int threads) {
    return dim3((nx + threads - 1) / threads, ny, nz);
}

static inline int stencil_threads(int nx) { return nx >= 128 ? 128 : (nx >= 64 ? 64 : 32); }

int stencil_apply(const Stencil7 &A, int nx, int ny, int nz, const double *x, double *y,
                  cudaStream_t st) {
    const int t = stencil_threads(nx);
    k_stencil<false><<<stencil_grid(nx, ny, nz, t), t, 0, st>>>(A, nx, ny, nz, nullptr, x, y);
    RAS_LAUNCHED();
    return RAS_OK;
}

int stencil_residual(const Stencil7 &A, int nx, int ny, int nz, const double *b, const double *x,
                     double *y, cudaStream_t st) {
    const int t = stencil_threads(nx);
    k_stencil<true><<<stencil_grid(nx, ny, nz, t), t, 0, st>>>(A, nx, ny, nz, b, x, y);
    RAS_LAUNCHED();
    return RAS_OK;
}

// ---------------------------------------------------------------------------
// problem creation: face transmissibilities (harmonic average), connections
// ---------------------------------------------------------------------------

__global__ void k_transmissibility(int nx, int ny, int nz, double hx, double hy, double hz,
                                   const double *__restrict__ kx, const double *__restrict__ ky,
                                   const double *__restrict__ kz, double *__restrict__ Tx,
                                   double *__restrict__ Ty, double *__restrict__ Tz) {
    const int N = nx * ny * nz;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        const int i = n % nx, j = (n / nx) % ny, k = n / (nx * ny);
        // T_f = A_f / (h/(2 k_i) + h/(2 k_j))
        Tx[n] = (i < nx - 1) ? (hy * hz) / (hx / (2.0 * kx[n]) + hx / (2.0 * kx[n + 1])) : 0.0;
        Ty[n] = (j < ny - 1) ? (hx * hz) / (hy / (2.0 * ky[n]) + hy / (2.0 * ky[n + nx])) : 0.0;
        Tz[n] = (k < nz - 1) ? (hx * hy) / (hz / (2.0 * kz[n]) + hz / (2.0 * kz[n + nx * ny])) : 0.0;
    }
}

__global__ void k_conn_ptr(const int *__restrict__ cell, int nconn, int N, int *__restrict__ ptr) {
    // ptr[n] = first connection index with cell >= n (cells sorted)
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n <= N; n += gridDim.x * blockDim.x) {
        int lo = 0, hi = nconn;
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (cell[mid] < n) lo = mid + 1; else hi = mid;
        }
        ptr[n] = lo;
    }
}

// ---------------------------------------------------------------------------
// Peng-Robinson EOS per cell
// ---------------------------------------------------------------------------

struct EosConst {
    double alpha, beta;   // A = alpha p, B = beta p (alpha = a/(RT)^2, beta = b/(RT))
    double inv_mu;
};

// Largest real root of Z^3 + c2 Z^2 + c1 Z + c0 in FP32 (Cardano / trigonometric
// form), used as the starting point of FP64 Newton steps on the cubic.
__device__ __forceinline__ float cubic_root_f32(float c2, float c1, float c0) {
    const float P = c1 - c2 * c2 * (1.0f / 3.0f);
    const float Q = 2.0f * c2 * c2 * c2 * (1.0f / 27.0f) - c2 * c1 * (1.0f / 3.0f) + c0;
    const float disc = Q * Q * 0.25f + P * P * P * (1.0f / 27.0f);
    float t;
    if (disc > 0.0f) {
        const float s = sqrtf(disc);
        t = cbrtf(-0.5f * Q + s) + cbrtf(-0.5f * Q - s);
    } else {
        const float r = sqrtf(fmaxf(-P * (1.0f / 3.0f), 0.0f));
        float arg = (r > 0.0f) ? (-0.5f * Q) / (r * r * r) : 0.0f;
        arg = fminf(fmaxf(arg, -1.0f), 1.0f);
        t = 2.0f * r * cosf(acosf(arg) * (1.0f / 3.0f));
    }
    return t - c2 * (1.0f / 3.0f);
}

struct EosOut {
    double c, dc, m, dm;
    double Z;
    bool ok;   // an admissible root: Z finite, Z > B, f_Z != 0
};

__device__ __forceinline__ EosOut eos_cell(double p, const EosConst &E) {
    const double be = E.beta, al = E.alpha;
    const double A = al * p, B = be * p;
    const double c2 = -(1.0 - B);
    const double c1 = A - 3.0 * B * B - 2.0 * B;
    const double c0 = -(A * B - B * B - B * B * B);
    double Z = (double)cubic_root_f32((float)c2, (float)c1, (float)c0);
    // three FP64 Newton steps on the cubic (FP32 start is ~1e-7 accurate)
#pragma unroll
    for (int it = 0; it < 3; ++it) {
        const double f = ((Z + c2) * Z + c1) * Z + c0;
        const double fz = (3.0 * Z + 2.0 * c2) * Z + c1;
        Z -= f / fz;
    }
    // Root selection in FP64: the FP32 closed form decides between one and three
    // real roots in FP32, and near a pair of close roots it can start Newton on
    // another root than the largest. The other two roots solve the deflated
    // quadratic t^2 + (c2 + Z) t + (c1 + (c2 + Z) Z) = 0; if it has a real root
    // above Z, that root is the largest: take it and polish it.
    {
        const double q1 = c2 + Z, q0 = c1 + q1 * Z;
        const double dq = q1 * q1 - 4.0 * q0;
        if (dq >= 0.0) {
            double Zq = 0.5 * (-q1 + sqrt(dq));
            if (Zq > Z) {
#pragma unroll
                for (int it = 0; it < 2; ++it) {
                    const double f = ((Zq + c2) * Zq + c1) * Zq + c0;
                    const double fz = (3.0 * Zq + 2.0 * c2) * Zq + c1;
                    const double step = f / fz;
                    if (isfinite(step)) Zq -= step;
                }
                Z = Zq;
            }
        }
    }
    // partial derivatives of f(Z, p) with A = alpha p, B = beta p
    const double fZ = 3.0 * Z * Z - 2.0 * (1.0 - B) * Z + (A - 3.0 * B * B - 2.0 * B);
    const double fp = be * Z * Z + (al - 6.0 * be * B - 2.0 * be) * Z
                      - (2.0 * al * B - 2.0 * be * B - 3.0 * be * B * B);
    const double fZZ = 6.0 * Z - 2.0 * (1.0 - B);
    const double fZp = 2.0 * be * Z + (al - 6.0 * be * B - 2.0 * be);
    const double fpp = -6.0 * be * be * Z - (2.0 * al * be - 2.0 * be * be - 6.0 * be * be * B);
    const double ifZ = 1.0 / fZ;
    const double dZ = -fp * ifZ;                                   // dZ/dp
    const double d2Z = -(fZZ * dZ * dZ + 2.0 * fZp * dZ + fpp) * ifZ;
    const double iZ = 1.0 / Z;
    const double iZ2 = iZ * iZ;
    EosOut o;
    o.c = iZ - p * dZ * iZ2;                                       // (p/Z)(1/p - Z'/Z)
    o.dc = -2.0 * dZ * iZ2 - p * d2Z * iZ2 + 2.0 * p * dZ * dZ * iZ2 * iZ;
    o.m = p * iZ * E.inv_mu;                                       // p / (mu Z)
    o.dm = o.c * E.inv_mu;
    o.Z = Z;
    o.ok = isfinite(Z) && Z > B && fZ != 0.0 && isfinite(o.c) && isfinite(o.dc);
    return o;
}

// pass 1: per-cell storage term and its derivative, and m, dm for the fluxes.
// Accumulation V phi c(p) D_t p (Eq. gover_sys), or in the conservative form
// V phi D_t(p/Z) with the same BDF weights on p/Z at the three levels (d(p/Z)/dp = c);
// fixed injection rates subtract (p/Z) Q from the cell's residual.
__global__ void __launch_bounds__(256) k_eos_storage(
    int N, EosConst E, double Vol, double inv_dt, int order, const double *__restrict__ p,
    const double *__restrict__ pl, const double *__restrict__ plm1, const double *__restrict__ phi,
    double *__restrict__ F, double *__restrict__ Jc, double *__restrict__ m_out,
    double *__restrict__ dm_out, int *__restrict__ noroot, int conservative,
    const double *__restrict__ rateQ) {
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        const double pn = p[n];
        EosOut o = eos_cell(pn, E);
        const double g = order == 1 ? inv_dt : 1.5 * inv_dt;
        const double vp = Vol * phi[n];
        double f, jc;
        if (conservative) {
            const EosOut ol = eos_cell(pl[n], E);
            if (!ol.ok) o.ok = false;
            double DtP;
            if (order == 1) {
                DtP = (pn / o.Z - pl[n] / ol.Z) * inv_dt;
            } else {
                const EosOut om = eos_cell(plm1[n], E);
                if (!om.ok) o.ok = false;
                DtP = (3.0 * (pn / o.Z) - 4.0 * (pl[n] / ol.Z) + plm1[n] / om.Z) * (0.5 * inv_dt);
            }
            f = vp * DtP;
            jc = vp * o.c * g;
        } else {
            const double Dt = order == 1 ? (pn - pl[n]) * inv_dt
                                         : (3.0 * pn - 4.0 * pl[n] + plm1[n]) * (0.5 * inv_dt);
            f = vp * o.c * Dt;
            jc = vp * (o.dc * Dt + o.c * g);
        }
        if (rateQ) {
            const double q = rateQ[n];
            f -= (pn / o.Z) * q;
            jc -= o.c * q;
        }
        if (!o.ok) {   // no admissible root: flag it and poison the cell's residual
            *noroot = 1;
            f = jc = o.m = o.dm = __longlong_as_double(0x7ff8000000000000LL);
        }
        F[n] = f;
        if (Jc) Jc[n] = jc;
        m_out[n] = o.m;
        dm_out[n] = o.dm;
    }
}

struct JacOut {
    double *c[7];
};

// pass 2: two-point fluxes, connections, Jacobian rows. Row order of the sum:
// storage, +x, -x, +y, -y, +z, -z, connections.
template <bool WANT_J>
__global__ void __launch_bounds__(128) k_flux(
    int nx, int ny, int nz, const double *__restrict__ p, const double *__restrict__ m,
    const double *__restrict__ dm, const double *__restrict__ Tx, const double *__restrict__ Ty,
    const double *__restrict__ Tz, const int *__restrict__ conn_ptr,
    const double *__restrict__ conn_p, const double *__restrict__ conn_T,
    const double *__restrict__ conn_m, double ghz, int upwind, double *__restrict__ F, JacOut J) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    const int nxy = nx * ny;
    const int n = i + nx * (j + ny * k);
    const double pn = p[n], mn = m[n], dmn = dm[n];
    double f = F[n];
    double jc = WANT_J ? J.c[0][n] : 0.0;
    double jn[6] = {0, 0, 0, 0, 0, 0};
    // potential difference p_n - p_q - rhobar g (h_n - h_q), rhobar g hz = ghz * mbar;
    // gz: +1 towards the deeper neighbour (+z), -1 towards the shallower, 0 level faces
    // face mobility: the mean, or the upstream cell's (weights wn, wq of m_n, m_q)
    auto face = [&](double T, int q, int slot, double gz) {
        const double mq = m[q], mbar = 0.5 * (mn + mq);
        const double gh = gz * ghz;
        const double dphi = (pn - p[q]) + gh * mbar;
        const bool up_n = dphi >= 0.0;
        const double mf = upwind ? (up_n ? mn : mq) : mbar;
        const double wn = upwind ? (up_n ? 1.0 : 0.0) : 0.5, wq = upwind ? 1.0 - wn : 0.5;
        f += T * mf * dphi;
        if (WANT_J) {
            jc += T * (wn * dmn * dphi + mf * (1.0 + 0.5 * gh * dmn));
            jn[slot] = T * (wq * dm[q] * dphi + mf * (-1.0 + 0.5 * gh * dm[q]));
        }
    };
    if (i < nx - 1) face(Tx[n], n + 1, 1, 0.0);
    if (i > 0) face(Tx[n - 1], n - 1, 0, 0.0);
    if (j < ny - 1) face(Ty[n], n + nx, 3, 0.0);
    if (j > 0) face(Ty[n - nx], n - nx, 2, 0.0);
    if (k < nz - 1) face(Tz[n], n + nxy, 5, 1.0);
    if (k > 0) face(Tz[n - nxy], n - nxy, 4, -1.0);
    for (int q = conn_ptr[n]; q < conn_ptr[n + 1]; ++q) {
        const double dp = pn - conn_p[q];
        const double mf = upwind ? (dp >= 0.0 ? mn : conn_m[q]) : 0.5 * (mn + conn_m[q]);
        const double wn = upwind ? (dp >= 0.0 ? 1.0 : 0.0) : 0.5;
        f += conn_T[q] * mf * dp;
        if (WANT_J) jc += conn_T[q] * (wn * dmn * dp + mf);
    }
    F[n] = f;
    if (WANT_J) {
        J.c[0][n] = jc;
#pragma unroll
        for (int s = 0; s < 6; ++s) J.c[s + 1][n] = jn[s];
    }
}

__global__ void k_conn_mobility(int nconn, EosConst E, const double *__restrict__ cp,
                                double *__restrict__ cm, int *__restrict__ noroot) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nconn; q += gridDim.x * blockDim.x) {
        const EosOut o = eos_cell(cp[q], E);
        if (!o.ok) *noroot = 1;
        cm[q] = o.m;
    }
}

// ---------------------------------------------------------------------------
// discrete adjoint of the time loop (no counterpart in the paper): J^T as a
// 7-point operator, the adjoint right-hand side with the BDF2 history terms,
// and (dF/dtheta)^T lambda for per-cell log-permeability multipliers theta
// ---------------------------------------------------------------------------

// JT[s][n] = J[opp(s)][neighbour s of n]: (J^T)_{n, n-1} = dF_{n-1}/dp_n = J[+x][n-1], ...
__global__ void __launch_bounds__(256) k_stencil_transpose(int nx, int ny, int nz, JacOut J,
                                                           JacOut JT) {
    const int N = nx * ny * nz, nxy = nx * ny;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        const int i = n % nx, j = (n / nx) % ny, k = n / nxy;
        JT.c[0][n] = J.c[0][n];
        JT.c[1][n] = i > 0 ? J.c[2][n - 1] : 0.0;
        JT.c[2][n] = i < nx - 1 ? J.c[1][n + 1] : 0.0;
        JT.c[3][n] = j > 0 ? J.c[4][n - nx] : 0.0;
        JT.c[4][n] = j < ny - 1 ? J.c[3][n + nx] : 0.0;
        JT.c[5][n] = k > 0 ? J.c[6][n - nxy] : 0.0;
        JT.c[6][n] = k < nz - 1 ? J.c[5][n + nxy] : 0.0;
    }
}

// rhs = -dphi + c1 s(p1) lam1 + c2 s(p2) lam2 with s(p) = V phi c(p); a term
// whose state is null is absent
__global__ void __launch_bounds__(256) k_adjoint_rhs(int N, EosConst E, double Vol,
                                                     const double *__restrict__ phi,
                                                     const double *__restrict__ dphi,
                                                     const double *__restrict__ p1,
                                                     const double *__restrict__ l1, double c1,
                                                     const double *__restrict__ p2,
                                                     const double *__restrict__ l2, double c2,
                                                     double *__restrict__ rhs) {
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        double r = dphi ? -dphi[n] : 0.0;
        if (p1) r += c1 * Vol * phi[n] * eos_cell(p1[n], E).c * l1[n];
        if (p2) r += c2 * Vol * phi[n] * eos_cell(p2[n], E).c * l2[n];
        rhs[n] = r;
    }
}

__global__ void __launch_bounds__(256) k_mobility(int N, EosConst E, const double *__restrict__ p,
                                                  double *__restrict__ m) {
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x)
        m[n] = eos_cell(p[n], E).m;
}

// grad_n += sum over the faces of n of (lam_n - lam_q) T mbar (p_n - p_q) k_q / (k_n + k_q)
//           + sum over the connections of n of lam_n T_c mbar (p_n - p_c)
// (dT_f / dtheta_n = T_f k_q / (k_n + k_q) for the harmonic face transmissibility,
// k along the face's axis; connection transmissibilities scale with k_n)
__global__ void __launch_bounds__(256) k_grad_logk(
    int nx, int ny, int nz, const double *__restrict__ p, const double *__restrict__ m,
    const double *__restrict__ lam, const double *__restrict__ kx, const double *__restrict__ ky,
    const double *__restrict__ kz, const double *__restrict__ Tx, const double *__restrict__ Ty,
    const double *__restrict__ Tz, const int *__restrict__ conn_ptr,
    const double *__restrict__ conn_p, const double *__restrict__ conn_T,
    const double *__restrict__ conn_m, double ghz, int upwind, double *__restrict__ grad) {
    const int N = nx * ny * nz, nxy = nx * ny;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        const int i = n % nx, j = (n / nx) % ny, k = n / nxy;
        const double pn = p[n], mn = m[n], ln = lam[n];
        double g = 0.0;
        auto face = [&](double T, int q, const double *ka, double gz) {
            const double mbar = 0.5 * (mn + m[q]);
            const double dphi = (pn - p[q]) + gz * ghz * mbar;
            const double mf = upwind ? (dphi >= 0.0 ? mn : m[q]) : mbar;
            const double flux = T * mf * dphi;   // the residual's face flux
            g += (ln - lam[q]) * flux * ka[q] / (ka[n] + ka[q]);
        };
        if (i < nx - 1) face(Tx[n], n + 1, kx, 0.0);
        if (i > 0) face(Tx[n - 1], n - 1, kx, 0.0);
        if (j < ny - 1) face(Ty[n], n + nx, ky, 0.0);
        if (j > 0) face(Ty[n - nx], n - nx, ky, 0.0);
        if (k < nz - 1) face(Tz[n], n + nxy, kz, 1.0);
        if (k > 0) face(Tz[n - nxy], n - nxy, kz, -1.0);
        for (int q = conn_ptr[n]; q < conn_ptr[n + 1]; ++q) {
            const double dp = pn - conn_p[q];
            const double mf = upwind ? (dp >= 0.0 ? mn : conn_m[q]) : 0.5 * (mn + conn_m[q]);
            g += ln * (conn_T[q] * mf * dp);
        }
        grad[n] += g;
    }
}

// reads and clears the problem's no-admissible-root flag (the stream must have
// been synchronised after the kernels that may set it)
bool noroot_take(ras_problem *P) {
    if (!P->noroot_h || !*reinterpret_cast<volatile int *>(P->noroot_h)) return false;
    *reinterpret_cast<volatile int *>(P->noroot_h) = 0;
    return true;
}

static EosConst eos_const(const ras_problem *P) {
    EosConst E;
    E.alpha = P->a / (P->R * P->R * P->T * P->T);
    E.beta = P->b / (P->R * P->T);
    E.inv_mu = 1.0 / P->mu;
    return E;
}

}  // namespace ras

using namespace ras;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

static double acentric_factor(double Tc, double pc, double Tb) {
    const double Tbr = Tb / Tc, tau = 1.0 - Tbr;
    const double f0 = (-5.97616 * tau + 1.29874 * pow(tau, 1.5) - 0.60394 * pow(tau, 2.5)
                       - 1.06841 * pow(tau, 5.0)) / Tbr;
    const double f1 = (-5.03365 * tau + 1.11505 * pow(tau, 1.5) - 5.41217 * pow(tau, 2.5)
                       - 7.46628 * pow(tau, 5.0)) / Tbr;
    return (-log(pc / 101325.0) - f0) / f1;
}

extern "C" int ras_problem_create(const ras_grid *grid, const ras_eos *eos, const ras_rock *rock,
                                  void *stream, ras_problem **out) {
    if (!grid || !eos || !rock || !out) return RAS_EINVAL;
    *out = nullptr;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return RAS_EINVAL;
    if (!(grid->hx > 0 && grid->hy > 0 && grid->hz > 0)) return RAS_EINVAL;
    if (!std::isfinite(grid->gz) || (grid->gz != 0.0 && !(eos->W > 0 && std::isfinite(eos->W)))) return RAS_EINVAL;
    if (grid->upwind != 0 && grid->upwind != 1) return RAS_EINVAL;
    if (grid->conservative != 0 && grid->conservative != 1) return RAS_EINVAL;
    const long long N = (long long)grid->nx * grid->ny * grid->nz;
    if (N > (1LL << 30)) return RAS_EINVAL;
    if (!rock->kx || !rock->ky || !rock->kz || !rock->phi) return RAS_EINVAL;
    if (rock->nconn < 0 || (rock->nconn > 0 && (!rock->conn_cell || !rock->conn_p || !rock->conn_T)))
        return RAS_EINVAL;
    if (!(eos->T > 0 && eos->R > 0 && eos->mu > 0 && eos->Tc > 0 && eos->pc > 0)) return RAS_EINVAL;
    cudaStream_t st = S(stream);
    ras_problem *P = new ras_problem();
    P->nx = grid->nx; P->ny = grid->ny; P->nz = grid->nz; P->N = (int)N;
    P->hx = grid->hx; P->hy = grid->hy; P->hz = grid->hz;
    P->V = grid->hx * grid->hy * grid->hz;
    P->R = eos->R; P->T = eos->T; P->mu = eos->mu; P->inv_mu = 1.0 / eos->mu;
    P->ghz = grid->gz * grid->hz * eos->W * eos->mu / (eos->R * eos->T);
    P->upwind = grid->upwind;
    P->conservative = grid->conservative;
    // Eq. attrfactor and the m(omega) fit (first branch at omega = 0.491)
    const double omega = eos->omega_from_Tb ? acentric_factor(eos->Tc, eos->pc, eos->Tb) : eos->omega;
    const double mfit = omega <= 0.491 ? 0.37464 + 1.54226 * omega - 0.26992 * omega * omega
                                       : 0.3796 + 1.485 * omega - 0.1644 * omega * omega +
                                             0.01667 * omega * omega * omega;
    const double sq = 1.0 + mfit * (1.0 - sqrt(eos->T / eos->Tc));
    P->a = 0.45724 * eos->R * eos->R * eos->Tc * eos->Tc / eos->pc * sq * sq;
    P->b = 0.0778 * eos->R * eos->Tc / eos->pc;
    int rc = RAS_OK;
    auto fail = [&](int s) { ras_problem_destroy(P); return s; };
    if ((rc = dalloc(&P->Tx, N)) || (rc = dalloc(&P->Ty, N)) || (rc = dalloc(&P->Tz, N)) ||
        (rc = dalloc(&P->phi, N)) || (rc = dalloc(&P->eos_m, N)) || (rc = dalloc(&P->eos_dm, N)) ||
        (rc = dalloc(&P->conn_ptr, N + 1)) || (rc = dalloc(&P->conn_p, rock->nconn)) ||
        (rc = dalloc(&P->conn_T, rock->nconn)) || (rc = dalloc(&P->conn_m, rock->nconn)) ||
        (rc = dalloc(&P->kx, N)) || (rc = dalloc(&P->ky, N)) || (rc = dalloc(&P->kz, N)) ||
        (rock->rate_Q && (rc = dalloc(&P->rateQ, N))))
        return fail(rc);
    if ((rc = reduce_ws_init(P->red))) return fail(rc);
    if (cudaHostAlloc((void **)&P->noroot_h, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&P->noroot_d, P->noroot_h, 0) != cudaSuccess)
        return fail(RAS_ENOMEM);
    *P->noroot_h = 0;
    P->nconn = rock->nconn;
    int *cell = nullptr;
    if ((rc = dalloc(&cell, rock->nconn))) return fail(rc);
    auto ck = [&](cudaError_t e) {
        if (e != cudaSuccess) record_error(e, "problem_create", __FILE__, __LINE__);
        return e == cudaSuccess;
    };
    bool ok = ck(cudaMemcpyAsync(P->phi, rock->phi, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    ok = ok && ck(cudaMemcpyAsync(P->kx, rock->kx, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    ok = ok && ck(cudaMemcpyAsync(P->ky, rock->ky, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    ok = ok && ck(cudaMemcpyAsync(P->kz, rock->kz, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (rock->rate_Q)
        ok = ok && ck(cudaMemcpyAsync(P->rateQ, rock->rate_Q, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (rock->nconn > 0) {
        ok = ok && ck(cudaMemcpyAsync(cell, rock->conn_cell, rock->nconn * sizeof(int),
                                      cudaMemcpyDeviceToDevice, st));
        ok = ok && ck(cudaMemcpyAsync(P->conn_p, rock->conn_p, rock->nconn * sizeof(double),
                                      cudaMemcpyDeviceToDevice, st));
        ok = ok && ck(cudaMemcpyAsync(P->conn_T, rock->conn_T, rock->nconn * sizeof(double),
                                      cudaMemcpyDeviceToDevice, st));
    }
    if (!ok) { dfree(cell); return fail(RAS_ECUDA); }
    k_transmissibility<<<grid_for((int)N), 256, 0, st>>>(P->nx, P->ny, P->nz, P->hx, P->hy, P->hz,
                                                          rock->kx, rock->ky, rock->kz, P->Tx, P->Ty,
                                                          P->Tz);
    counted();
    k_conn_ptr<<<grid_for((int)N + 1), 256, 0, st>>>(cell, rock->nconn, (int)N, P->conn_ptr);
    counted();
    if (rock->nconn > 0) {
        k_conn_mobility<<<grid_for(rock->nconn), 256, 0, st>>>(rock->nconn, eos_const(P), P->conn_p,
                                                               P->conn_m, P->noroot_d);
        counted();
    }
    ok = ck(cudaGetLastError()) && ck(cudaStreamSynchronize(st));
    dfree(cell);
    if (!ok) return fail(RAS_ECUDA);
    if (noroot_take(P)) return fail(RAS_ENOROOT);   // a fixed connection pressure has no admissible Z
    *out = P;
    return RAS_OK;
}

extern "C" void ras_problem_destroy(ras_problem *P) {
    if (!P) return;
    dfree(P->Tx); dfree(P->Ty); dfree(P->Tz); dfree(P->phi);
    dfree(P->kx); dfree(P->ky); dfree(P->kz); dfree(P->rateQ);
    dfree(P->eos_m); dfree(P->eos_dm);
    dfree(P->conn_ptr); dfree(P->conn_p); dfree(P->conn_T); dfree(P->conn_m);
    reduce_ws_free(P->red);
    dfree(P->kV); dfree(P->kZ); dfree(P->kw); dfree(P->kr);
    for (int b = 0; b < 2; ++b) {
        dfree(P->nX[b]); dfree(P->nF[b]);
        for (int s = 0; s < 7; ++s) dfree(P->nJ[b][s]);
    }
    dfree(P->ns); dfree(P->nrhs); dfree(P->ntmp);
    if (P->noroot_h) cudaFreeHost(P->noroot_h);
    delete P;
}

namespace ras {
int residual_eval_impl(ras_problem *P, const double *p, const double *pl, const double *plm1,
                       double dt, int order, double *F, double *const *J, cudaStream_t st) {
    const EosConst E = eos_const(P);
    k_eos_storage<<<grid_for(P->N), 256, 0, st>>>(P->N, E, P->V, 1.0 / dt, order, p, pl,
                                                   order == 2 ? plm1 : pl, P->phi, F,
                                                   J ? J[0] : nullptr, P->eos_m, P->eos_dm,
                                                   P->noroot_d, P->conservative, P->rateQ);
    RAS_LAUNCHED();
    const int t = stencil_threads(P->nx);
    const dim3 g = stencil_grid(P->nx, P->ny, P->nz, t);
    JacOut jo;
    for (int s = 0; s < 7; ++s) jo.c[s] = J ? J[s] : nullptr;
    if (J) {
        k_flux<true><<<g, t, 0, st>>>(P->nx, P->ny, P->nz, p, P->eos_m, P->eos_dm, P->Tx, P->Ty,
                                      P->Tz, P->conn_ptr, P->conn_p, P->conn_T, P->conn_m, P->ghz, P->upwind, F, jo);
    } else {
        k_flux<false><<<g, t, 0, st>>>(P->nx, P->ny, P->nz, p, P->eos_m, P->eos_dm, P->Tx, P->Ty,
                                       P->Tz, P->conn_ptr, P->conn_p, P->conn_T, P->conn_m, P->ghz, P->upwind, F, jo);
    }
    RAS_LAUNCHED();
    return RAS_OK;
}
}  // namespace ras

extern "C" int residual_eval(ras_problem *P, const double *p, const double *p_l,
                             const double *p_lm1, double dt, int bdf_order, double *F,
                             const ras_stencil *J, double *normF, void *stream) {
    if (!P || !p || !p_l || !F || !(dt > 0) || (bdf_order != 1 && bdf_order != 2)) return RAS_EINVAL;
    if (bdf_order == 2 && !p_lm1) return RAS_EINVAL;
    if (J) for (int s = 0; s < 7; ++s) if (!J->c[s]) return RAS_EINVAL;
    cudaStream_t st = S(stream);
    RAS_TRY(residual_eval_impl(P, p, p_l, p_lm1, dt, bdf_order, F, J ? J->c : nullptr, st));
    if (normF) {
        RAS_TRY(norm2_sync(P->red, F, P->N, normF, st));
        if (noroot_take(P)) return RAS_ENOROOT;
        if (!std::isfinite(*normF)) return RAS_ENAN;
    }
    return RAS_OK;
}

extern "C" int ras_stencil_matvec(const ras_problem *P, const ras_stencil *J, const double *x,
                                  double *y, void *stream) {
    if (!P || !J || !x || !y || x == y) return RAS_EINVAL;
    Stencil7 A;
    for (int s = 0; s < 7; ++s) {
        if (!J->c[s]) return RAS_EINVAL;
        A.c[s] = J->c[s];
    }
    return stencil_apply(A, P->nx, P->ny, P->nz, x, y, S(stream));
}

extern "C" const char *ras_status_string(int s) {
    switch (s) {
        case RAS_OK: return "ok";
        case RAS_GMRES_MAXIT: return "FGMRES reached its iteration limit";
        case RAS_NEWTON_MAXIT: return "Newton reached its iteration limit";
        case RAS_LINESEARCH_FAIL: return "line search: step length below the minimum";
        case RAS_EINVAL: return "invalid argument";
        case RAS_ECUDA: return "CUDA runtime error";
        case RAS_ENOMEM: return "device out of memory";
        case RAS_ENAN: return "NaN or Inf detected";
        case RAS_EZEROPIVOT: return "zero or non-finite pivot";
        case RAS_ENOROOT: return "no admissible EOS root";
        case RAS_ETIMEOUT: return "bounded device wait timed out";
        default: return "unknown status";
    }
}

extern "C" long long ras_kernel_launches(void) { return g_launches.load(); }

extern "C" const char *ras_last_error(void) {
    std::lock_guard<std::mutex> lk(ras::g_err_mu);
    return ras::g_last_error.c_str();
}

extern "C" int ras_stencil_transpose(const ras_problem *P, const ras_stencil *J, ras_stencil *JT,
                                     void *stream) {
    if (!P || !J || !JT) return RAS_EINVAL;
    for (int s = 0; s < 7; ++s) {
        if (!J->c[s] || !JT->c[s]) return RAS_EINVAL;
        for (int t = 0; t < 7; ++t) if (J->c[s] == JT->c[t]) return RAS_EINVAL;   // no aliasing
    }
    JacOut a, b;
    for (int s = 0; s < 7; ++s) { a.c[s] = J->c[s]; b.c[s] = JT->c[s]; }
    k_stencil_transpose<<<grid_for(P->N), 256, 0, S(stream)>>>(P->nx, P->ny, P->nz, a, b);
    RAS_LAUNCHED();
    return RAS_OK;
}

extern "C" int ras_adjoint_rhs(const ras_problem *P, const double *dphi, const double *p1,
                               const double *lam1, double c1, const double *p2,
                               const double *lam2, double c2, double *rhs, void *stream) {
    if (!P || !rhs || (p1 && !lam1) || (p2 && !lam2)) return RAS_EINVAL;
    k_adjoint_rhs<<<grid_for(P->N), 256, 0, S(stream)>>>(P->N, eos_const(P), P->V, P->phi, dphi,
                                                          p1, lam1, c1, p2, lam2, c2, rhs);
    RAS_LAUNCHED();
    return RAS_OK;
}

extern "C" int ras_grad_logk(ras_problem *P, const double *p, const double *lam, double *grad,
                             void *stream) {
    if (!P || !p || !lam || !grad) return RAS_EINVAL;
    cudaStream_t st = S(stream);
    k_mobility<<<grid_for(P->N), 256, 0, st>>>(P->N, eos_const(P), p, P->eos_m);
    RAS_LAUNCHED();
    k_grad_logk<<<grid_for(P->N), 256, 0, st>>>(P->nx, P->ny, P->nz, p, P->eos_m, lam, P->kx, P->ky,
                                                 P->kz, P->Tx, P->Ty, P->Tz, P->conn_ptr, P->conn_p,
                                                 P->conn_T, P->conn_m, P->ghz, P->upwind, grad);
    RAS_LAUNCHED();
    return RAS_OK;
}
