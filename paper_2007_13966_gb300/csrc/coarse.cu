// Coarse-grid correction of the two-level Schwarz preconditioners
// (Section 3.2): interpolation I_0^1 (Eq. equ:inter-second, tensor-product
// linear between cell-centred coarse centres), restriction R = P^T, the
// Galerkin coarse operator A_c = R A P (125-point stencil) and its exact solve
// by a dense block LU.
//
// Dense block LU: coarse cells are renumbered with the axes sorted by size
// (fastest = smallest). A_c couples cells at most two cells apart, so two
// consecutive planes of the slowest axis form one dense block of size T and
// A_c is block tridiagonal: A = tridiag(Lo_{k-1}, D_k, Up_k). Block Thomas:
//     D_0 = A_00,  E_k = D_k^{-1},  C_k = Lo_k E_k,  F_k = E_k Up_k,
//     D_{k+1} = A_{k+1,k+1} - C_k Up_k.
// Solve: g_k -= C_{k-1} g_{k-1} (forward), x_k = E_k g_k - F_k x_{k+1}.
// Each E_k is computed in place by a blocked Gauss-Jordan inversion without
// pivoting (64 x 64 tiles); Lo_k / Up_k are sparse and stored in ELL form.
#include "precond.cuh"

#include <algorithm>
#include <numeric>

namespace ras {

constexpr int TILE = 64;
constexpr int ELLW = 64;   // max couplings of one cell into the neighbouring block (<= 50)

struct Coarse {
    int prec = 64;
    int nx, ny, nz, N;
    int n[3], r[3], c[3], Nc;
    int *d_ia[3] = {}, *d_ib[3] = {};
    double *d_wa[3] = {}, *d_wb[3] = {};
    int *d_lo[3] = {}, *d_hi[3] = {};
    int af, am, as;                 // axis order: fastest, middle, slowest
    int T = 0, nb = 0;              // block size (multiple of TILE), number of blocks
    int *d_pos = nullptr;           // natural coarse index -> block position
    int *d_cell = nullptr;          // block position -> natural coarse index or -1
    void *Ac = nullptr;             // [125][Nc] Galerkin stencil (prec)
    void *D = nullptr, *C = nullptr, *F = nullptr;   // [nb][T][T]
    int *lo_q = nullptr, *up_q = nullptr;            // ELL column / row indices
    void *lo_v = nullptr, *up_v = nullptr;           // ELL values
    void *g = nullptr, *x = nullptr;                 // [nb*T]
    int *d_err = nullptr;
    size_t esz = 8;
};

// ---------------------------------------------------------------------------
// geometry helpers (device)
// ---------------------------------------------------------------------------

struct Interp {
    const int *ia[3], *ib[3];
    const double *wa[3], *wb[3];
    const int *lo[3], *hi[3];
};

__device__ __forceinline__ double w1(const Interp &P, int ax, int a, int I) {
    double w = 0.0;
    if (P.ia[ax][a] == I) w += P.wa[ax][a];
    if (P.ib[ax][a] == I) w += P.wb[ax][a];
    return w;
}

struct CGeom {
    int nx, ny, nz;       // fine
    int cx, cy, cz, Nc;   // coarse
    int T, nb;
};

// ---------------------------------------------------------------------------
// Galerkin product A_c[I][I + d] = sum_s sum_a P(a,I) A_s(a) P(a + e_s, I + d)
// ---------------------------------------------------------------------------

template <typename AT>
__global__ void __launch_bounds__(128) k_rap(Stencil7 A, Interp P, CGeom G, AT *__restrict__ Ac) {
    const int I = blockIdx.x;
    const int t = threadIdx.x;
    if (t >= 125) return;
    const int dx = t % 5 - 2, dy = (t / 5) % 5 - 2, dz = t / 25 - 2;
    const int Ix = I % G.cx, Iy = (I / G.cx) % G.cy, Iz = I / (G.cx * G.cy);
    const int Jx = Ix + dx, Jy = Iy + dy, Jz = Iz + dz;
    AT acc = 0;
    if (Jx >= 0 && Jx < G.cx && Jy >= 0 && Jy < G.cy && Jz >= 0 && Jz < G.cz) {
        const int nx = G.nx, nxy = G.nx * G.ny;
#pragma unroll 1
        for (int s = 0; s < 7; ++s) {
            // stencil term s: 0 centre, 1 -x, 2 +x, 3 -y, 4 +y, 5 -z, 6 +z
            const int sgn = (s & 1) ? -1 : 1;
            const int sx = (s == 1 || s == 2) ? sgn : 0;
            const int sy = (s == 3 || s == 4) ? sgn : 0;
            const int sz = (s == 5 || s == 6) ? sgn : 0;
            const int x0 = max(P.lo[0][Ix], P.lo[0][Jx] - sx), x1 = min(P.hi[0][Ix], P.hi[0][Jx] - sx);
            const int y0 = max(P.lo[1][Iy], P.lo[1][Jy] - sy), y1 = min(P.hi[1][Iy], P.hi[1][Jy] - sy);
            const int z0 = max(P.lo[2][Iz], P.lo[2][Jz] - sz), z1 = min(P.hi[2][Iz], P.hi[2][Jz] - sz);
            if (x0 >= x1 || y0 >= y1 || z0 >= z1) continue;
            const double *As = A.c[s];
            for (int az = z0; az < z1; ++az) {
                const AT wz = (AT)(w1(P, 2, az, Iz) * w1(P, 2, az + sz, Jz));
                for (int ay = y0; ay < y1; ++ay) {
                    const AT wyz = wz * (AT)(w1(P, 1, ay, Iy) * w1(P, 1, ay + sy, Jy));
                    const long long rowb = (long long)nx * ay + (long long)nxy * az;
                    for (int ax = x0; ax < x1; ++ax) {
                        const AT wx = (AT)(w1(P, 0, ax, Ix) * w1(P, 0, ax + sx, Jx));
                        acc += wyz * wx * (AT)As[rowb + ax];
                    }
                }
            }
        }
    }
    Ac[(long long)t * G.Nc + I] = acc;
}

// natural coarse index -> coordinates, offset helpers
__device__ __forceinline__ int nbr_index(const CGeom &G, int I, int o) {
    const int dx = o % 5 - 2, dy = (o / 5) % 5 - 2, dz = o / 25 - 2;
    const int x = I % G.cx + dx, y = (I / G.cx) % G.cy + dy, z = I / (G.cx * G.cy) + dz;
    if (x < 0 || x >= G.cx || y < 0 || y >= G.cy || z < 0 || z >= G.cz) return -1;
    return x + G.cx * (y + G.cy * z);
}

// D_k = within-block entries of A_c; identity on padding positions
template <typename AT>
__global__ void k_assemble(const AT *__restrict__ Ac, const int *__restrict__ pos,
                           const int *__restrict__ cell, CGeom G, AT *__restrict__ D) {
    const long long tot = (long long)G.nb * G.T;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < tot;
         p += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(p / G.T), r = (int)(p % G.T);
        AT *Dk = D + (long long)k * G.T * G.T;
        const int I = cell[p];
        if (I < 0) { Dk[(long long)r * G.T + r] = (AT)1; continue; }
        for (int o = 0; o < 125; ++o) {
            const int J = nbr_index(G, I, o);
            if (J < 0) continue;
            const int pj = pos[J];
            if (pj / G.T != k) continue;
            Dk[(long long)r * G.T + (pj % G.T)] = Ac[(long long)o * G.Nc + I];
        }
    }
}

// ELL forms of the couplings between block k and k+1:
//   lo: rows of block k+1 -> (column in block k, A_c value)   [Lo_k]
//   up: columns of block k+1 -> (row in block k, A_c value)   [Up_k, by column]
template <typename AT>
__global__ void k_ell(const AT *__restrict__ Ac, const int *__restrict__ pos,
                      const int *__restrict__ cell, CGeom G, int *__restrict__ lo_q,
                      AT *__restrict__ lo_v, int *__restrict__ up_q, AT *__restrict__ up_v,
                      int *__restrict__ err) {
    const long long tot = (long long)(G.nb - 1) * G.T;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < tot;
         p += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(p / G.T);
        const long long row = p + G.T;   // position in block k+1
        const int I = cell[row];
        int nl = 0, nu = 0;
        if (I >= 0) {
            for (int o = 0; o < 125; ++o) {
                const int J = nbr_index(G, I, o);
                if (J < 0) continue;
                const int pj = pos[J];
                if (pj / G.T != k) continue;
                // Lo_k[I][J] = A_c[I][J] (offset o of row I)
                if (nl < ELLW) {
                    lo_q[p * ELLW + nl] = pj % G.T;
                    lo_v[p * ELLW + nl] = Ac[(long long)o * G.Nc + I];
                }
                ++nl;
                // Up_k[J][I] = A_c[J][I] (offset 124 - o of row J)
                if (nu < ELLW) {
                    up_q[p * ELLW + nu] = pj % G.T;
                    up_v[p * ELLW + nu] = Ac[(long long)(124 - o) * G.Nc + J];
                }
                ++nu;
            }
        }
        if (nl > ELLW || nu > ELLW) atomicExch(err, 2);
        for (int e = min(nl, ELLW); e < ELLW; ++e) { lo_q[p * ELLW + e] = 0; lo_v[p * ELLW + e] = 0; }
        for (int e = min(nu, ELLW); e < ELLW; ++e) { up_q[p * ELLW + e] = 0; up_v[p * ELLW + e] = 0; }
    }
}

// ---------------------------------------------------------------------------
// blocked Gauss-Jordan inversion (in place, no pivoting) of one T x T block
// ---------------------------------------------------------------------------

template <typename AT>
__device__ void tile_load(AT (*s)[TILE + 1], const AT *M, int ld, int ti, int tj) {
    for (int e = threadIdx.x; e < TILE * TILE; e += blockDim.x) {
        const int i = e / TILE, j = e % TILE;
        s[i][j] = M[(long long)(ti * TILE + i) * ld + tj * TILE + j];
    }
}
template <typename AT>
__device__ void tile_store(AT (*s)[TILE + 1], AT *M, int ld, int ti, int tj) {
    for (int e = threadIdx.x; e < TILE * TILE; e += blockDim.x) {
        const int i = e / TILE, j = e % TILE;
        M[(long long)(ti * TILE + i) * ld + tj * TILE + j] = s[i][j];
    }
}

// in-place inverse of the 64 x 64 tile held in shared memory
template <typename AT>
__device__ void tile_invert(AT (*a)[TILE + 1], AT *col, int *err) {
    for (int kk = 0; kk < TILE; ++kk) {
        const AT p = a[kk][kk];
        if (threadIdx.x == 0 && (!(p != (AT)0) || !isfinite((double)p))) atomicExch(err, 1);
        const AT ip = (AT)1 / p;
        __syncthreads();
        for (int j = threadIdx.x; j < TILE; j += blockDim.x) {
            col[j] = a[j][kk];
            if (j != kk) a[kk][j] *= ip;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < TILE * TILE; e += blockDim.x) {
            const int i = e / TILE, j = e % TILE;
            if (i == kk) continue;
            if (j == kk) a[i][j] = -col[i] * ip;
            else a[i][j] -= col[i] * a[kk][j];
        }
        __syncthreads();
        if (threadIdx.x == 0) a[kk][kk] = ip;
        __syncthreads();
    }
}

// out = (sign) * X * Y (+ base), all 64 x 64 tiles in shared memory, 256 threads
template <typename AT>
__device__ __forceinline__ void tile_mma(AT (*X)[TILE + 1], AT (*Y)[TILE + 1], AT acc[4][4]) {
    const int tr = (threadIdx.x / 16) * 4, tc = (threadIdx.x % 16) * 4;
#pragma unroll 4
    for (int k = 0; k < TILE; ++k) {
        AT xa[4], yb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) { xa[u] = X[tr + u][k]; yb[u] = Y[k][tc + u]; }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] += xa[u] * yb[v];
    }
}

struct GJArgs {
    void *D;
    int ld, nt, p;
    int *err;
};

// job 0: invert the diagonal tile p (one CTA)
// shared-memory carve-up of the Gauss-Jordan kernels (dynamic: the FP64 tiles
// exceed the 48 KB static limit)
template <typename AT>
struct GJSmem {
    AT X[TILE][TILE + 1];
    AT Y[TILE][TILE + 1];
    AT col[TILE];
};

template <typename AT>
__device__ __forceinline__ GJSmem<AT> &gj_smem() {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    return *reinterpret_cast<GJSmem<AT> *>(smem_raw);
}

template <typename AT>
__global__ void __launch_bounds__(256) k_gj_diag(GJArgs a) {
    GJSmem<AT> &sm = gj_smem<AT>();
    auto &t = sm.X;
    auto &col = sm.col;
    AT *D = (AT *)a.D;
    tile_load(t, D, a.ld, a.p, a.p);
    __syncthreads();
    tile_invert(t, col, a.err);
    tile_store(t, D, a.ld, a.p, a.p);
}

// row panel: D_pj = Dpp^{-1} D_pj for j != p (CTA per j)
template <typename AT>
__global__ void __launch_bounds__(256) k_gj_row(GJArgs a) {
    GJSmem<AT> &sm = gj_smem<AT>();
    auto &X = sm.X;
    auto &Y = sm.Y;
    AT *D = (AT *)a.D;
    const int j = blockIdx.x < a.p ? blockIdx.x : blockIdx.x + 1;
    tile_load(X, D, a.ld, a.p, a.p);
    tile_load(Y, D, a.ld, a.p, j);
    __syncthreads();
    AT acc[4][4] = {};
    tile_mma(X, Y, acc);
    const int tr = (threadIdx.x / 16) * 4, tc = (threadIdx.x % 16) * 4;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v)
            D[(long long)(a.p * TILE + tr + u) * a.ld + j * TILE + tc + v] = acc[u][v];
}

// trailing update: D_ij -= D_ip D_pj for i, j != p (CTA per (i, j))
template <typename AT>
__global__ void __launch_bounds__(256) k_gj_update(GJArgs a) {
    GJSmem<AT> &sm = gj_smem<AT>();
    auto &X = sm.X;
    auto &Y = sm.Y;
    AT *D = (AT *)a.D;
    const int bi = blockIdx.x / (a.nt - 1), bj = blockIdx.x % (a.nt - 1);
    const int i = bi < a.p ? bi : bi + 1, j = bj < a.p ? bj : bj + 1;
    tile_load(X, D, a.ld, i, a.p);
    tile_load(Y, D, a.ld, a.p, j);
    __syncthreads();
    AT acc[4][4] = {};
    tile_mma(X, Y, acc);
    const int tr = (threadIdx.x / 16) * 4, tc = (threadIdx.x % 16) * 4;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const long long e = (long long)(i * TILE + tr + u) * a.ld + j * TILE + tc + v;
            D[e] -= acc[u][v];
        }
}

// column panel for step p (D_ip = -D_ip Dpp^{-1}, CTA per i != p) and, in the
// last CTA, the inversion of the next diagonal tile p + 1
template <typename AT>
__global__ void __launch_bounds__(256) k_gj_col(GJArgs a, int do_next) {
    GJSmem<AT> &sm = gj_smem<AT>();
    auto &X = sm.X;
    auto &Y = sm.Y;
    auto &col = sm.col;
    AT *D = (AT *)a.D;
    if ((int)blockIdx.x == a.nt - 1) {
        if (!do_next) return;
        tile_load(X, D, a.ld, a.p + 1, a.p + 1);
        __syncthreads();
        tile_invert(X, col, a.err);
        tile_store(X, D, a.ld, a.p + 1, a.p + 1);
        return;
    }
    const int i = blockIdx.x < a.p ? blockIdx.x : blockIdx.x + 1;
    tile_load(X, D, a.ld, i, a.p);
    tile_load(Y, D, a.ld, a.p, a.p);
    __syncthreads();
    AT acc[4][4] = {};
    tile_mma(X, Y, acc);
    const int tr = (threadIdx.x / 16) * 4, tc = (threadIdx.x % 16) * 4;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v)
            D[(long long)(i * TILE + tr + u) * a.ld + a.p * TILE + tc + v] = -acc[u][v];
}

// ---------------------------------------------------------------------------
// sparse-dense block products of the block Thomas recursion
// ---------------------------------------------------------------------------

// C_k[r][:] = sum_e lo_v[r][e] E_k[lo_q[r][e]][:]   (CTA per row r of block k+1)
template <typename AT>
__global__ void __launch_bounds__(256) k_lo_times(const int *__restrict__ lo_q,
                                                   const AT *__restrict__ lo_v,
                                                   const AT *__restrict__ E, AT *__restrict__ Cm,
                                                   int T) {
    const int r = blockIdx.x;
    const int *q = lo_q + (long long)r * ELLW;
    const AT *v = lo_v + (long long)r * ELLW;
    for (int c = threadIdx.x; c < T; c += blockDim.x) {
        AT acc = 0;
        for (int e = 0; e < ELLW; ++e) acc += v[e] * E[(long long)q[e] * T + c];
        Cm[(long long)r * T + c] = acc;
    }
}

// Out[r][c] (=, or -=) sum_e M[r][up_q[c][e]] up_v[c][e]   (CTA per row r)
template <typename AT>
__global__ void __launch_bounds__(256) k_times_up(const int *__restrict__ up_q,
                                                   const AT *__restrict__ up_v,
                                                   const AT *__restrict__ M, AT *__restrict__ Out,
                                                   int T, int subtract) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AT *row = reinterpret_cast<AT *>(smem_raw);
    const int r = blockIdx.x;
    for (int c = threadIdx.x; c < T; c += blockDim.x) row[c] = M[(long long)r * T + c];
    __syncthreads();
    for (int c = threadIdx.x; c < T; c += blockDim.x) {
        const int *q = up_q + (long long)c * ELLW;
        const AT *v = up_v + (long long)c * ELLW;
        AT acc = 0;
        for (int e = 0; e < ELLW; ++e) acc += row[q[e]] * v[e];
        if (subtract) Out[(long long)r * T + c] -= acc;
        else Out[(long long)r * T + c] = acc;
    }
}

// ---------------------------------------------------------------------------
// solve kernels
// ---------------------------------------------------------------------------

// y[b][r] = (subtract ? y[b][r] - : ) sum_c M[b][r][c] x[b][c]   (warp per row)
template <typename AT>
__global__ void __launch_bounds__(256) k_gemv(const AT *__restrict__ M, long long mstride,
                                              const AT *__restrict__ x, long long xstride,
                                              AT *__restrict__ y, long long ystride, int T,
                                              int subtract) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AT *xs = reinterpret_cast<AT *>(smem_raw);
    const int b = blockIdx.y;
    M += b * mstride; x += b * xstride; y += b * ystride;
    for (int c = threadIdx.x; c < T; c += blockDim.x) xs[c] = x[c];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (r >= T) return;
    const AT *row = M + (long long)r * T;
    AT acc = 0;
    for (int c = lane; c < T; c += 32) acc += row[c] * xs[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) y[r] = subtract ? y[r] - acc : acc;
}

// g[pos(I)] = sum_a P(a, I) t[a]   (warp per coarse cell)
template <typename AT>
__global__ void __launch_bounds__(256) k_restrict(const double *__restrict__ t, Interp P, CGeom G,
                                                  const int *__restrict__ pos, AT *__restrict__ g) {
    const int lane = threadIdx.x & 31;
    const int I = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (I >= G.Nc) return;
    const int Ix = I % G.cx, Iy = (I / G.cx) % G.cy, Iz = I / (G.cx * G.cy);
    const int x0 = P.lo[0][Ix], x1 = P.hi[0][Ix];
    const int y0 = P.lo[1][Iy], y1 = P.hi[1][Iy];
    const int z0 = P.lo[2][Iz], z1 = P.hi[2][Iz];
    const int wx = x1 - x0, wy = y1 - y0;
    const int tot = wx * wy * (z1 - z0);
    AT acc = 0;
    for (int e = lane; e < tot; e += 32) {
        const int ax = x0 + e % wx, ay = y0 + (e / wx) % wy, az = z0 + e / (wx * wy);
        const double w = w1(P, 0, ax, Ix) * w1(P, 1, ay, Iy) * w1(P, 2, az, Iz);
        acc += (AT)w * (AT)t[ax + (long long)G.nx * (ay + (long long)G.ny * az)];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) g[pos[I]] = acc;
}

// z[a] (+)= sum over the 8 bracketing coarse cells P(a, I) x[pos(I)]
template <typename AT>
__global__ void __launch_bounds__(256) k_prolong(const AT *__restrict__ x, Interp P, CGeom G,
                                                 const int *__restrict__ pos, double *__restrict__ z,
                                                 int accumulate) {
    const long long N = (long long)G.nx * G.ny * G.nz;
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < N;
         a += (long long)gridDim.x * blockDim.x) {
        const int ax = (int)(a % G.nx), ay = (int)((a / G.nx) % G.ny), az = (int)(a / ((long long)G.nx * G.ny));
        const int Ix[2] = {P.ia[0][ax], P.ib[0][ax]};
        const int Iy[2] = {P.ia[1][ay], P.ib[1][ay]};
        const int Iz[2] = {P.ia[2][az], P.ib[2][az]};
        const double Wx[2] = {P.wa[0][ax], P.wb[0][ax]};
        const double Wy[2] = {P.wa[1][ay], P.wb[1][ay]};
        const double Wz[2] = {P.wa[2][az], P.wb[2][az]};
        AT s = 0;
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int v = 0; v < 2; ++v)
#pragma unroll
                for (int w = 0; w < 2; ++w) {
                    const double wt = Wx[w] * Wy[v] * Wz[u];
                    if (wt == 0.0) continue;
                    const int I = Ix[w] + G.cx * (Iy[v] + G.cy * Iz[u]);
                    s += (AT)wt * x[pos[I]];
                }
        if (accumulate) z[a] += (double)s; else z[a] = (double)s;
    }
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------

static int grid_of(long long n, int threads = 256) {
    long long g = (n + threads - 1) / threads;
    return (int)std::max(1LL, std::min(g, 152LL * 16));
}

static void interp_axis(int n, int r, std::vector<int> &ia, std::vector<int> &ib,
                        std::vector<double> &wa, std::vector<double> &wb, std::vector<int> &lo,
                        std::vector<int> &hi, int &nc) {
    nc = n > 1 ? (n + r - 1) / r : 1;
    ia.assign(n, 0); ib.assign(n, 0); wa.assign(n, 1.0); wb.assign(n, 0.0);
    std::vector<double> xc(nc);
    for (int I = 0; I < nc; ++I) xc[I] = (r * I + std::min(r * I + r, n)) / 2.0;
    if (n > 1) {
        for (int i = 0; i < n; ++i) {
            const double x = i + 0.5;
            int I0 = (int)(std::upper_bound(xc.begin(), xc.end(), x) - xc.begin()) - 1;
            if (I0 < 0) { ia[i] = ib[i] = 0; wa[i] = 1.0; wb[i] = 0.0; }
            else if (I0 >= nc - 1) { ia[i] = ib[i] = nc - 1; wa[i] = 1.0; wb[i] = 0.0; }
            else {
                const double t = (x - xc[I0]) / (xc[I0 + 1] - xc[I0]);
                ia[i] = I0; wa[i] = 1.0 - t; ib[i] = I0 + 1; wb[i] = t;
            }
        }
    }
    lo.assign(nc, n); hi.assign(nc, 0);
    for (int i = 0; i < n; ++i) {
        const int Is[2] = {ia[i], ib[i]};
        for (int Ii : Is) { lo[Ii] = std::min(lo[Ii], i); hi[Ii] = std::max(hi[Ii], i + 1); }
    }
}

static Interp interp_of(const Coarse *c) {
    Interp P;
    for (int a = 0; a < 3; ++a) {
        P.ia[a] = c->d_ia[a]; P.ib[a] = c->d_ib[a];
        P.wa[a] = c->d_wa[a]; P.wb[a] = c->d_wb[a];
        P.lo[a] = c->d_lo[a]; P.hi[a] = c->d_hi[a];
    }
    return P;
}

static CGeom geom_of(const Coarse *c) {
    CGeom G;
    G.nx = c->nx; G.ny = c->ny; G.nz = c->nz;
    G.cx = c->c[0]; G.cy = c->c[1]; G.cz = c->c[2]; G.Nc = c->Nc;
    G.T = c->T; G.nb = c->nb;
    return G;
}

template <typename AT>
static int set_smem_attrs_t() {
    const int big = 227 * 1024;
    RAS_CK(cudaFuncSetAttribute(k_times_up<AT>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    RAS_CK(cudaFuncSetAttribute(k_gemv<AT>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    RAS_CK(cudaFuncSetAttribute(k_gj_diag<AT>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    RAS_CK(cudaFuncSetAttribute(k_gj_row<AT>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    RAS_CK(cudaFuncSetAttribute(k_gj_update<AT>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    RAS_CK(cudaFuncSetAttribute(k_gj_col<AT>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    return RAS_OK;
}

static int set_smem_attrs(int prec) {
    return prec == 64 ? set_smem_attrs_t<double>() : set_smem_attrs_t<float>();
}

int coarse_setup(Coarse **out, const ras_problem *Pb, const ras_opts &o) {
    *out = nullptr;
    if (o.interp_order != 2) return RAS_EINVAL;
    if (o.coarse_prec != 64 && o.coarse_prec != 32) return RAS_EINVAL;
    for (int a = 0; a < 3; ++a) if (o.coarsen[a] < 1) return RAS_EINVAL;
    Coarse *c = new Coarse();
    auto fail = [&](int s) { coarse_free(c); return s; };
    c->prec = o.coarse_prec;
    c->esz = c->prec == 64 ? 8 : 4;
    c->nx = Pb->nx; c->ny = Pb->ny; c->nz = Pb->nz; c->N = Pb->N;
    c->n[0] = Pb->nx; c->n[1] = Pb->ny; c->n[2] = Pb->nz;
    for (int a = 0; a < 3; ++a) {
        c->r[a] = o.coarsen[a];
        std::vector<int> ia, ib, lo, hi;
        std::vector<double> wa, wb;
        interp_axis(c->n[a], c->r[a], ia, ib, wa, wb, lo, hi, c->c[a]);
        int rc = 0;
        if ((rc = dalloc(&c->d_ia[a], ia.size())) || (rc = dalloc(&c->d_ib[a], ib.size())) ||
            (rc = dalloc(&c->d_wa[a], wa.size())) || (rc = dalloc(&c->d_wb[a], wb.size())) ||
            (rc = dalloc(&c->d_lo[a], lo.size())) || (rc = dalloc(&c->d_hi[a], hi.size())))
            return fail(rc);
        cudaMemcpy(c->d_ia[a], ia.data(), ia.size() * 4, cudaMemcpyHostToDevice);
        cudaMemcpy(c->d_ib[a], ib.data(), ib.size() * 4, cudaMemcpyHostToDevice);
        cudaMemcpy(c->d_wa[a], wa.data(), wa.size() * 8, cudaMemcpyHostToDevice);
        cudaMemcpy(c->d_wb[a], wb.data(), wb.size() * 8, cudaMemcpyHostToDevice);
        cudaMemcpy(c->d_lo[a], lo.data(), lo.size() * 4, cudaMemcpyHostToDevice);
        cudaMemcpy(c->d_hi[a], hi.data(), hi.size() * 4, cudaMemcpyHostToDevice);
    }
    c->Nc = c->c[0] * c->c[1] * c->c[2];
    // axes sorted by coarse size: fastest = smallest
    int ax[3] = {0, 1, 2};
    std::stable_sort(ax, ax + 3, [&](int p, int q) { return c->c[p] < c->c[q]; });
    c->af = ax[0]; c->am = ax[1]; c->as = ax[2];
    const int nf = c->c[c->af], nm = c->c[c->am], ns = c->c[c->as];
    const int planes = ns >= 2 ? 2 : 1;
    const int Treal = planes * nf * nm;
    c->T = ((Treal + TILE - 1) / TILE) * TILE;
    c->nb = (ns + planes - 1) / planes;
    if ((long long)c->T * c->T * c->nb * c->esz > (8LL << 30)) return fail(RAS_EINVAL);
    std::vector<int> pos(c->Nc), cell((size_t)c->nb * c->T, -1);
    for (int z = 0; z < c->c[2]; ++z)
        for (int y = 0; y < c->c[1]; ++y)
            for (int x = 0; x < c->c[0]; ++x) {
                const int co[3] = {x, y, z};
                const int I = x + c->c[0] * (y + c->c[1] * z);
                const int cf = co[c->af], cm = co[c->am], cs = co[c->as];
                const int k = cs / planes;
                const int local = cf + nf * (cm + nm * (cs % planes));
                pos[I] = k * c->T + local;
                cell[pos[I]] = I;
            }
    const size_t bsz = (size_t)c->T * c->T;
    int rc = 0;
    if ((rc = dalloc(&c->d_pos, pos.size())) || (rc = dalloc(&c->d_cell, cell.size())) ||
        (rc = dalloc(&c->d_err, 1)))
        return fail(rc);
    unsigned char *p_ac, *p_d, *p_c, *p_f, *p_lv, *p_uv, *p_g, *p_x;
    const size_t nbm1 = (size_t)std::max(c->nb - 1, 1);
    if ((rc = dalloc(&p_ac, (size_t)125 * c->Nc * c->esz)) || (rc = dalloc(&p_d, c->nb * bsz * c->esz)) ||
        (rc = dalloc(&p_c, nbm1 * bsz * c->esz)) || (rc = dalloc(&p_f, nbm1 * bsz * c->esz)) ||
        (rc = dalloc(&c->lo_q, nbm1 * c->T * ELLW)) || (rc = dalloc(&c->up_q, nbm1 * c->T * ELLW)) ||
        (rc = dalloc(&p_lv, nbm1 * c->T * ELLW * c->esz)) ||
        (rc = dalloc(&p_uv, nbm1 * c->T * ELLW * c->esz)) ||
        (rc = dalloc(&p_g, (size_t)c->nb * c->T * c->esz)) ||
        (rc = dalloc(&p_x, (size_t)c->nb * c->T * c->esz)))
        return fail(rc);
    c->Ac = p_ac; c->D = p_d; c->C = p_c; c->F = p_f; c->lo_v = p_lv; c->up_v = p_uv;
    c->g = p_g; c->x = p_x;
    if (cudaMemcpy(c->d_pos, pos.data(), pos.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_cell, cell.data(), cell.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(c->d_err, 0, 4) != cudaSuccess ||
        cudaMemset(c->g, 0, (size_t)c->nb * c->T * c->esz) != cudaSuccess ||
        cudaMemset(c->x, 0, (size_t)c->nb * c->T * c->esz) != cudaSuccess)
        return fail(RAS_ECUDA);
    const int sm = (int)(c->T * c->esz);
    if (sm > 227 * 1024) return fail(RAS_EINVAL);
    if ((rc = set_smem_attrs(c->prec)) != RAS_OK) return fail(rc);
    *out = c;
    return RAS_OK;
}

void coarse_free(Coarse *c) {
    if (!c) return;
    for (int a = 0; a < 3; ++a) {
        dfree(c->d_ia[a]); dfree(c->d_ib[a]); dfree(c->d_wa[a]); dfree(c->d_wb[a]);
        dfree(c->d_lo[a]); dfree(c->d_hi[a]);
    }
    dfree(c->d_pos); dfree(c->d_cell); dfree(c->d_err);
    dfree(c->lo_q); dfree(c->up_q);
    for (void *p : {c->Ac, c->D, c->C, c->F, c->lo_v, c->up_v, c->g, c->x})
        if (p) cudaFree(p);
    delete c;
}

template <typename AT>
static int gj_invert(Coarse *c, AT *Dk, cudaStream_t st) {
    const int nt = c->T / TILE;
    GJArgs a{Dk, c->T, nt, 0, c->d_err};
    const size_t sm = sizeof(GJSmem<AT>);
    k_gj_diag<AT><<<1, 256, sm, st>>>(a);
    RAS_LAUNCHED();
    for (int p = 0; p < nt; ++p) {
        a.p = p;
        if (nt > 1) {
            k_gj_row<AT><<<nt - 1, 256, sm, st>>>(a);
            RAS_LAUNCHED();
            k_gj_update<AT><<<(nt - 1) * (nt - 1), 256, sm, st>>>(a);
            RAS_LAUNCHED();
            k_gj_col<AT><<<nt, 256, sm, st>>>(a, p + 1 < nt ? 1 : 0);
            RAS_LAUNCHED();
        }
    }
    return RAS_OK;
}

template <typename AT>
static int factor_t(Coarse *c, const Stencil7 &A, cudaStream_t st) {
    const CGeom G = geom_of(c);
    const Interp P = interp_of(c);
    AT *Ac = (AT *)c->Ac, *D = (AT *)c->D, *Cm = (AT *)c->C, *Fm = (AT *)c->F;
    const size_t bsz = (size_t)c->T * c->T;
    k_rap<AT><<<c->Nc, 128, 0, st>>>(A, P, G, Ac);
    RAS_LAUNCHED();
    RAS_CK(cudaMemsetAsync(D, 0, c->nb * bsz * sizeof(AT), st));
    k_assemble<AT><<<grid_of((long long)c->nb * c->T), 256, 0, st>>>(Ac, c->d_pos, c->d_cell, G, D);
    RAS_LAUNCHED();
    if (c->nb > 1) {
        k_ell<AT><<<grid_of((long long)(c->nb - 1) * c->T), 256, 0, st>>>(
            Ac, c->d_pos, c->d_cell, G, c->lo_q, (AT *)c->lo_v, c->up_q, (AT *)c->up_v, c->d_err);
        RAS_LAUNCHED();
    }
    const size_t ell = (size_t)c->T * ELLW;
    for (int k = 0; k < c->nb; ++k) {
        AT *Dk = D + k * bsz;
        RAS_TRY(gj_invert<AT>(c, Dk, st));           // E_k = D_k^{-1} in place
        if (k + 1 < c->nb) {
            AT *Ck = Cm + k * bsz, *Fk = Fm + k * bsz;
            const int *lq = c->lo_q + k * ell, *uq = c->up_q + k * ell;
            const AT *lv = (const AT *)c->lo_v + k * ell, *uv = (const AT *)c->up_v + k * ell;
            k_lo_times<AT><<<c->T, 256, 0, st>>>(lq, lv, Dk, Ck, c->T);          // C_k = Lo_k E_k
            RAS_LAUNCHED();
            k_times_up<AT><<<c->T, 256, c->T * sizeof(AT), st>>>(uq, uv, Dk, Fk, c->T, 0);  // F_k
            RAS_LAUNCHED();
            k_times_up<AT><<<c->T, 256, c->T * sizeof(AT), st>>>(uq, uv, Ck, Dk + bsz, c->T, 1);
            RAS_LAUNCHED();                                                   // D_{k+1} -= C_k Up_k
        }
    }
    return RAS_OK;
}

int coarse_factor(Coarse *c, const Stencil7 &A, cudaStream_t st) {
    return c->prec == 64 ? factor_t<double>(c, A, st) : factor_t<float>(c, A, st);
}

int coarse_check(Coarse *c, cudaStream_t st) {
    int h = 0;
    RAS_CK(cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    RAS_CK(cudaStreamSynchronize(st));
    if (h) {
        RAS_CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), st));
        return h == 2 ? RAS_EINVAL : RAS_EZEROPIVOT;
    }
    return RAS_OK;
}

template <typename AT>
static int correct_t(Coarse *c, const double *t, double *z, int accumulate, cudaStream_t st) {
    const CGeom G = geom_of(c);
    const Interp P = interp_of(c);
    AT *g = (AT *)c->g, *x = (AT *)c->x;
    const AT *E = (const AT *)c->D, *Cm = (const AT *)c->C, *Fm = (const AT *)c->F;
    const long long bsz = (long long)c->T * c->T;
    const int T = c->T;
    k_restrict<AT><<<(c->Nc + 7) / 8, 256, 0, st>>>(t, P, G, c->d_pos, g);
    RAS_LAUNCHED();
    const dim3 rows((T + 7) / 8, 1);
    const size_t sm = T * sizeof(AT);
    for (int k = 1; k < c->nb; ++k) {            // g_k -= C_{k-1} g_{k-1}
        k_gemv<AT><<<rows, 256, sm, st>>>(Cm + (k - 1) * bsz, 0, g + (long long)(k - 1) * T, 0,
                                          g + (long long)k * T, 0, T, 1);
        RAS_LAUNCHED();
    }
    // x_k = E_k g_k for every block at once
    k_gemv<AT><<<dim3((T + 7) / 8, c->nb), 256, sm, st>>>(E, bsz, g, T, x, T, T, 0);
    RAS_LAUNCHED();
    for (int k = c->nb - 2; k >= 0; --k) {       // x_k -= F_k x_{k+1}
        k_gemv<AT><<<rows, 256, sm, st>>>(Fm + k * bsz, 0, x + (long long)(k + 1) * T, 0,
                                          x + (long long)k * T, 0, T, 1);
        RAS_LAUNCHED();
    }
    k_prolong<AT><<<grid_of(c->N), 256, 0, st>>>(x, P, G, c->d_pos, z, accumulate);
    RAS_LAUNCHED();
    return RAS_OK;
}

int coarse_correct(Coarse *c, const double *t, double *z, int accumulate, cudaStream_t st) {
    return c->prec == 64 ? correct_t<double>(c, t, z, accumulate, st)
                         : correct_t<float>(c, t, z, accumulate, st);
}

double coarse_bytes(const Coarse *c) {
    // E, C, F read once per solve
    return (double)c->esz * c->T * c->T * (c->nb + 2.0 * (c->nb - 1));
}

}  // namespace ras
