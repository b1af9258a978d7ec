// Restricted additive Schwarz on a coarse level of the multilevel method
// (Section 3.2, Algorithm 1), on sm_103a.
//
// A coarse-level operator is the Galerkin product of the level above; with
// linear interpolation its couplings reach two cells along each axis, so it
// is stored as 125 offset arrays [125][N] (many slots are structurally zero:
// 81 are used for a 7-point fine operator). The subdomain solver is ILU(0) in
// the natural order of each overlapped box on the operator's nonzero pattern.
//
// GPU mapping: one CTA per subdomain, one warp per matrix row. A row's 62
// lower (or upper) couplings are spread over the 32 lanes and reduced with
// shuffles; rows with no mutual dependency form a level (a static wavefront
// schedule computed per box shape on the host from the full 5x5x5
// neighbourhood, a superset of every pattern), and levels are separated by CTA
// barriers. The working vector of a subdomain lives in shared memory.
#include "ras125.cuh"

#include <algorithm>
#include <map>
#include <tuple>

namespace ras {

__host__ __device__ __forceinline__ int off_dx(int o) { return o % 5 - 2; }
__host__ __device__ __forceinline__ int off_dy(int o) { return (o / 5) % 5 - 2; }
__host__ __device__ __forceinline__ int off_dz(int o) { return o / 25 - 2; }
__host__ __device__ __forceinline__ int off_enc(int dx, int dy, int dz) {
    return (dx + 2) + 5 * (dy + 2) + 25 * (dz + 2);
}

// ---------------------------------------------------------------------------
// level operator product
// ---------------------------------------------------------------------------

template <bool RES>
__global__ void __launch_bounds__(256) k_spmv125(const double *__restrict__ A, int nx, int ny,
                                                 int nz, const double *__restrict__ x,
                                                 const double *__restrict__ b,
                                                 double *__restrict__ y) {
    const int N = nx * ny * nz;
    const int nxy = nx * ny;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        const int i = n % nx, j = (n / nx) % ny, k = n / nxy;
        double acc = 0.0;
#pragma unroll
        for (int dz = -2; dz <= 2; ++dz) {
            if ((unsigned)(k + dz) >= (unsigned)nz) continue;
#pragma unroll
            for (int dy = -2; dy <= 2; ++dy) {
                if ((unsigned)(j + dy) >= (unsigned)ny) continue;
#pragma unroll
                for (int dx = -2; dx <= 2; ++dx) {
                    if ((unsigned)(i + dx) >= (unsigned)nx) continue;
                    const int o = off_enc(dx, dy, dz);
                    acc = fma(__ldg(A + (long long)o * N + n), __ldg(x + n + dx + nx * dy + nxy * dz),
                              acc);
                }
            }
        }
        y[n] = RES ? b[n] - acc : acc;
    }
}

int spmv125(const double *A, int nx, int ny, int nz, const double *x, const double *b, double *y,
            cudaStream_t st) {
    const long long N = (long long)nx * ny * nz;
    if (N <= 0) return RAS_OK;
    const int grid = (int)std::min<long long>((N + 255) / 256, 152LL * 16);
    if (b) k_spmv125<true><<<grid, 256, 0, st>>>(A, nx, ny, nz, x, b, y);
    else k_spmv125<false><<<grid, 256, 0, st>>>(A, nx, ny, nz, x, nullptr, y);
    RAS_LAUNCHED();
    return RAS_OK;
}

// ---------------------------------------------------------------------------
// factor records
// ---------------------------------------------------------------------------

template <int PREC> struct Val125;
template <> struct Val125<64> { using T = double; using Acc = double; };
template <> struct Val125<32> { using T = float; using Acc = float; };
template <> struct Val125<16> { using T = __nv_bfloat16; using Acc = float; };

// FP64 -> stored precision (BF16 through FP32, each round to nearest even)
template <int PREC>
__device__ __forceinline__ void store_val(void *base, long long idx, double v) {
    if constexpr (PREC == 64) reinterpret_cast<double *>(base)[idx] = v;
    else if constexpr (PREC == 32) reinterpret_cast<float *>(base)[idx] = (float)v;
    else reinterpret_cast<__nv_bfloat16 *>(base)[idx] = __float2bfloat16_rn((float)v);
}

template <int PREC>
__device__ __forceinline__ typename Val125<PREC>::Acc load_val(const void *base, long long idx) {
    if constexpr (PREC == 64) return __ldg(reinterpret_cast<const double *>(base) + idx);
    else if constexpr (PREC == 32) return __ldg(reinterpret_cast<const float *>(base) + idx);
    else return __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(base)[idx]);
}

// shape tables copied to shared memory by the whole CTA
__device__ __forceinline__ void copy_shape(Shape125 &dst, const Shape125 &src) {
    static_assert(sizeof(Shape125) % 4 == 0, "shape table size");
    const int *s = reinterpret_cast<const int *>(&src);
    int *d = reinterpret_cast<int *>(&dst);
    for (int t = threadIdx.x; t < (int)(sizeof(Shape125) / 4); t += blockDim.x) d[t] = s[t];
}

constexpr int PD = 3;        // pivots in flight in the factorisation
constexpr int AD = 4;        // levels of solve records in flight

__device__ __forceinline__ double sel4(const double (&w)[4], int r) {
    return r == 0 ? w[0] : (r == 1 ? w[1] : (r == 2 ? w[2] : w[3]));
}

// ---------------------------------------------------------------------------
// numeric ILU(0)
// ---------------------------------------------------------------------------

struct Fac125 {
    const Sub125 *subs;
    const Shape125 *shapes;
    const int *lvl;
    const unsigned *cells;
    const double *A;          // [125][N]
    int nx, ny, nz;
    double *work;             // [nrow][64]: upper row of U (upper slots) and 1/u_nn (slot 63)
    void *fwd, *bwd;          // records: L (lower slots); U (upper slots) and 1/u_nn (slot 63)
    int *err;
    const unsigned *mask;     // ILU(k) patterns (null: the nonzeros of A plus the diagonal)
};

// IKJ incomplete LU of one overlapped box in natural order, no pivoting: for
// every lower column m of row n's pattern, in ascending order,
//     w_m <- w_m / u_mm,   w_c <- w_c - w_m u_mc   (pattern columns c > m),
// (the division taken as a product with 1/u_mm, formed once per row: FP64
// instructions are scarce on this GPU and every lane would repeat it),
// where the pattern is the nonzeros of A_i plus the diagonal; the row's final
// w holds L (c < n) and U (c >= n). One warp per row: lane t holds the values
// at offsets t, t + 32, t + 64, t + 96. The U row of each pivot m is read from
// the FP64 work rows written at earlier levels (the U values of the next PD
// pivots are in flight while the current one is applied).
template <int PREC>
__global__ void __launch_bounds__(512) k_ras125_factor(Fac125 P) {
    extern __shared__ int posq[];                 // natural local index -> level-order row
    __shared__ Shape125 sh;
    const Sub125 si = P.subs[blockIdx.x];
    copy_shape(sh, P.shapes[si.shape]);
    __syncthreads();
    const int *lvl = P.lvl + sh.lvl_off;
    const unsigned *cells = P.cells + sh.cell_off;
    const int bx = sh.bx, by = sh.by, bz = sh.bz, bxy = bx * by;
    for (int q = threadIdx.x; q < sh.ncell; q += blockDim.x) {
        const unsigned e = cells[q];
        posq[(int)(e & 255u) + bx * (int)((e >> 8) & 255u) + bxy * (int)((e >> 16) & 255u)] = q;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long N = (long long)P.nx * P.ny * P.nz;
    const long long nxy = (long long)P.nx * P.ny;
    const long long g0 = si.e0x + P.nx * (long long)si.e0y + nxy * si.e0z;
    int ox[4], oy[4], oz[4], od[4];
    bool live[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int o = lane + 32 * r;
        live[r] = o < OP125;
        ox[r] = off_dx(o); oy[r] = off_dy(o); oz[r] = off_dz(o);
        od[r] = ox[r] + bx * oy[r] + bxy * oz[r];
    }
    const int nL = sh.nL;
    double *work = P.work + si.foff * RREC;
    auto inbox = [&](int i, int j, int k) {
        return (unsigned)i < (unsigned)bx && (unsigned)j < (unsigned)by && (unsigned)k < (unsigned)bz;
    };

    for (int l = 0; l < sh.nlev; ++l) {
        const int q1 = lvl[l + 1];
        for (int q = lvl[l] + wid; q < q1; q += nw) {
            const unsigned e = cells[q];
            const int i = e & 255u, j = (e >> 8) & 255u, k = (e >> 16) & 255u;
            const int n = i + bx * j + bxy * k;
            const long long g = g0 + i + P.nx * (long long)j + nxy * k;
            double w[4];
            bool pat[4];
            const unsigned *msk = P.mask ? P.mask + sh.mask_off + 4LL * n : nullptr;
            auto in_pattern = [&](int o, double v) {   // o in the box
                return msk ? ((msk[o >> 5] >> (o & 31)) & 1u) != 0u : (v != 0.0 || o == CENTRE125);
            };
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const bool inb = live[r] && inbox(i + ox[r], j + oy[r], k + oz[r]);
                const double v = inb ? P.A[(long long)(lane + 32 * r) * N + g] : 0.0;
                w[r] = v;
                pat[r] = inb && in_pattern(lane + 32 * r, v);
            }
            // lower pattern columns in ascending natural order (slot order)
            bool p0 = false, p1 = false;
            if (lane < nL) {
                const int o = sh.lowo[lane];
                p0 = inbox(i + off_dx(o), j + off_dy(o), k + off_dz(o)) &&
                     in_pattern(o, P.A[(long long)o * N + g]);
            }
            if (lane + 32 < nL) {
                const int o = sh.lowo[lane + 32];
                p1 = inbox(i + off_dx(o), j + off_dy(o), k + off_dz(o)) &&
                     in_pattern(o, P.A[(long long)o * N + g]);
            }
            unsigned m0 = __ballot_sync(0xffffffffu, p0), m1 = __ballot_sync(0xffffffffu, p1);
            auto take = [&]() -> int {
                if (m0) { const int s = __ffs(m0) - 1; m0 &= m0 - 1; return s; }
                if (m1) { const int s = 31 + __ffs(m1); m1 &= m1 - 1; return s; }
                return -1;
            };
            struct Pivot { int om; unsigned need; double pinv; double u[4]; };
            auto fetch = [&](int s, Pivot &f) {
                const int om = sh.lowo[s];
                const int mx = off_dx(om), my = off_dy(om), mz = off_dz(om);
                const int dm = mx + bx * my + bxy * mz;
                const double *wr = work + (long long)posq[n + dm] * RREC;
                f.om = om;
                f.need = 0;
                f.pinv = wr[RREC - 1];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int cx = ox[r] - mx, cy = oy[r] - my, cz = oz[r] - mz;
                    const bool need = pat[r] && od[r] > dm && cx >= -2 && cx <= 2 && cy >= -2 &&
                                      cy <= 2 && cz >= -2 && cz <= 2;
                    f.u[r] = need ? wr[sh.uslot[off_enc(cx, cy, cz)]] : 0.0;
                    if (need) f.need |= 1u << r;
                }
            };
            // pivots in order, their U rows fetched PD pivots ahead (register ring)
            Pivot pb[PD];
            int ps[PD];
#pragma unroll
            for (int u = 0; u < PD; ++u) {
                ps[u] = take();
                if (ps[u] >= 0) fetch(ps[u], pb[u]);
            }
            bool more = ps[0] >= 0;
            while (more) {
#pragma unroll
                for (int u = 0; u < PD; ++u) {
                    if (ps[u] < 0) { more = false; break; }
                    const Pivot cur = pb[u];
                    ps[u] = take();
                    if (ps[u] >= 0) fetch(ps[u], pb[u]);
                    const int rm = cur.om >> 5, lm_lane = cur.om & 31;
                    const double wm = __shfl_sync(0xffffffffu, sel4(w, rm), lm_lane);
                    const double lm = wm * cur.pinv;
                    if (lane == lm_lane) {
                        if (rm == 0) w[0] = lm;
                        else if (rm == 1) w[1] = lm;
                        else if (rm == 2) w[2] = lm;
                        else w[3] = lm;
                    }
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (cur.need & (1u << r)) w[r] -= lm * cur.u[r];
                }
            }
            const double piv = __shfl_sync(0xffffffffu, w[1], CENTRE125 - 32);
            if (lane == 0 && (!(piv != 0.0) || !isfinite(piv))) atomicExch(P.err, 1);
            const long long row = si.foff + q;
            double *wrow = work + (long long)q * RREC;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int o = lane + 32 * r;
                if (!live[r]) continue;
                if (od[r] > 0) {
                    const int us = sh.uslot[o];
                    wrow[us] = w[r];
                    store_val<PREC>(P.bwd, row * RREC + us, w[r]);
                } else if (od[r] < 0) {
                    const int ls = nL - 1 - sh.uslot[OP125 - 1 - o];
                    store_val<PREC>(P.fwd, row * RREC + ls, w[r]);
                } else if (o == CENTRE125) {
                    const double pinv = 1.0 / piv;
                    wrow[RREC - 1] = pinv;
                    store_val<PREC>(P.bwd, row * RREC + RREC - 1, pinv);
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// subdomain solves
// ---------------------------------------------------------------------------

struct App125 {
    const Sub125 *subs;
    const Shape125 *shapes;
    const int *lvl;
    const unsigned *cells;
    const void *fwd, *bwd;
    const double *r;
    double *z;
    int nx, ny, nz;
    int accumulate;
    int ycap;
};

// z = sum_i (R_i^0)^T U_i^{-1} L_i^{-1} R_i^delta r with, per row (one warp),
//     forward   y_n = r_n - sum_{m<n} l_nm y_m,
//     backward  z_n = (y_n - sum_{m>n} u_nm z_m) / u_nn,
// lane t taking the couplings of slots t and t + 32 (slot 63 of the backward
// record holds 1/u_nn). Accumulation in FP64 (64) or FP32 (32, 16). Each
// warp's first row of a level is loaded AD levels ahead (register ring).
template <int PREC>
__global__ void __launch_bounds__(512) k_ras125_apply(App125 P) {
    using Acc = typename Val125<PREC>::Acc;
    extern __shared__ __align__(16) unsigned char smem[];
    Acc *Y = reinterpret_cast<Acc *>(smem);
    int *lvl_s = reinterpret_cast<int *>(smem + (size_t)P.ycap * sizeof(Acc));
    __shared__ Shape125 sh;
    const Sub125 si = P.subs[blockIdx.x];
    copy_shape(sh, P.shapes[si.shape]);
    __syncthreads();
    const int *lvl = P.lvl + sh.lvl_off;
    const unsigned *cells = P.cells + sh.cell_off;
    const int bx = sh.bx, by = sh.by, bz = sh.bz, bxy = bx * by;
    const int nx = P.nx;
    const long long nxy = (long long)P.nx * P.ny;
    const long long g0 = si.e0x + nx * (long long)si.e0y + nxy * si.e0z;
    for (int t = threadIdx.x; t < sh.ncell; t += blockDim.x) {
        const int i = t % bx, j = (t / bx) % by, k = t / bxy;
        Y[t] = (Acc)__ldg(P.r + g0 + i + nx * (long long)j + nxy * k);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nL = sh.nL;
    int lx[2], ly[2], lz[2], ld[2], ux[2], uy[2], uz[2], ud[2];
    bool lv[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int s = lane + 32 * h;
        lv[h] = s < nL;
        const int ol = lv[h] ? sh.lowo[s] : CENTRE125, ou = lv[h] ? sh.upo[s] : CENTRE125;
        lx[h] = off_dx(ol); ly[h] = off_dy(ol); lz[h] = off_dz(ol);
        ld[h] = lx[h] + bx * ly[h] + bxy * lz[h];
        ux[h] = off_dx(ou); uy[h] = off_dy(ou); uz[h] = off_dz(ou);
        ud[h] = ux[h] + bx * uy[h] + bxy * uz[h];
    }
    auto inbox = [&](int i, int j, int k) {
        return (unsigned)i < (unsigned)bx && (unsigned)j < (unsigned)by && (unsigned)k < (unsigned)bz;
    };
    const long long fbase = si.foff * RREC;
    for (int t = threadIdx.x; t <= sh.nlev; t += blockDim.x) lvl_s[t] = lvl[t];
    __syncthreads();

    // the first row of each level for this warp, fetched AD levels ahead
    struct Row { int q; unsigned e; Acc v0, v1; };
    auto fetch = [&](int l, const void *rec) {
        Row rw;
        rw.q = -1;
        rw.e = 0;
        rw.v0 = rw.v1 = 0;
        if (l >= 0 && l < sh.nlev) {
            const int q = lvl_s[l] + wid;
            if (q < lvl_s[l + 1]) {
                const long long rb = fbase + (long long)q * RREC;
                rw.q = q;
                rw.e = __ldg(cells + q);
                rw.v0 = load_val<PREC>(rec, rb + lane);
                rw.v1 = load_val<PREC>(rec, rb + lane + 32);
            }
        }
        return rw;
    };
    // forward row: y_n = r_n - sum_{m<n} l_nm y_m
    auto fwd_row = [&](unsigned e, Acc a0, Acc a1) {
        const int i = e & 255u, j = (e >> 8) & 255u, k = (e >> 16) & 255u;
        const int n = i + bx * j + bxy * k;
        Acc acc = 0;
        if (lv[0] && inbox(i + lx[0], j + ly[0], k + lz[0])) acc += a0 * Y[n + ld[0]];
        if (lv[1] && inbox(i + lx[1], j + ly[1], k + lz[1])) acc += a1 * Y[n + ld[1]];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) Y[n] -= acc;
    };
    // backward row: z_n = (y_n - sum_{m>n} u_nm z_m) / u_nn (slot 63 = 1/u_nn)
    auto bwd_row = [&](unsigned e, Acc b0, Acc b1) {
        const int i = e & 255u, j = (e >> 8) & 255u, k = (e >> 16) & 255u;
        const int n = i + bx * j + bxy * k;
        Acc acc = 0;
        if (lv[0] && inbox(i + ux[0], j + uy[0], k + uz[0])) acc += b0 * Y[n + ud[0]];
        if (lv[1] && inbox(i + ux[1], j + uy[1], k + uz[1])) acc += b1 * Y[n + ud[1]];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        const Acc dinv = __shfl_sync(0xffffffffu, b1, 31);
        if (lane == 0) Y[n] = (Y[n] - acc) * dinv;
    };

    Row ring[AD];
#pragma unroll
    for (int u = 0; u < AD; ++u) ring[u] = fetch(u, P.fwd);
    for (int lb = 0; lb < sh.nlev; lb += AD) {
#pragma unroll
        for (int u = 0; u < AD; ++u) {
            const int l = lb + u;
            if (l < sh.nlev) {
                const Row cur = ring[u];
                ring[u] = fetch(l + AD, P.fwd);
                if (cur.q >= 0) fwd_row(cur.e, cur.v0, cur.v1);
                for (int q = lvl_s[l] + wid + nw; q < lvl_s[l + 1]; q += nw) {
                    const long long rb = fbase + (long long)q * RREC;
                    fwd_row(__ldg(cells + q), load_val<PREC>(P.fwd, rb + lane),
                            load_val<PREC>(P.fwd, rb + lane + 32));
                }
                __syncthreads();
            }
        }
    }
#pragma unroll
    for (int u = 0; u < AD; ++u) ring[u] = fetch(sh.nlev - 1 - u, P.bwd);
    for (int lb = 0; lb < sh.nlev; lb += AD) {
#pragma unroll
        for (int u = 0; u < AD; ++u) {
            const int l = sh.nlev - 1 - (lb + u);
            if (l >= 0) {
                const Row cur = ring[u];
                ring[u] = fetch(l - AD, P.bwd);
                if (cur.q >= 0) bwd_row(cur.e, cur.v0, cur.v1);
                for (int q = lvl_s[l] + wid + nw; q < lvl_s[l + 1]; q += nw) {
                    const long long rb = fbase + (long long)q * RREC;
                    bwd_row(__ldg(cells + q), load_val<PREC>(P.bwd, rb + lane),
                            load_val<PREC>(P.bwd, rb + lane + 32));
                }
                __syncthreads();
            }
        }
    }
    for (int t = threadIdx.x; t < sh.ncell; t += blockDim.x) {
        const int i = t % bx, j = (t / bx) % by, k = t / bxy;
        if (i < si.ox0 || i >= si.ox1 || j < si.oy0 || j >= si.oy1 || k < si.oz0 || k >= si.oz1)
            continue;
        double *dst = P.z + g0 + i + nx * (long long)j + nxy * k;
        const double v = (double)Y[t];
        if (P.accumulate) *dst += v; else *dst = v;
    }
}

// ---------------------------------------------------------------------------
// host set-up
// ---------------------------------------------------------------------------

static std::vector<int> split_even(int n, int parts) {
    std::vector<int> s(parts + 1);
    const int q = n / parts, r = n % parts;
    for (int p = 0; p <= parts; ++p) s[p] = p * q + std::min(p, r);
    return s;
}

// offset tables and wavefront schedule of one box shape
static void build_shape(Shape125 &sh, std::vector<int> &lvl_tab, std::vector<unsigned> &cell_tab) {
    const int bx = sh.bx, by = sh.by, bz = sh.bz, bxy = bx * by;
    auto delta = [&](int o) { return off_dx(o) + bx * off_dy(o) + bxy * off_dz(o); };
    std::vector<int> lower;
    for (int o = 0; o < OP125; ++o)
        if (o != CENTRE125 && delta(o) < 0) lower.push_back(o);
    std::stable_sort(lower.begin(), lower.end(), [&](int a, int b) { return delta(a) < delta(b); });
    sh.nL = (int)lower.size();                        // <= 62
    for (int s = 0; s < 64; ++s) { sh.lowo[s] = CENTRE125; sh.upo[s] = CENTRE125; }
    for (int o = 0; o < 128; ++o) sh.uslot[o] = -1;
    for (int s = 0; s < sh.nL; ++s) {
        sh.lowo[s] = (unsigned char)lower[s];
        sh.upo[s] = (unsigned char)(OP125 - 1 - lower[sh.nL - 1 - s]);
        sh.uslot[sh.upo[s]] = (signed char)s;
    }
    // level(n) = 1 + max level of its in-box lower neighbours (0 if none)
    std::vector<int> lev(sh.ncell, 0);
    int nlev = 0;
    for (int k = 0; k < bz; ++k)
        for (int j = 0; j < by; ++j)
            for (int i = 0; i < bx; ++i) {
                int L = 0;
                for (int s = 0; s < sh.nL; ++s) {
                    const int o = lower[s];
                    const int a = i + off_dx(o), b = j + off_dy(o), c = k + off_dz(o);
                    if (a < 0 || a >= bx || b < 0 || b >= by || c < 0 || c >= bz) continue;
                    L = std::max(L, lev[a + bx * b + bxy * c] + 1);
                }
                lev[i + bx * j + bxy * k] = L;
                nlev = std::max(nlev, L + 1);
            }
    sh.nlev = nlev;
    std::vector<int> cnt(nlev + 1, 0);
    for (int n = 0; n < sh.ncell; ++n) ++cnt[lev[n] + 1];
    for (int l = 0; l < nlev; ++l) cnt[l + 1] += cnt[l];
    sh.lvl_off = (int)lvl_tab.size();
    sh.cell_off = (int)cell_tab.size();
    sh.maxw = 0;
    for (int l = 0; l < nlev; ++l) {
        lvl_tab.push_back(cnt[l]);
        sh.maxw = std::max(sh.maxw, cnt[l + 1] - cnt[l]);
    }
    lvl_tab.push_back(cnt[nlev]);
    std::vector<unsigned> ordered(sh.ncell);
    std::vector<int> fill(cnt.begin(), cnt.end() - 1);
    for (int n = 0; n < sh.ncell; ++n) {     // natural order inside a level
        const int i = n % bx, j = (n / bx) % by, k = n / bxy;
        ordered[fill[lev[n]]++] = (unsigned)i | ((unsigned)j << 8) | ((unsigned)k << 16);
    }
    cell_tab.insert(cell_tab.end(), ordered.begin(), ordered.end());
}

// Level-of-fill ILU(k) pattern of one box shape on the 7-point structure:
// lev(n, c) = 0 for the couplings of the 7-point stencil inside the box and
// the diagonal; for every lower entry m of row n with lev(n, m) <= k, taken in
// ascending natural order, and every upper entry c of row m with
// lev(m, c) <= k: lev(n, c) = min(lev(n, c), lev(n, m) + lev(m, c) + 1) when
// that is <= k. Returns RAS_EINVAL if a kept entry lies outside the 5x5x5
// neighbourhood.
static int build_iluk_mask(Shape125 &sh, int k, std::vector<unsigned> &mask_tab) {
    const int bx = sh.bx, by = sh.by, bz = sh.bz, bxy = bx * by, nc = sh.ncell;
    const int ax7[6] = {off_enc(-1, 0, 0), off_enc(1, 0, 0), off_enc(0, -1, 0),
                        off_enc(0, 1, 0), off_enc(0, 0, -1), off_enc(0, 0, 1)};
    std::vector<signed char> lev((size_t)nc * OP125, 127);
    sh.mask_off = (int)mask_tab.size();
    for (int n = 0; n < nc; ++n) {
        const int i = n % bx, j = (n / bx) % by, kk = n / bxy;
        signed char *L = &lev[(size_t)n * OP125];
        L[CENTRE125] = 0;
        for (int o : ax7) {
            const int a = i + off_dx(o), b = j + off_dy(o), c = kk + off_dz(o);
            if (a >= 0 && a < bx && b >= 0 && b < by && c >= 0 && c < bz) L[o] = 0;
        }
        for (int s = 0; s < sh.nL; ++s) {
            const int om = sh.lowo[s];
            if (L[om] > k) continue;
            const int mx = off_dx(om), my = off_dy(om), mz = off_dz(om);
            const signed char *Lm = &lev[(size_t)(n + mx + bx * my + bxy * mz) * OP125];
            for (int u = 0; u < sh.nL; ++u) {
                const int ou = sh.upo[u];
                if (Lm[ou] > k) continue;
                const int nl = L[om] + Lm[ou] + 1;
                if (nl > k) continue;
                const int cx = mx + off_dx(ou), cy = my + off_dy(ou), cz = mz + off_dz(ou);
                if (cx < -2 || cx > 2 || cy < -2 || cy > 2 || cz < -2 || cz > 2) return RAS_EINVAL;
                const int oc = off_enc(cx, cy, cz);
                if (nl < L[oc]) L[oc] = (signed char)nl;
            }
        }
        unsigned wds[4] = {0u, 0u, 0u, 0u};
        for (int o = 0; o < OP125; ++o)
            if (L[o] <= k) wds[o >> 5] |= 1u << (o & 31);
        mask_tab.insert(mask_tab.end(), wds, wds + 4);
    }
    return RAS_OK;
}

__global__ void __launch_bounds__(256) k_embed7(Stencil7 A, int nx, int ny, int nz,
                                                double *__restrict__ A125) {
    const long long N = (long long)nx * ny * nz;
    const int slot[7] = {CENTRE125, off_enc(-1, 0, 0), off_enc(1, 0, 0), off_enc(0, -1, 0),
                         off_enc(0, 1, 0), off_enc(0, 0, -1), off_enc(0, 0, 1)};
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int s = 0; s < 7; ++s) A125[(long long)slot[s] * N + n] = A.c[s][n];
    }
}

int embed7(const Stencil7 &A, int nx, int ny, int nz, double *A125, cudaStream_t st) {
    const long long N = (long long)nx * ny * nz;
    const int grid = (int)std::min<long long>((N + 255) / 256, 152LL * 16);
    k_embed7<<<grid, 256, 0, st>>>(A, nx, ny, nz, A125);
    RAS_LAUNCHED();
    return RAS_OK;
}

// bytes one apply reads and writes: both 64-value records per row at the
// stored precision, r read and z written once
double ras125_bytes(const Ras125 &R) {
    const double esz = R.prec == 64 ? 8.0 : (R.prec == 32 ? 4.0 : 2.0);
    return 2.0 * RREC * esz * (double)R.nrow + 16.0 * (double)R.N;
}

constexpr int SMEM125_MAX = 200 * 1024;

int ras125_setup(Ras125 &R, int nx, int ny, int nz, int px, int py, int pz, int overlap, int prec,
                 int ilu_k) {
    if (nx < 1 || ny < 1 || nz < 1) return RAS_EINVAL;
    if (ilu_k < 0) return RAS_EINVAL;
    R.ilu_k = ilu_k;
    if (px < 1 || py < 1 || pz < 1 || overlap < 0) return RAS_EINVAL;
    if (px > nx || py > ny || pz > nz) return RAS_EINVAL;
    if (prec != 64 && prec != 32 && prec != 16) return RAS_EINVAL;
    R.nx = nx; R.ny = ny; R.nz = nz; R.N = nx * ny * nz;
    R.prec = prec;
    const int dims[3] = {nx, ny, nz};
    const int parts[3] = {px, py, pz};
    std::vector<int> cuts[3];
    for (int a = 0; a < 3; ++a) cuts[a] = split_even(dims[a], parts[a]);
    std::map<std::tuple<int, int, int>, int> shape_id;
    std::vector<int> lvl_tab;
    std::vector<unsigned> cell_tab;
    std::vector<unsigned> mask_tab;
    R.subs.clear();
    R.shapes.clear();
    long long foff = 0;
    int ycap = 0, lcap = 0, maxw = 1;
    for (int kz = 0; kz < pz; ++kz)
        for (int jy = 0; jy < py; ++jy)
            for (int ix = 0; ix < px; ++ix) {
                const int p[3] = {ix, jy, kz};
                int o0[3], o1[3], e0[3], e1[3];
                for (int a = 0; a < 3; ++a) {
                    o0[a] = cuts[a][p[a]];
                    o1[a] = cuts[a][p[a] + 1];
                    e0[a] = std::max(o0[a] - overlap, 0);
                    e1[a] = std::min(o1[a] + overlap, dims[a]);
                }
                const int bx = e1[0] - e0[0], by = e1[1] - e0[1], bz = e1[2] - e0[2];
                if (bx > 255 || by > 255 || bz > 255) return RAS_EINVAL;
                const int ncell = bx * by * bz;
                if (ncell > 16384) return RAS_EINVAL;
                const auto key = std::make_tuple(bx, by, bz);
                const auto it = shape_id.find(key);
                int sid = it == shape_id.end() ? -1 : it->second;
                if (sid < 0) {
                    Shape125 sh{};
                    sh.bx = bx; sh.by = by; sh.bz = bz; sh.ncell = ncell;
                    build_shape(sh, lvl_tab, cell_tab);
                    sh.mask_off = 0;
                    if (ilu_k > 0) RAS_TRY(build_iluk_mask(sh, ilu_k, mask_tab));
                    sid = (int)R.shapes.size();
                    shape_id[key] = sid;
                    R.shapes.push_back(sh);
                    ycap = std::max(ycap, ncell);
                    lcap = std::max(lcap, sh.nlev + 1);
                    maxw = std::max(maxw, sh.maxw);
                }
                Sub125 si{};
                si.e0x = e0[0]; si.e0y = e0[1]; si.e0z = e0[2];
                si.shape = sid;
                si.ox0 = o0[0] - e0[0]; si.oy0 = o0[1] - e0[1]; si.oz0 = o0[2] - e0[2];
                si.ox1 = o1[0] - e0[0]; si.oy1 = o1[1] - e0[1]; si.oz1 = o1[2] - e0[2];
                si.foff = foff;
                foff += ncell;
                R.subs.push_back(si);
            }
    R.nsub = (int)R.subs.size();
    for (const Sub125 &si : R.subs) {
        const Shape125 &sh = R.shapes[si.shape];
        if (si.e0x < 0 || si.e0y < 0 || si.e0z < 0 || si.e0x + sh.bx > nx ||
            si.e0y + sh.by > ny || si.e0z + sh.bz > nz)
            return RAS_EINVAL;
    }
    R.nrow = foff;
    R.ycap = ycap;
    R.lcap = lcap;
    R.nwarps = std::min(16, std::max(4, maxw));
    const size_t acc = prec == 64 ? 8 : 4;
    R.ycap = (ycap + 3) & ~3;
    R.smem_apply = (size_t)R.ycap * acc + (size_t)lcap * sizeof(int);
    R.smem_factor = (size_t)ycap * sizeof(int);
    if (R.smem_apply > (size_t)SMEM125_MAX || R.smem_factor > (size_t)SMEM125_MAX) return RAS_EINVAL;
    const size_t esz = prec == 64 ? 8 : (prec == 32 ? 4 : 2);
    const size_t nval = (size_t)R.nrow * RREC;
    unsigned char *fw = nullptr, *bw = nullptr;
    RAS_TRY(dalloc(&R.d_subs, R.subs.size()));
    RAS_TRY(dalloc(&R.d_shapes, R.shapes.size()));
    RAS_TRY(dalloc(&R.d_lvl, lvl_tab.size()));
    RAS_TRY(dalloc(&R.d_cells, cell_tab.size()));
    RAS_TRY(dalloc(&R.d_err, 1));
    if (ilu_k > 0) {
        RAS_TRY(dalloc(&R.d_mask, mask_tab.size()));
        RAS_CK(cudaMemcpy(R.d_mask, mask_tab.data(), mask_tab.size() * sizeof(unsigned),
                          cudaMemcpyHostToDevice));
    }
    RAS_TRY(dalloc(&R.d_work, nval));
    RAS_TRY(dalloc(&fw, nval * esz));
    R.d_fwd = fw;
    RAS_TRY(dalloc(&bw, nval * esz));
    R.d_bwd = bw;
    RAS_CK(cudaMemcpy(R.d_subs, R.subs.data(), R.subs.size() * sizeof(Sub125), cudaMemcpyHostToDevice));
    RAS_CK(cudaMemcpy(R.d_shapes, R.shapes.data(), R.shapes.size() * sizeof(Shape125),
                      cudaMemcpyHostToDevice));
    RAS_CK(cudaMemcpy(R.d_lvl, lvl_tab.data(), lvl_tab.size() * sizeof(int), cudaMemcpyHostToDevice));
    RAS_CK(cudaMemcpy(R.d_cells, cell_tab.data(), cell_tab.size() * sizeof(unsigned),
                      cudaMemcpyHostToDevice));
    RAS_CK(cudaMemset(R.d_err, 0, sizeof(int)));
    // slots that no offset uses stay zero for good
    RAS_CK(cudaMemset(R.d_work, 0, nval * sizeof(double)));
    RAS_CK(cudaMemset(R.d_fwd, 0, nval * esz));
    RAS_CK(cudaMemset(R.d_bwd, 0, nval * esz));
    const int big = SMEM125_MAX;
    if (prec == 64) {
        RAS_CK(cudaFuncSetAttribute(k_ras125_factor<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
        RAS_CK(cudaFuncSetAttribute(k_ras125_apply<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    } else if (prec == 32) {
        RAS_CK(cudaFuncSetAttribute(k_ras125_factor<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
        RAS_CK(cudaFuncSetAttribute(k_ras125_apply<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    } else {
        RAS_CK(cudaFuncSetAttribute(k_ras125_factor<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
        RAS_CK(cudaFuncSetAttribute(k_ras125_apply<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    }
    return RAS_OK;
}

void ras125_free(Ras125 &R) {
    dfree(R.d_subs); dfree(R.d_shapes); dfree(R.d_lvl); dfree(R.d_cells); dfree(R.d_err);
    dfree(R.d_work);
    dfree(R.d_mask);
    if (R.d_fwd) cudaFree(R.d_fwd);
    if (R.d_bwd) cudaFree(R.d_bwd);
    R.d_fwd = R.d_bwd = nullptr;
}

int ras125_factor(Ras125 &R, const double *A, cudaStream_t st) {
    Fac125 P;
    P.subs = R.d_subs; P.shapes = R.d_shapes; P.lvl = R.d_lvl; P.cells = R.d_cells;
    P.A = A; P.nx = R.nx; P.ny = R.ny; P.nz = R.nz;
    P.work = R.d_work; P.fwd = R.d_fwd; P.bwd = R.d_bwd; P.err = R.d_err;
    P.mask = R.d_mask;
    const int threads = 32 * R.nwarps;
    if (R.prec == 64) k_ras125_factor<64><<<R.nsub, threads, R.smem_factor, st>>>(P);
    else if (R.prec == 32) k_ras125_factor<32><<<R.nsub, threads, R.smem_factor, st>>>(P);
    else k_ras125_factor<16><<<R.nsub, threads, R.smem_factor, st>>>(P);
    RAS_LAUNCHED();
    return RAS_OK;
}

int ras125_check(Ras125 &R, cudaStream_t st) {
    int h = 0;
    RAS_CK(cudaMemcpyAsync(&h, R.d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    RAS_CK(cudaStreamSynchronize(st));
    if (h) {
        RAS_CK(cudaMemsetAsync(R.d_err, 0, sizeof(int), st));
        return RAS_EZEROPIVOT;
    }
    return RAS_OK;
}

int ras125_apply(Ras125 &R, const double *r, double *z, int accumulate, cudaStream_t st) {
    App125 P;
    P.subs = R.d_subs; P.shapes = R.d_shapes; P.lvl = R.d_lvl; P.cells = R.d_cells;
    P.fwd = R.d_fwd; P.bwd = R.d_bwd; P.r = r; P.z = z;
    P.nx = R.nx; P.ny = R.ny; P.nz = R.nz; P.accumulate = accumulate;
    P.ycap = R.ycap;
    const int threads = 32 * R.nwarps;
    if (R.prec == 64) k_ras125_apply<64><<<R.nsub, threads, R.smem_apply, st>>>(P);
    else if (R.prec == 32) k_ras125_apply<32><<<R.nsub, threads, R.smem_apply, st>>>(P);
    else k_ras125_apply<16><<<R.nsub, threads, R.smem_apply, st>>>(P);
    RAS_LAUNCHED();
    return RAS_OK;
}

}  // namespace ras
