// Coarse-grid correction of the two-level Schwarz preconditioners
// (Section 3.2): interpolation I_0^1 (Eq. equ:inter-second, tensor-product
// linear between cell-centred coarse centres), restriction R = P^T, the
// Galerkin coarse operator A_c = R A P (125-point stencil) and its exact solve
// by a dense block LU.
//
// Dense block LU: coarse cells are renumbered with the axes sorted by size
// (fastest = smallest). A_c couples cells at most two cells apart, so two
// consecutive planes of the slowest axis form one dense block of size T and
// A_c is block tridiagonal: A = tridiag(Lo_{k-1}, D_k, Up_k). Block
// elimination from both ends towards a middle block m (a "twisted" block
// Thomas: two independent chains of half the length). Edge e joins blocks e
// and e+1; a top edge (e < m) eliminates its pivot block e into target block
// e+1, a bottom edge (e >= m) its pivot block e+1 into target block e:
//     Inv_pivot = S_pivot^{-1},  C_e = A(target, pivot) Inv,  F_e = Inv A(pivot, target),
//     S_target = A(target, target) - C_e A(pivot, target),
// with S = the block after the Schur updates it has received; the middle
// block receives one update from each side. Solve: g_target -= C_e g_pivot
// along both chains, x_m = S_m^{-1} g_m, then x_pivot = Inv g_pivot - F_e x_target
// back along both chains. Each inverse is computed in place by a blocked
// Gauss-Jordan inversion without pivoting (64 x 64 tiles); the off-diagonal
// blocks are sparse and stored in ELL form.
//
// The factorisation and the solve each run as ONE cooperative persistent
// kernel whose phases are separated by a grid barrier; the barrier gives up
// after a bounded number of polls and reports RAS_ETIMEOUT instead of hanging.
// The solve of a single handle hands the prolongation z (+)= P x to a separate
// full-occupancy kernel (k_coarse_prolong) that reads the coarse solution in
// natural order; FP32 handles may take the cyclic reduction of the block
// tridiagonal system instead of the two-ended elimination (RAS_COARSE_CR=1).
#include "precond.cuh"

#include <algorithm>
#include <cstddef>
#include <cstdlib>
#include <numeric>
#include <type_traits>

namespace ras {

constexpr int TILE = 64;
constexpr int ELLW = 64;    // max couplings of one cell into the neighbouring block (<= 50)
constexpr int FROWS = 8;    // rows of a dense block staged per CTA in the sparse products
constexpr int FWAVE_CTAS = 16;   // least CTAs per handle in a batched block elimination
constexpr int ERR_PIVOT = 1, ERR_ELL = 2, ERR_TIMEOUT = 7;
constexpr long long BAR_POLLS = 1LL << 22;   // ~1-2 s of polling before a barrier gives up

// arrival counter on a 128-byte line of its own, and the launch's poll limit
struct GridBar {
    unsigned count;
    unsigned pad0[31];
    long long polls;   // poll limit of this launch (<= 0: BAR_POLLS)
};

struct Coarse {
    int prec = 64;
    int nx, ny, nz, N;
    int n[3], r[3], c[3], Nc;
    int wmax[3];                    // widest fine support of a coarse cell per axis
    int *d_ia[3] = {}, *d_ib[3] = {};
    double *d_wa[3] = {}, *d_wb[3] = {};
    int *d_lo[3] = {}, *d_hi[3] = {};
    double *d_wt[3] = {};           // per coarse index: the weights of its fine support (w1's values)
    int af, am, as;                 // axis order: fastest, middle, slowest
    int T = 0, nb = 0;              // block size (multiple of TILE), number of blocks
    int mid = 0;                    // middle block of the two-ended elimination
    int *d_pos = nullptr;           // natural coarse index -> block position
    int *d_cell = nullptr;          // block position -> natural coarse index or -1
    void *Ac = nullptr;             // [125][Nc] Galerkin stencil (prec)
    void *D = nullptr, *C = nullptr, *F = nullptr;   // [nb][T][T]
    int *lo_q = nullptr, *up_q = nullptr;            // ELL column / row indices
    int *lo_n = nullptr, *up_n = nullptr;            // ELL entries used per row / column
    void *lo_v = nullptr, *up_v = nullptr;           // ELL values
    void *g = nullptr, *x = nullptr;                 // [nb*T]
    void *xn = nullptr;                              // [Nc] the coarse solution in natural order
    void *Zs = nullptr;                              // scratch tile strips [2][TILE][T]
    void *rx = nullptr, *ry = nullptr;               // restriction passes [cx][ny][nz], [cx][cy][nz]
    int *d_err = nullptr;
    GridBar *d_bar = nullptr;
    size_t esz = 8;
    size_t rap_smem = 0, rap125_smem = 0, fac_smem = 0, sol_smem = 0;
    int rap_zs = 0;                 // 0: k_rap (whole support boxes); > 0: k_rap_slab, slabs of rap_zs planes
    int need125 = 0;                // the handle's operator is 125-point (three levels): k_rap125 must fit
    int rap125_ng = 25;             // offsets staged per round in k_rap125
    int fac_grid = 0, sol_grid = 0;
    int sol_npf = 0;                // rows per warp prefetched by the solve
    int use_tc = 0;                 // FP32 inverses: trailing updates on the tcgen05 tensor cores
    int cr = 0;                     // cyclic reduction instead of the two-ended elimination
    int *d_crf = nullptr, *d_crs = nullptr;   // its factorisation and solve schedules
    void *W = nullptr;              // its dense couplings and products [nslot][T][T]
    int cr_maxE = 0;                // most blocks it inverts concurrently
    long long cr_mats = 0;          // T x T matrices one of its solves reads
};

// ---------------------------------------------------------------------------
// geometry helpers (device)
// ---------------------------------------------------------------------------

struct Interp {
    const int *ia[3], *ib[3];
    const double *wa[3], *wb[3];
    const int *lo[3], *hi[3];
    const double *wt[3];   // [I][m]: P(lo[I] + m, I), m < W (the same values as w1)
    int W[3];
};

// P(a, I) along one axis (ia == ib only where the second weight is zero, so
// a selection suffices: no floating-point arithmetic)
__device__ __forceinline__ double w1(const Interp &P, int ax, int a, int I) {
    if (P.ia[ax][a] == I) return P.wa[ax][a];
    if (P.ib[ax][a] == I) return P.wb[ax][a];
    return 0.0;
}

struct CGeom {
    int nx, ny, nz;       // fine
    int cx, cy, cz, Nc;   // coarse
    int T, nb, mid;
};

// ---------------------------------------------------------------------------
// Galerkin product, sum-factorised per coarse row I:
//   A_c[I][I+d] = sum_s sum_a P(a,I) A_s(a) P(a + e_s, I + d),
// P = Px Py Pz, contracted z, then y, then x inside shared memory.
// ---------------------------------------------------------------------------

struct RapDims {
    int wx, wy, wz;   // maximum support widths (shared-memory capacity)
};

// The second and third contractions (y, then x) of a term whose U is complete.
template <typename AT>
__device__ __forceinline__ void rap_yx(const AT *Wy, const AT *Wx, int dstride, const AT *U, AT *V, AT *out,
                                       const int *vix, int wx, int wy, int WX, int WY) {
    const int nV = 25 * wx, plane = WY * WX;
    for (int e = threadIdx.x; e < nV; e += blockDim.x) {
        const int code = vix[e];
        const int dz = code >> 16, dy = (code >> 8) & 0xff, ax = code & 0xff;
        const AT *wy_ = Wy + dy * dstride;
        const AT *u = U + dz * plane + ax;
        AT acc = 0;
        for (int ay = 0; ay < wy; ++ay) acc += wy_[ay] * u[ay * WX];
        V[(dz * 5 + dy) * WX + ax] = acc;
    }
    __syncthreads();
    if (threadIdx.x < 125) {
        const int e = threadIdx.x;
        const int dx = e % 5, dy = (e / 5) % 5, dz = e / 25;
        const AT *wx_ = Wx + dx * dstride;
        AT acc = 0;
        for (int ax = 0; ax < wx; ++ax) acc += wx_[ax] * V[(dz * 5 + dy) * WX + ax];
        out[e] += acc;
    }
    __syncthreads();
}

// The three sum-factorised contractions of one fine-operator term for one
// coarse row (z, then y, then x):
//   U[dz][ay][ax] = sum_az Wz[dz][az] A[az][ay][ax],
//   V[dz][dy][ax] = sum_ay Wy[dy][ay] U[dz][ay][ax],
//   out[dz][dy][dx] += sum_ax Wx[dx][ax] V[dz][dy][ax].
// uix / vix hold the index decomposition of the first two passes (computed once
// per coarse row: dz << 16 | ay * WX + ax, and dz << 16 | dy << 8 | ax).
template <typename AT>
__device__ __forceinline__ void rap_term(const AT *Ab, const AT *Wz, const AT *Wy, const AT *Wx,
                                         int dstride, AT *U, AT *V, AT *out, const int *uix,
                                         const int *vix, int wx, int wy, int wz, int WX, int WY) {
    const int nU = 5 * wy * wx, plane = WY * WX;
    for (int e = threadIdx.x; e < nU; e += blockDim.x) {
        const int code = uix[e];
        const int dz = code >> 16, ab = code & 0xffff;
        const AT *wz_ = Wz + dz * dstride;
        AT acc = 0;
        for (int az = 0; az < wz; ++az) acc += wz_[az] * Ab[az * plane + ab];
        U[dz * plane + ab] = acc;
    }
    __syncthreads();
    rap_yx(Wy, Wx, dstride, U, V, out, vix, wx, wy, WX, WY);
}

// the index tables of rap_term for a coarse row with supports wx, wy
__device__ __forceinline__ void rap_tables(int *uix, int *vix, int wx, int wy, int WX) {
    for (int e = threadIdx.x; e < 5 * wy * wx; e += blockDim.x) {
        const int dz = e / (wy * wx), ay = (e / wx) % wy, ax = e % wx;
        uix[e] = (dz << 16) | (ay * WX + ax);
    }
    for (int e = threadIdx.x; e < 25 * wx; e += blockDim.x) {
        const int dz = e / (5 * wx), dy = (e / wx) % 5, ax = e % wx;
        vix[e] = (dz << 16) | (dy << 8) | ax;
    }
}

template <typename AT>
__global__ void __launch_bounds__(256) k_rap(Stencil7 A, Interp P, CGeom G, RapDims W,
                                             AT *__restrict__ Ac) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AT *sm = reinterpret_cast<AT *>(smem_raw);
    const int WX = W.wx, WY = W.wy, WZ = W.wz;
    const int WM = max(WX, max(WY, WZ));
    AT *Abox = sm;                              // [7][WZ][WY][WX]
    AT *Wt = Abox + 7 * WX * WY * WZ;           // [3][5][3][WM]
    AT *U = Wt + 45 * WM;                       // [5][WY][WX]
    AT *V = U + 5 * WY * WX;                    // [25][WX]
    AT *out = V + 25 * WX;                      // [125]
    int *uix = reinterpret_cast<int *>(out + 128);   // [5][WY][WX]
    int *vix = uix + 5 * WY * WX;                    // [25][WX]

    const int I = blockIdx.x;
    const int Ic[3] = {I % G.cx, (I / G.cx) % G.cy, I / (G.cx * G.cy)};
    const int cdim[3] = {G.cx, G.cy, G.cz};
    const int ndim[3] = {G.nx, G.ny, G.nz};
    const int lo[3] = {P.lo[0][Ic[0]], P.lo[1][Ic[1]], P.lo[2][Ic[2]]};
    const int wx = P.hi[0][Ic[0]] - lo[0], wy = P.hi[1][Ic[1]] - lo[1], wz = P.hi[2][Ic[2]] - lo[2];
    const int box = wx * wy * wz;
    const long long nxy = (long long)G.nx * G.ny;
    rap_tables(uix, vix, wx, wy, WX);

    for (int e = threadIdx.x; e < 7 * box; e += blockDim.x) {
        const int s = e / box, q = e % box;
        const int ax = q % wx, ay = (q / wx) % wy, az = q / (wx * wy);
        const long long g = (lo[0] + ax) + (long long)G.nx * (lo[1] + ay) + nxy * (lo[2] + az);
        const double *src = s == 0 ? A.c[0] : s == 1 ? A.c[1] : s == 2 ? A.c[2] : s == 3 ? A.c[3]
                          : s == 4 ? A.c[4] : s == 5 ? A.c[5] : A.c[6];   // no indexed parameter copy
        Abox[((s * WZ + az) * WY + ay) * WX + ax] = (AT)src[g];
    }
    // pair weights W[axis][d][s][a] = P(a, I) P(a + s, I + d)
    for (int e = threadIdx.x; e < 45 * WM; e += blockDim.x) {
        const int q = e % WM, si = (e / WM) % 3, d = (e / (3 * WM)) % 5, axis = e / (15 * WM);
        const int wa = axis == 0 ? wx : (axis == 1 ? wy : wz);
        double w = 0.0;
        if (q < wa) {
            const int a = lo[axis] + q, as = a + si - 1, J = Ic[axis] + d - 2;
            if (J >= 0 && J < cdim[axis] && as >= 0 && as < ndim[axis])
                w = w1(P, axis, a, Ic[axis]) * w1(P, axis, as, J);
        }
        Wt[e] = (AT)w;
    }
    if (threadIdx.x < 125) out[threadIdx.x] = 0;
    __syncthreads();

    for (int s = 0; s < 7; ++s) {
        // stencil term s: 0 centre, 1 -x, 2 +x, 3 -y, 4 +y, 5 -z, 6 +z
        const int sgn = (s & 1) ? -1 : 1;
        const int sx = (s == 1 || s == 2) ? sgn : 0;
        const int sy = (s == 3 || s == 4) ? sgn : 0;
        const int sz = (s == 5 || s == 6) ? sgn : 0;
        const AT *As = Abox + s * WZ * WY * WX;
        const AT *Wz = Wt + (2 * 15) * WM + (sz + 1) * WM;   // + dz * 3 * WM
        const AT *Wy = Wt + (1 * 15) * WM + (sy + 1) * WM;
        const AT *Wx = Wt + (0 * 15) * WM + (sx + 1) * WM;
        rap_term(As, Wz, Wy, Wx, 3 * WM, U, V, out, uix, vix, wx, wy, wz, WX, WY);
    }
    if (threadIdx.x < 125) Ac[(long long)threadIdx.x * G.Nc + I] = out[threadIdx.x];
}

// The same product for support boxes too large to stage whole (large
// coarse-to-fine ratios: a box is 2r cells wide per axis for linear
// interpolation): the seven terms one at a time, each term's box streamed
// through shared memory in slabs of ZS fine planes along z. U carries the z
// contraction from slab to slab and adds the planes in rap_term's order, in
// the same precision, so the result has k_rap's bits.
template <typename AT>
__global__ void __launch_bounds__(256) k_rap_slab(Stencil7 A, Interp P, CGeom G, RapDims W, int ZS,
                                                  AT *__restrict__ Ac) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AT *sm = reinterpret_cast<AT *>(smem_raw);
    const int WX = W.wx, WY = W.wy, WZ = W.wz;
    const int WM = max(WX, max(WY, WZ));
    const int plane = WY * WX;
    AT *slab = sm;                              // [ZS][WY][WX]
    AT *Wt = slab + ZS * plane;                 // [3][5][3][WM]
    AT *U = Wt + 45 * WM;                       // [5][WY][WX]
    AT *V = U + 5 * plane;                      // [25][WX]
    AT *out = V + 25 * WX;                      // [125]
    int *uix = reinterpret_cast<int *>(out + 128);   // [5][WY][WX]
    int *vix = uix + 5 * plane;                      // [25][WX]

    const int I = blockIdx.x;
    const int Ic[3] = {I % G.cx, (I / G.cx) % G.cy, I / (G.cx * G.cy)};
    const int cdim[3] = {G.cx, G.cy, G.cz};
    const int ndim[3] = {G.nx, G.ny, G.nz};
    const int lo[3] = {P.lo[0][Ic[0]], P.lo[1][Ic[1]], P.lo[2][Ic[2]]};
    const int wx = P.hi[0][Ic[0]] - lo[0], wy = P.hi[1][Ic[1]] - lo[1], wz = P.hi[2][Ic[2]] - lo[2];
    const int sbox = wx * wy, nU = 5 * wy * wx;
    const long long nxy = (long long)G.nx * G.ny;
    rap_tables(uix, vix, wx, wy, WX);
    for (int e = threadIdx.x; e < 45 * WM; e += blockDim.x) {   // pair weights, as in k_rap
        const int q = e % WM, si = (e / WM) % 3, d = (e / (3 * WM)) % 5, axis = e / (15 * WM);
        const int wa = axis == 0 ? wx : (axis == 1 ? wy : wz);
        double w = 0.0;
        if (q < wa) {
            const int a = lo[axis] + q, as = a + si - 1, J = Ic[axis] + d - 2;
            if (J >= 0 && J < cdim[axis] && as >= 0 && as < ndim[axis])
                w = w1(P, axis, a, Ic[axis]) * w1(P, axis, as, J);
        }
        Wt[e] = (AT)w;
    }
    if (threadIdx.x < 125) out[threadIdx.x] = 0;
    __syncthreads();

    for (int s = 0; s < 7; ++s) {
        const int sgn = (s & 1) ? -1 : 1;
        const int sx = (s == 1 || s == 2) ? sgn : 0;
        const int sy = (s == 3 || s == 4) ? sgn : 0;
        const int sz = (s == 5 || s == 6) ? sgn : 0;
        const AT *Wz = Wt + (2 * 15) * WM + (sz + 1) * WM;
        const AT *Wy = Wt + (1 * 15) * WM + (sy + 1) * WM;
        const AT *Wx = Wt + (0 * 15) * WM + (sx + 1) * WM;
        const double *src = s == 0 ? A.c[0] : s == 1 ? A.c[1] : s == 2 ? A.c[2] : s == 3 ? A.c[3]
                          : s == 4 ? A.c[4] : s == 5 ? A.c[5] : A.c[6];   // no indexed parameter copy
        for (int z0 = 0; z0 < wz; z0 += ZS) {
            const int zn = min(ZS, wz - z0);
            for (int e = threadIdx.x; e < zn * sbox; e += blockDim.x) {
                const int ax = e % wx, ay = (e / wx) % wy, az = e / sbox;
                const long long g = (lo[0] + ax) + (long long)G.nx * (lo[1] + ay) + nxy * (lo[2] + z0 + az);
                slab[(az * WY + ay) * WX + ax] = (AT)src[g];
            }
            __syncthreads();
            for (int e = threadIdx.x; e < nU; e += blockDim.x) {
                const int code = uix[e];
                const int dz = code >> 16, ab = code & 0xffff;
                const AT *wz_ = Wz + dz * 3 * WM + z0;
                AT acc = z0 == 0 ? (AT)0 : U[dz * plane + ab];
                for (int az = 0; az < zn; ++az) acc += wz_[az] * slab[az * plane + ab];
                U[dz * plane + ab] = acc;
            }
            __syncthreads();
        }
        rap_yx(Wy, Wx, 3 * WM, U, V, out, vix, wx, wy, WX, WY);
    }
    if (threadIdx.x < 125) Ac[(long long)threadIdx.x * G.Nc + I] = out[threadIdx.x];
}

// Shared memory of the Galerkin kernels of the 7-point operator for support
// widths w (elements of esz bytes): k_rap (zs = 0: the seven terms' whole boxes)
// or k_rap_slab (slabs of zs planes).
static size_t rap_smem_of(const int w[3], int zs, size_t esz) {
    const size_t WX = w[0], WY = w[1], WZ = w[2], WM = std::max(WX, std::max(WY, WZ));
    const size_t box = zs == 0 ? 7 * WX * WY * WZ : (size_t)zs * WX * WY;
    return esz * (box + 45 * WM + 5 * WY * WX + 25 * WX + 128) + sizeof(int) * (5 * WY * WX + 25 * WX);
}

// The form that fits in cap bytes: whole boxes when they fit, else the tallest
// slab that does (RAS_RAP_SLAB=n at set-up, a test knob, asks for slabs of at
// most n planes); RAS_EINVAL when not even one plane fits, or when the support
// is wider than rap_tables' packed indices hold (x < 256, one x-y plane < 2^16).
static int rap_plan(const int w[3], size_t esz, size_t cap, int &zs, size_t &smem) {
    zs = 0;
    smem = 0;
    if (w[0] > 255 || (long long)w[0] * w[1] > 0xffff) return RAS_EINVAL;
    int force = 0;
    if (const char *e = getenv("RAS_RAP_SLAB")) force = atoi(e);
    zs = 0;
    smem = rap_smem_of(w, 0, esz);
    if (force < 1 && smem <= cap) return RAS_OK;
    for (zs = force >= 1 ? std::min(force, w[2]) : w[2]; zs >= 1; --zs) {
        smem = rap_smem_of(w, zs, esz);
        if (smem <= cap) return RAS_OK;
    }
    zs = 0;
    return RAS_EINVAL;
}

// Galerkin product of a 125-point level operator A (the coarse operator of
// the level above), same sum factorisation, one fine offset t at a time:
//   A_c[I][I+d] = sum_t sum_a P(a,I) A_t(a) P(a + t, I + d).
// The support boxes of NG consecutive offsets are staged together (one round
// of loads per group); offsets whose values vanish on the box are skipped.
template <typename AT>
__global__ void __launch_bounds__(256) k_rap125(const double *__restrict__ Af, Interp P, CGeom G,
                                                RapDims W, int NG, AT *__restrict__ Ac) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AT *sm = reinterpret_cast<AT *>(smem_raw);
    const int WX = W.wx, WY = W.wy, WZ = W.wz;
    const int WM = max(WX, max(WY, WZ));
    const int BOX = WX * WY * WZ;
    AT *Abox = sm;                              // [NG][WZ][WY][WX]
    AT *Wt = Abox + (long long)NG * BOX;        // [3][5 d][5 t][WM]
    AT *U = Wt + 75 * WM;                       // [5][WY][WX]
    AT *V = U + 5 * WY * WX;                    // [25][WX]
    AT *out = V + 25 * WX;                      // [125]
    int *nzf = reinterpret_cast<int *>(out + 128);   // [NG] offset has a nonzero in the box
    int *uix = nzf + 32;                             // [5][WY][WX]
    int *vix = uix + 5 * WY * WX;                    // [25][WX]

    const int I = blockIdx.x;
    const int Ic[3] = {I % G.cx, (I / G.cx) % G.cy, I / (G.cx * G.cy)};
    const int cdim[3] = {G.cx, G.cy, G.cz};
    const int ndim[3] = {G.nx, G.ny, G.nz};
    const int lo[3] = {P.lo[0][Ic[0]], P.lo[1][Ic[1]], P.lo[2][Ic[2]]};
    const int wx = P.hi[0][Ic[0]] - lo[0], wy = P.hi[1][Ic[1]] - lo[1], wz = P.hi[2][Ic[2]] - lo[2];
    const int box = wx * wy * wz;
    const long long nxy = (long long)G.nx * G.ny;
    const long long Nf = nxy * G.nz;
    rap_tables(uix, vix, wx, wy, WX);

    // pair weights W[axis][d][t][a] = P(a, I) P(a + t - 2, I + d - 2)
    for (int e = threadIdx.x; e < 75 * WM; e += blockDim.x) {
        const int q = e % WM, ti = (e / WM) % 5, d = (e / (5 * WM)) % 5, axis = e / (25 * WM);
        const int wa = axis == 0 ? wx : (axis == 1 ? wy : wz);
        double w = 0.0;
        if (q < wa) {
            const int a = lo[axis] + q, as = a + ti - 2, J = Ic[axis] + d - 2;
            if (J >= 0 && J < cdim[axis] && as >= 0 && as < ndim[axis])
                w = w1(P, axis, a, Ic[axis]) * w1(P, axis, as, J);
        }
        Wt[e] = (AT)w;
    }
    if (threadIdx.x < 125) out[threadIdx.x] = 0;

    for (int t0 = 0; t0 < 125; t0 += NG) {
        const int ng = min(NG, 125 - t0);
        for (int g = threadIdx.x; g < ng; g += blockDim.x) nzf[g] = 0;
        __syncthreads();
        for (int e = threadIdx.x; e < ng * box; e += blockDim.x) {
            const int g = e / box, q = e % box;
            const int ax = q % wx, ay = (q / wx) % wy, az = q / (wx * wy);
            const long long gi = (lo[0] + ax) + (long long)G.nx * (lo[1] + ay) + nxy * (lo[2] + az);
            const double v = Af[(long long)(t0 + g) * Nf + gi];
            if (v != 0.0) nzf[g] = 1;
            Abox[(long long)g * BOX + (az * WY + ay) * WX + ax] = (AT)v;
        }
        __syncthreads();
        for (int g = 0; g < ng; ++g) {
            if (!nzf[g]) continue;
            const int t = t0 + g;
            const int tx = t % 5 - 2, ty = (t / 5) % 5 - 2, tz = t / 25 - 2;
            const AT *Ab = Abox + (long long)g * BOX;
            const AT *Wz = Wt + (2 * 25) * WM + (tz + 2) * WM;   // + dz * 5 * WM
            const AT *Wy = Wt + (1 * 25) * WM + (ty + 2) * WM;
            const AT *Wx = Wt + (0 * 25) * WM + (tx + 2) * WM;
            rap_term(Ab, Wz, Wy, Wx, 5 * WM, U, V, out, uix, vix, wx, wy, wz, WX, WY);
        }
    }
    if (threadIdx.x < 125) Ac[(long long)threadIdx.x * G.Nc + I] = out[threadIdx.x];
}

// FP32 Galerkin values into the FP64 level-operator storage
__global__ void k_widen(const float *__restrict__ src, double *__restrict__ dst, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = (double)src[i];
}

// natural coarse index -> neighbour at offset o (or -1)
__host__ __device__ __forceinline__ int nbr_index(const CGeom &G, int I, int o) {
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

// pivot / target block of edge e (see the header)
__host__ __device__ __forceinline__ int edge_pivot(int e, int mid) { return e < mid ? e : e + 1; }
__host__ __device__ __forceinline__ int edge_target(int e, int mid) { return e < mid ? e + 1 : e; }

// ELL forms of the couplings across edge e:
//   row ELL: rows of the target block -> (column in the pivot block, A_c value)  [A(target, pivot)]
//   col ELL: columns of the target block -> (row in the pivot block, A_c value)  [A(pivot, target), by column]
template <typename AT>
__global__ void k_ell(const AT *__restrict__ Ac, const int *__restrict__ pos,
                      const int *__restrict__ cell, CGeom G, int *__restrict__ lo_q,
                      AT *__restrict__ lo_v, int *__restrict__ up_q, AT *__restrict__ up_v,
                      int *__restrict__ lo_n, int *__restrict__ up_n, int *__restrict__ err) {
    const long long tot = (long long)(G.nb - 1) * G.T;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < tot;
         p += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(p / G.T);
        const int pv = edge_pivot(e, G.mid), tg = edge_target(e, G.mid);
        const int I = cell[(long long)tg * G.T + p % G.T];   // row of the target block
        int nl = 0, nu = 0;
        if (I >= 0) {
            for (int o = 0; o < 125; ++o) {
                const int J = nbr_index(G, I, o);
                if (J < 0) continue;
                const int pj = pos[J];
                if (pj / G.T != pv) continue;
                if (nl < ELLW) {   // A(target, pivot)[I][J] (offset o of row I)
                    lo_q[p * ELLW + nl] = pj % G.T;
                    lo_v[p * ELLW + nl] = Ac[(long long)o * G.Nc + I];
                }
                ++nl;
                if (nu < ELLW) {   // A(pivot, target)[J][I] (offset -o of row J), [e][T] layout
                    const long long u = (long long)e * ELLW * G.T + (long long)nu * G.T + (p % G.T);
                    up_q[u] = pj % G.T;
                    up_v[u] = Ac[(long long)(124 - o) * G.Nc + J];
                }
                ++nu;
            }
        }
        if (nl > ELLW || nu > ELLW) atomicExch(err, ERR_ELL);
        lo_n[p] = min(nl, ELLW);
        up_n[p] = min(nu, ELLW);
        for (int q = min(nl, ELLW); q < ELLW; ++q) { lo_q[p * ELLW + q] = 0; lo_v[p * ELLW + q] = 0; }
        for (int q = min(nu, ELLW); q < ELLW; ++q) {
            const long long u = (long long)e * ELLW * G.T + (long long)q * G.T + (p % G.T);
            up_q[u] = 0;
            up_v[u] = 0;
        }
    }
}

// Dense copies of the off-diagonal blocks for the first round of the cyclic
// reduction (edges oriented pivot e -> target e + 1): L(e + 1) = A(e + 1, e) from
// the row-wise couplings, U(e) = A(e, e + 1) from the column-wise ones. Lc and Uc
// are [nb][T][T] and zero on entry.
template <typename AT>
__global__ void k_cr_couplings(const int *__restrict__ lo_q, const AT *__restrict__ lo_v,
                               const int *__restrict__ lo_n, const int *__restrict__ up_q,
                               const AT *__restrict__ up_v, const int *__restrict__ up_n, int T, int nb,
                               AT *__restrict__ Lc, AT *__restrict__ Uc) {
    const long long tot = (long long)(nb - 1) * T, bsz = (long long)T * T;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < tot;
         p += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(p / T), r = (int)(p % T);
        AT *Lr = Lc + (e + 1) * bsz + (long long)r * T;
        for (int m = 0; m < lo_n[p]; ++m) Lr[lo_q[p * ELLW + m]] = lo_v[p * ELLW + m];
        for (int m = 0; m < up_n[p]; ++m) {
            const long long u = (long long)e * ELLW * T + (long long)m * T + r;
            Uc[e * bsz + (long long)up_q[u] * T + r] = up_v[u];
        }
    }
}

// ---------------------------------------------------------------------------
// bounded grid barrier (all CTAs are co-resident: cooperative launch)
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_add_release(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid barrier on a monotonically increasing arrival counter: barrier number e
// (1, 2, ...) of a launch is complete when the counter reaches e * G. After the
// CTA's threads meet, one thread adds its arrival with a release reduction (its
// CTA's earlier writes become visible with it) and polls the counter with acquire
// loads, at most the launch's poll limit; a second CTA barrier releases the
// other threads. The counter is reset to zero before every launch. (Measured on
// GB300 with 304 co-resident CTAs: 1.6 us per barrier, against 2.5 us for an
// atomic arrival whose last arriver publishes a separate release word between
// two full fences, and 2.0-2.7 us for two-level arrival trees.) The error word is
// read at entry without waiting for it (its value is consulted after the
// barrier) and every 1024 polls. G: the number of CTAs that take part (default:
// the grid; a group of co-resident CTAs with a barrier word of its own). Returns
// false if this or any CTA has flagged an error or the wait ran out (ERR_TIMEOUT
// is then set).
__device__ bool grid_barrier(GridBar *bar, int *err, unsigned &epoch, unsigned G = 0) {
    __shared__ int s_ok;
    ++epoch;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned e0 = *reinterpret_cast<volatile const unsigned *>(err);
        int ok = 1;
        const long long lim = bar->polls > 0 ? bar->polls : BAR_POLLS;
        const unsigned target = epoch * (G ? G : gridDim.x);
        red_add_release(&bar->count, 1u);
        long long it = 0;
        while (ld_acquire(&bar->count) < target) {
            if (++it > lim) { atomicExch(err, ERR_TIMEOUT); ok = 0; break; }
            if ((it & 1023) == 0 && ld_acquire((const unsigned *)err) != 0) { ok = 0; break; }
        }
        if (e0 != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---------------------------------------------------------------------------
// 64 x 64 tile helpers (256 threads; thread t owns rows tr..tr+3, cols tc..tc+3)
// ---------------------------------------------------------------------------

template <typename AT>
struct TileSmem {
    AT X[TILE][TILE + 1];
    AT Y[TILE][TILE + 1];
    AT rowb[2][4][TILE];   // four pivot rows (double buffered)
    AT colb[2][TILE][4];   // four pivot columns (double buffered)
    AT piv[2][4][4];       // inverse of the current / next 4 x 4 pivot block
};

// correctly rounded reciprocal (IEEE round to nearest)
__device__ __forceinline__ float recip_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip_rn(double x) { return __drcp_rn(x); }

// In-place inverse of a 4 x 4 block held in registers by the Laplace expansion in the
// 2 x 2 minors of rows (0, 1) and (2, 3): A^{-1} = adj(A) / det(A), one reciprocal
// (FP32: the hardware reciprocal, a few ulp; FP64 the correctly rounded one) and a
// short dependency chain (sequential Gauss-Jordan pivots took ~1 us more per 64 x 64
// tile inverse). False if the block is singular or not finite.
__device__ __forceinline__ float recip_fast(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double recip_fast(double x) { return recip_rn(x); }
template <typename AT>
__device__ __forceinline__ bool invert4(AT a[4][4]) {
    const AT s0 = a[0][0] * a[1][1] - a[1][0] * a[0][1], s1 = a[0][0] * a[1][2] - a[1][0] * a[0][2];
    const AT s2 = a[0][0] * a[1][3] - a[1][0] * a[0][3], s3 = a[0][1] * a[1][2] - a[1][1] * a[0][2];
    const AT s4 = a[0][1] * a[1][3] - a[1][1] * a[0][3], s5 = a[0][2] * a[1][3] - a[1][2] * a[0][3];
    const AT c5 = a[2][2] * a[3][3] - a[3][2] * a[2][3], c4 = a[2][1] * a[3][3] - a[3][1] * a[2][3];
    const AT c3 = a[2][1] * a[3][2] - a[3][1] * a[2][2], c2 = a[2][0] * a[3][3] - a[3][0] * a[2][3];
    const AT c1 = a[2][0] * a[3][2] - a[3][0] * a[2][2], c0 = a[2][0] * a[3][1] - a[3][0] * a[2][1];
    const AT det = s0 * c5 - s1 * c4 + s2 * c3 + s3 * c2 - s4 * c1 + s5 * c0;
    const bool ok = det != (AT)0 && isfinite(det);
    const AT i = recip_fast(det);
    AT b[4][4];
    b[0][0] = ( a[1][1] * c5 - a[1][2] * c4 + a[1][3] * c3) * i;
    b[0][1] = (-a[0][1] * c5 + a[0][2] * c4 - a[0][3] * c3) * i;
    b[0][2] = ( a[3][1] * s5 - a[3][2] * s4 + a[3][3] * s3) * i;
    b[0][3] = (-a[2][1] * s5 + a[2][2] * s4 - a[2][3] * s3) * i;
    b[1][0] = (-a[1][0] * c5 + a[1][2] * c2 - a[1][3] * c1) * i;
    b[1][1] = ( a[0][0] * c5 - a[0][2] * c2 + a[0][3] * c1) * i;
    b[1][2] = (-a[3][0] * s5 + a[3][2] * s2 - a[3][3] * s1) * i;
    b[1][3] = ( a[2][0] * s5 - a[2][2] * s2 + a[2][3] * s1) * i;
    b[2][0] = ( a[1][0] * c4 - a[1][1] * c2 + a[1][3] * c0) * i;
    b[2][1] = (-a[0][0] * c4 + a[0][1] * c2 - a[0][3] * c0) * i;
    b[2][2] = ( a[3][0] * s4 - a[3][1] * s2 + a[3][3] * s0) * i;
    b[2][3] = (-a[2][0] * s4 + a[2][1] * s2 - a[2][3] * s0) * i;
    b[3][0] = (-a[1][0] * c3 + a[1][1] * c1 - a[1][2] * c0) * i;
    b[3][1] = ( a[0][0] * c3 - a[0][1] * c1 + a[0][2] * c0) * i;
    b[3][2] = (-a[3][0] * s3 + a[3][1] * s1 - a[3][2] * s0) * i;
    b[3][3] = ( a[2][0] * s3 - a[2][1] * s1 + a[2][2] * s0) * i;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) a[u][v] = b[u][v];
    return ok;
}

// a[u][v] (rows tr + u, columns tc + v of a tile) -= X Y for 64 x 64 tiles X, Y of
// row stride ld, staged in shared memory: the arithmetic of subtile_product (the same
// k order, out = prev + (-1) acc), so that a tile update followed by its inverse needs
// no store and reload of the tile.
template <typename AT>
__device__ __forceinline__ void tile_pre_update(TileSmem<AT> &sm, AT (&a)[4][4], const AT *X, const AT *Y,
                                                int ld, int tr, int tc) {
    constexpr int VEC = 16 / sizeof(AT);
    using V16 = typename std::conditional<sizeof(AT) == 4, float4, double2>::type;
    constexpr int NV = TILE * TILE / VEC / 256;
    V16 bx[NV], by[NV];
#pragma unroll
    for (int m = 0; m < NV; ++m) {
        const int e = threadIdx.x + 256 * m, r = e / (TILE / VEC), k = (e % (TILE / VEC)) * VEC;
        bx[m] = __ldcg(reinterpret_cast<const V16 *>(X + (long long)r * ld + k));
        by[m] = __ldcg(reinterpret_cast<const V16 *>(Y + (long long)r * ld + k));
    }
#pragma unroll
    for (int m = 0; m < NV; ++m) {
        const int e = threadIdx.x + 256 * m, r = e / (TILE / VEC), k = (e % (TILE / VEC)) * VEC;
        const AT *vx = reinterpret_cast<const AT *>(&bx[m]), *vy = reinterpret_cast<const AT *>(&by[m]);
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
            sm.X[r][k + q] = vx[q];
            sm.Y[r][k + q] = vy[q];
        }
    }
    __syncthreads();
    AT acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0;
#pragma unroll 4
    for (int k = 0; k < TILE; ++k) {
        AT xa[4], yb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) xa[u] = sm.X[tr + u][k];
#pragma unroll
        for (int v = 0; v < 4; ++v) yb[v] = sm.Y[k][tc + v];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] += xa[u] * yb[v];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) a[u][v] = a[u][v] + (AT)(-1) * acc[u][v];
}

// In-place Gauss-Jordan inverse of tile (ti, ti) of M without pivoting, four
// pivots per step (block column K = kb..kb+3, Pi = A_KK^{-1}):
//     A_Kj <- Pi A_Kj,  A_ij <- A_ij - A_iK (Pi A_Kj),  A_iK <- -A_iK Pi,  A_KK <- Pi.
// Thread t owns rows tr..tr+3 and columns tc..tc+3 (no runtime register
// indexing). Per step: the pivot-row owners form Pi A_Kj and publish it, the
// pivot-column owners publish A_iK (barrier), every other thread applies the
// rank-4 update; the owner of the next pivot block inverts it as soon as its
// own update is done and publishes Pi for the next step (barrier). The 4 x 4
// inverse takes approximate reciprocals (FP32 preconditioner factors).
template <typename AT>
__device__ void tile_invert_b4(TileSmem<AT> &sm, AT *M, int ld, int ti, int *err, const AT *X = nullptr,
                               const AT *Y = nullptr) {
    const int tr = (threadIdx.x / 16) * 4, tc = (threadIdx.x % 16) * 4;
    AT a[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v)
            a[u][v] = __ldcg(M + (long long)(ti * TILE + tr + u) * ld + ti * TILE + tc + v);
    if (X) tile_pre_update(sm, a, X, Y, ld, tr, tc);   // the tile's last update first
    auto invert_publish = [&](int par) {
        AT P[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) P[u][v] = a[u][v];
        if (!invert4(P)) atomicExch(err, ERR_PIVOT);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) sm.piv[par][u][v] = P[u][v];
    };
    if (tr == 0 && tc == 0) invert_publish(0);
    __syncthreads();
    for (int kb = 0; kb < TILE; kb += 4) {
        const int par = (kb >> 2) & 1;
        AT Pi[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) Pi[u][v] = sm.piv[par][u][v];
        if (tr == kb && tc == kb) {                  // pivot block -> its inverse
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) a[u][v] = Pi[u][v];
        } else if (tr == kb) {                       // pivot rows: Pi A_Kj, published
            AT W[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    AT t = 0;
#pragma unroll
                    for (int q = 0; q < 4; ++q) t += Pi[u][q] * a[q][v];
                    W[u][v] = t;
                }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    a[u][v] = W[u][v];
                    sm.rowb[par][u][tc + v] = W[u][v];
                }
        } else if (tc == kb) {                       // pivot columns: publish A_iK, then -A_iK Pi
            AT c[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    c[u][v] = a[u][v];
                    sm.colb[par][tr + u][v] = a[u][v];
                }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    AT t = 0;
#pragma unroll
                    for (int m = 0; m < 4; ++m) t += c[u][m] * Pi[m][v];
                    a[u][v] = -t;
                }
        }
        __syncthreads();
        if (tr != kb && tc != kb) {                  // rank-4 update a -= A_iK (Pi A_Kj)
            AT W[4][4];
#pragma unroll
            for (int m = 0; m < 4; ++m)
#pragma unroll
                for (int v = 0; v < 4; ++v) W[m][v] = sm.rowb[par][m][tc + v];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                AT c[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) c[m] = sm.colb[par][tr + u][m];
#pragma unroll
                for (int v = 0; v < 4; ++v)
#pragma unroll
                    for (int m = 0; m < 4; ++m) a[u][v] -= c[m] * W[m][v];
            }
            if (tr == kb + 4 && tc == kb + 4) invert_publish(par ^ 1);   // next pivot block
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v)
            M[(long long)(ti * TILE + tr + u) * ld + ti * TILE + tc + v] = a[u][v];
}

// Scalar Gauss-Jordan (one pivot per barrier): fewest operations, used for
// FP64 where the arithmetic pipe, not the barrier, bounds the tile inverse.
template <typename AT>
__device__ void tile_invert_s(TileSmem<AT> &sm, AT *M, int ld, int ti, int *err, const AT *X = nullptr,
                              const AT *Y = nullptr) {
    const int tr = (threadIdx.x / 16) * 4, tc = (threadIdx.x % 16) * 4;
    AT a[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v)
            a[u][v] = __ldcg(M + (long long)(ti * TILE + tr + u) * ld + ti * TILE + tc + v);
    if (X) tile_pre_update(sm, a, X, Y, ld, tr, tc);   // the tile's last update first
    for (int kk = 0; kk < TILE; ++kk) {
        const int par = kk & 1;
        if (tr <= kk && kk < tr + 4) {
            const int u = kk - tr;
#pragma unroll
            for (int v = 0; v < 4; ++v)
                sm.rowb[par][0][tc + v] = u == 0 ? a[0][v] : (u == 1 ? a[1][v] : (u == 2 ? a[2][v] : a[3][v]));
        }
        if (tc <= kk && kk < tc + 4) {
            const int v = kk - tc;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                sm.colb[par][tr + u][0] = v == 0 ? a[u][0] : (v == 1 ? a[u][1] : (v == 2 ? a[u][2] : a[u][3]));
        }
        __syncthreads();
        const AT piv = sm.rowb[par][0][kk];
        if (threadIdx.x == 0 && (!(piv != (AT)0) || !isfinite(piv))) atomicExch(err, ERR_PIVOT);
        const AT ip = recip_rn(piv);
        AT rb[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) rb[v] = sm.rowb[par][0][tc + v] * ip;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool ri = (tr + u == kk);
            const AT ci = sm.colb[par][tr + u][0];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const bool cj = (tc + v == kk);
                AT nv = a[u][v] - ci * rb[v];
                if (ri) nv = cj ? ip : rb[v];
                else if (cj) nv = -ci * ip;
                a[u][v] = nv;
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v)
            M[(long long)(ti * TILE + tr + u) * ld + ti * TILE + tc + v] = a[u][v];
}

// (X, Y: tiles whose product the tile receives first, tile -= X Y; null: none)
template <typename AT>
__device__ __forceinline__ void tile_invert(TileSmem<AT> &sm, AT *M, int ld, int ti, int *err,
                                            const AT *X = nullptr, const AT *Y = nullptr) {
    if constexpr (sizeof(AT) == 8) tile_invert_s(sm, M, ld, ti, err, X, Y);
    else tile_invert_b4(sm, M, ld, ti, err, X, Y);
}

// Sub-tile product: rows [r0, r0 + RR) and columns [c0, c0 + CC) of
//     out(oi, oj) = sign * tile(xi, xj) * tile(yi, yj)  (+ out if accumulate),
// 256 threads x BR x BC outputs. In-place use is safe when the output part
// depends only on the staged part of the aliased input: a row panel
// (out = P * out) is split by columns, a column panel (out = out * P) by rows.
template <typename AT, int RR, int CC, int BR, int BC>
__device__ void subtile_product(TileSmem<AT> &sm, const AT *Xb, const AT *Yb, AT *Ob, int ld, int xi,
                                int xj, int yi, int yj, int oi, int oj, int r0, int c0, AT sign,
                                bool accumulate) {
    static_assert((RR / BR) * (CC / BC) == 256, "256 threads");
    AT (*X)[TILE + 1] = sm.X;   // X[r][k], r < RR
    AT (*Y)[TILE + 1] = sm.Y;   // Y[k][c], c < CC
    // stage both parts with 16-byte loads, all issued before any is consumed
    constexpr int VEC = 16 / sizeof(AT);
    using V16 = typename std::conditional<sizeof(AT) == 4, float4, double2>::type;
    constexpr int NX = RR * TILE / VEC / 256, NY = TILE * CC / VEC / 256;
    static_assert(NX >= 1 && NY >= 1, "staging split");
    V16 bx[NX], by[NY];
#pragma unroll
    for (int m = 0; m < NX; ++m) {
        const int e = threadIdx.x + 256 * m;            // vector index
        const int r = e / (TILE / VEC), k = (e % (TILE / VEC)) * VEC;
        bx[m] = __ldcg(reinterpret_cast<const V16 *>(Xb + (long long)(xi * TILE + r0 + r) * ld +
                                                     xj * TILE + k));
    }
#pragma unroll
    for (int m = 0; m < NY; ++m) {
        const int e = threadIdx.x + 256 * m;
        const int k = e / (CC / VEC), c = (e % (CC / VEC)) * VEC;
        by[m] = __ldcg(reinterpret_cast<const V16 *>(Yb + (long long)(yi * TILE + k) * ld + yj * TILE +
                                                     c0 + c));
    }
#pragma unroll
    for (int m = 0; m < NX; ++m) {
        const int e = threadIdx.x + 256 * m;
        const int r = e / (TILE / VEC), k = (e % (TILE / VEC)) * VEC;
        const AT *v = reinterpret_cast<const AT *>(&bx[m]);
#pragma unroll
        for (int q = 0; q < VEC; ++q) X[r][k + q] = v[q];
    }
#pragma unroll
    for (int m = 0; m < NY; ++m) {
        const int e = threadIdx.x + 256 * m;
        const int k = e / (CC / VEC), c = (e % (CC / VEC)) * VEC;
        const AT *v = reinterpret_cast<const AT *>(&by[m]);
#pragma unroll
        for (int q = 0; q < VEC; ++q) Y[k][c + q] = v[q];
    }
    __syncthreads();
    constexpr int TPR = CC / BC;
    const int rr = (threadIdx.x / TPR) * BR, cc = (threadIdx.x % TPR) * BC;
    AT acc[BR][BC];
#pragma unroll
    for (int u = 0; u < BR; ++u)
#pragma unroll
        for (int v = 0; v < BC; ++v) acc[u][v] = 0;
#pragma unroll 4
    for (int k = 0; k < TILE; ++k) {
        AT xa[BR], yb[BC];
#pragma unroll
        for (int u = 0; u < BR; ++u) xa[u] = X[rr + u][k];
#pragma unroll
        for (int v = 0; v < BC; ++v) yb[v] = Y[k][cc + v];
#pragma unroll
        for (int u = 0; u < BR; ++u)
#pragma unroll
            for (int v = 0; v < BC; ++v) acc[u][v] += xa[u] * yb[v];
    }
    __syncthreads();   // the output may alias a staged input
    // all reads of the old output before any store (one round of loads)
    AT prev[BR][BC];
#pragma unroll
    for (int u = 0; u < BR; ++u)
#pragma unroll
        for (int v = 0; v < BC; ++v)
            prev[u][v] = accumulate
                ? __ldcg(Ob + (long long)(oi * TILE + r0 + rr + u) * ld + oj * TILE + c0 + cc + v)
                : (AT)0;
#pragma unroll
    for (int u = 0; u < BR; ++u)
#pragma unroll
        for (int v = 0; v < BC; ++v)
            Ob[(long long)(oi * TILE + r0 + rr + u) * ld + oj * TILE + c0 + cc + v] =
                prev[u][v] + sign * acc[u][v];
}

// ---------------------------------------------------------------------------
// trailing updates of the FP32 Gauss-Jordan inverses on the tcgen05 tensor cores
//
// Two vertically adjacent 64 x 64 tiles of a block, rows 128 x columns of tile j,
// are updated together: Out -= X Y with X the 128 x 64 column strip of the pivot
// panel and Y the 64 x 64 pivot-row tile, one group of MMAs (M = 128, N = 64,
// K = 8 per instruction) with FP32 accuracy from the TF32 path by the three-term
// split X Y ~ Xh Yh + Xh Yl + Xl Yh (h: rounded to TF32, l: the FP32 remainder),
// accumulated in FP32 in tensor memory (64 columns per CTA, allocated for the
// launch). Operands are split and written by the CTA's threads into shared memory
// in the canonical K-major layout without swizzle (8-row x 16-byte core matrices,
// 128 B apart along k, 2048 B apart along rows); one thread issues the MMAs and
// commits them to an mbarrier that the CTA waits on (bounded).
// ---------------------------------------------------------------------------

struct TcSmem {
    alignas(128) unsigned char xh[128 * 64 * 4], xl[128 * 64 * 4];   // X: 128 rows x 64 k
    alignas(128) unsigned char yh[64 * 64 * 4], yl[64 * 64 * 4];     // Y^T: 64 columns x 64 k
};

struct TcState {
    bool on;                     // tensor memory held: the tensor path is in use
    unsigned tmem;               // accumulator base (64 columns; any value, 0 included)
    unsigned long long *mbar;    // MMA completion
    unsigned phase;              // completed waits of this CTA
};

constexpr unsigned TC_LBO = 128, TC_SBO = 2048;
constexpr unsigned TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
constexpr long long TC_POLLS = 1LL << 26;

__device__ __forceinline__ int tc_off(int row, int k) {
    return (row >> 3) * TC_SBO + (k >> 2) * TC_LBO + (row & 7) * 16 + (k & 3) * 4;
}
__device__ __forceinline__ unsigned long long tc_desc(unsigned addr) {
    unsigned long long d = (unsigned long long)((addr & 0x3FFFFu) >> 4);
    d |= (unsigned long long)((TC_LBO >> 4) & 0x3FFF) << 16;
    d |= (unsigned long long)((TC_SBO >> 4) & 0x3FFF) << 32;
    d |= 1ull << 46;
    return d;
}
__device__ __forceinline__ float tc_head(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
__device__ __forceinline__ void tc_put(unsigned char *h, unsigned char *l, int off, float v) {
    const float vh = tc_head(v);
    *reinterpret_cast<float *>(h + off) = vh;
    *reinterpret_cast<float *>(l + off) = v - vh;
}

// Out(tiles i0, i0 + 1; tile column j) -= D(same rows, tile column p) D(p, j), T x T
// row-major block M. All 256 threads; the CTA's smem overlay is free on entry.
__device__ void tc_pair_update(TcSmem &ts, TcState &st, float *M, int T, int i0, int p, int j, int *err) {
    const int tid = threadIdx.x;
    // the updated tiles (rows 64 i0 .. + 127, column tile j) are read together with the
    // operands: no other item of the phase writes them, and they overlap neither X
    // (column tile p) nor Y (row tile p); warp w: rows 32 (w % 4) + lane, columns
    // 32 (w / 4) .. + 31
    const int w = tid >> 5, lane = tid & 31, wq = w & 3, wh = w >> 2;
    float *out = M + (long long)(i0 * TILE + 32 * wq + lane) * T + j * TILE + 32 * wh;
    float4 prev[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) prev[u] = __ldcg(reinterpret_cast<const float4 *>(out) + u);
    {   // X: rows 64 i0 .. + 127, columns 64 p .. + 63; thread t: row t / 2, k half (t & 1)
        const int r = tid >> 1, k0 = (tid & 1) * 32;
        const float4 *src = reinterpret_cast<const float4 *>(M + (long long)(i0 * TILE + r) * T + p * TILE + k0);
        float4 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = __ldcg(src + q);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float *e = reinterpret_cast<const float *>(&v[q]);
#pragma unroll
            for (int u = 0; u < 4; ++u) tc_put(ts.xh, ts.xl, tc_off(r, k0 + 4 * q + u), e[u]);
        }
    }
    {   // Y^T: Y = D(p, j), element (k, n) to row n, column k; thread t: k = t / 4, n block (t & 3)
        const int k = tid >> 2, n0 = (tid & 3) * 16;
        const float4 *src = reinterpret_cast<const float4 *>(M + (long long)(p * TILE + k) * T + j * TILE + n0);
        float4 v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = __ldcg(src + q);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float *e = reinterpret_cast<const float *>(&v[q]);
#pragma unroll
            for (int u = 0; u < 4; ++u) tc_put(ts.yh, ts.yl, tc_off(n0 + 4 * q + u, k), e[u]);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned xh = (unsigned)__cvta_generic_to_shared(ts.xh), xl = (unsigned)__cvta_generic_to_shared(ts.xl);
        const unsigned yh = (unsigned)__cvta_generic_to_shared(ts.yh), yl = (unsigned)__cvta_generic_to_shared(ts.yl);
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const unsigned o = s * 2 * TC_LBO;   // k-step of 8: two core matrices along k
            const unsigned long long d[3][2] = {{tc_desc(xl + o), tc_desc(yh + o)},
                                                {tc_desc(xh + o), tc_desc(yl + o)},
                                                {tc_desc(xh + o), tc_desc(yh + o)}};
#pragma unroll
            for (int t3 = 0; t3 < 3; ++t3) {
                const unsigned acc = (s > 0 || t3 > 0) ? 1u : 0u;
                asm volatile(
                    "{\n.reg .pred pp;\n"
                    "setp.ne.b32 pp, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, pp;\n}\n"
                    ::"r"(st.tmem), "l"(d[t3][0]), "l"(d[t3][1]), "r"(TC_IDESC), "r"(acc) : "memory");
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"((unsigned)__cvta_generic_to_shared(st.mbar)) : "memory");
    }
    {   // bounded wait for the MMAs
        const unsigned a = (unsigned)__cvta_generic_to_shared(st.mbar), par = st.phase & 1;
        bool done = false;
        for (long long it = 0; it < TC_POLLS && !done; ++it) {
            unsigned ok;
            asm volatile(
                "{\n.reg .pred pp;\n"
                "mbarrier.try_wait.parity.shared::cta.b64 pp, [%1], %2;\n"
                "selp.u32 %0, 1, 0, pp;\n}\n"
                : "=r"(ok) : "r"(a), "r"(par) : "memory");
            done = ok != 0;
        }
        if (!done) atomicExch(err, ERR_TIMEOUT);
        ++st.phase;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    {
        unsigned r[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
              "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
              "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
              "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(st.tmem + ((unsigned)(32 * wq) << 16) + 32u * wh));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            float4 o = prev[u];
            o.x -= __uint_as_float(r[4 * u]);
            o.y -= __uint_as_float(r[4 * u + 1]);
            o.z -= __uint_as_float(r[4 * u + 2]);
            o.w -= __uint_as_float(r[4 * u + 3]);
            reinterpret_cast<float4 *>(out)[u] = o;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();   // the smem overlay and the accumulator are free again
}

// One product of tc_gemm_core: A (its first row and chunk; leading dimension
// lda) times B (its first chunk row and column; leading dimension ldb) over nk
// chunks of 64 along k. With bidx, row k of B is row bidx[k] of B (negative: a
// zero row), so that B can be a gathered set of rows.
struct TcOp {
    const float *A, *B;
    int lda, ldb, nk;
    const int *bidx;
};

// Out[0 .. nrows) x [0 .. 64) (leading dimension ldo) (=, +=) sign (o1 [+ o2]) for
// FP32 row-major operands, on tcgen05 (M = 128, N = 64, K = 8, the three-term TF32
// split of tc_pair_update), accumulated in tensor memory; the next chunk's global
// loads are issued before the wait for the current chunk's MMAs. nrows is 64 or
// 128 (rows past it enter as zeros and are not written). All 256 threads; the
// CTA's shared-memory overlay is free on entry and on return.
__device__ void tc_gemm_core(TcSmem &ts, TcState &st, float *Out, int ldo, int nrows, const TcOp &o1,
                             const TcOp *o2, bool acc, float sign, int *err) {
    const int tid = threadIdx.x, nk1 = o1.nk, nch = nk1 + (o2 ? o2->nk : 0);
    const int xr = tid >> 1, xk0 = (tid & 1) * 32;        // A chunk: row, k half
    const int yk = tid >> 2, yn0 = (tid & 3) * 16;        // B chunk: k, 16 columns
    float4 vx[8], vy[4];
    auto load = [&](int ch) {
        const TcOp &o = ch < nk1 ? o1 : *o2;
        const int kc = (ch < nk1 ? ch : ch - nk1) * TILE;
        if (xr < nrows) {
            const float4 *src = reinterpret_cast<const float4 *>(o.A + (long long)xr * o.lda + kc + xk0);
#pragma unroll
            for (int q = 0; q < 8; ++q) vx[q] = __ldcg(src + q);
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) vx[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const long long br = o.bidx ? (long long)o.bidx[kc + yk] : (long long)(kc + yk);
        if (br >= 0) {
            const float4 *srcy = reinterpret_cast<const float4 *>(o.B + br * o.ldb + yn0);
#pragma unroll
            for (int q = 0; q < 4; ++q) vy[q] = __ldcg(srcy + q);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) vy[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    auto wait_mma = [&]() {
        const unsigned a = (unsigned)__cvta_generic_to_shared(st.mbar), par = st.phase & 1;
        bool done = false;
        for (long long it = 0; it < TC_POLLS && !done; ++it) {
            unsigned ok;
            asm volatile(
                "{\n.reg .pred pp;\n"
                "mbarrier.try_wait.parity.shared::cta.b64 pp, [%1], %2;\n"
                "selp.u32 %0, 1, 0, pp;\n}\n"
                : "=r"(ok) : "r"(a), "r"(par) : "memory");
            done = ok != 0;
        }
        if (!done) atomicExch(err, ERR_TIMEOUT);
        ++st.phase;
    };
    load(0);
    for (int ch = 0; ch < nch; ++ch) {
        if (ch > 0) wait_mma();                             // the MMAs of the previous chunk are done
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float *e = reinterpret_cast<const float *>(&vx[q]);
#pragma unroll
            for (int u = 0; u < 4; ++u) tc_put(ts.xh, ts.xl, tc_off(xr, xk0 + 4 * q + u), e[u]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float *e = reinterpret_cast<const float *>(&vy[q]);
#pragma unroll
            for (int u = 0; u < 4; ++u) tc_put(ts.yh, ts.yl, tc_off(yn0 + 4 * q + u, yk), e[u]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned xh = (unsigned)__cvta_generic_to_shared(ts.xh), xl = (unsigned)__cvta_generic_to_shared(ts.xl);
            const unsigned yh = (unsigned)__cvta_generic_to_shared(ts.yh), yl = (unsigned)__cvta_generic_to_shared(ts.yl);
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                const unsigned o = s * 2 * TC_LBO;
                const unsigned long long d[3][2] = {{tc_desc(xl + o), tc_desc(yh + o)},
                                                    {tc_desc(xh + o), tc_desc(yl + o)},
                                                    {tc_desc(xh + o), tc_desc(yh + o)}};
#pragma unroll
                for (int t3 = 0; t3 < 3; ++t3) {
                    const unsigned accum = (ch > 0 || s > 0 || t3 > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n.reg .pred pp;\n"
                        "setp.ne.b32 pp, %4, 0;\n"
                        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, pp;\n}\n"
                        ::"r"(st.tmem), "l"(d[t3][0]), "l"(d[t3][1]), "r"(TC_IDESC), "r"(accum) : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"((unsigned)__cvta_generic_to_shared(st.mbar)) : "memory");
        }
        if (ch + 1 < nch) load(ch + 1);
    }
    wait_mma();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    {   // warp w: rows 32 (w % 4) + lane, columns 32 (w / 4) .. + 31
        const int w = tid >> 5, lane = tid & 31, q = w & 3, h = w >> 2;
        unsigned r[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
              "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
              "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
              "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(st.tmem + ((unsigned)(32 * q) << 16) + 32u * h));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int row = 32 * q + lane;
        if (row < nrows) {
            float *out = Out + (long long)row * ldo + 32 * h;
            float4 prev[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                prev[u] = acc ? __ldcg(reinterpret_cast<const float4 *>(out) + u) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                float4 o = prev[u];
                o.x += sign * __uint_as_float(r[4 * u]);
                o.y += sign * __uint_as_float(r[4 * u + 1]);
                o.z += sign * __uint_as_float(r[4 * u + 2]);
                o.w += sign * __uint_as_float(r[4 * u + 3]);
                reinterpret_cast<float4 *>(out)[u] = o;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();   // the smem overlay and the accumulator are free again
}

// Out(tile rows 2 pr, 2 pr + 1, the second only if it exists; tile column j)
// (=, +=) sign (A1 B1 [+ A2 B2]) for T x T blocks, over the full inner dimension.
__device__ __forceinline__ void tc_gemm_pair(TcSmem &ts, TcState &st, float *Out, int T, int pr, int j,
                                             const float *A1, const float *B1, const float *A2,
                                             const float *B2, bool acc, float sign, int *err) {
    const int nk = T / TILE;
    const long long r0 = (long long)2 * pr * TILE * T;
    const TcOp o1{A1 + r0, B1 + j * TILE, T, T, nk, nullptr};
    const TcOp o2{A2 ? A2 + r0 : nullptr, B2 ? B2 + j * TILE : nullptr, T, T, nk, nullptr};
    tc_gemm_core(ts, st, Out + r0 + j * TILE, T, 2 * pr + 1 < nk ? 128 : 64, o1, A2 ? &o2 : nullptr, acc, sign,
                 err);
}

// ---------------------------------------------------------------------------
// cooperative factorisation: block Thomas with in-place Gauss-Jordan inverses
// ---------------------------------------------------------------------------

template <typename AT>
struct FacArgs {
    AT *D, *C, *F;
    AT *Z;   // scratch: per chain 64 rows x T (tile (0, 0) used) for -D_{p+1,p} P_p
    const int *lo_q, *up_q, *lo_n, *up_n;
    const AT *lo_v, *up_v;
    int T, nt, nb, mid;
    GridBar *bar;
    int *err;
    int cr;            // cyclic reduction (FP32, tensor cores) instead of the two-ended elimination
    const int *crs;    // its schedule
    AT *W;             // its dense couplings and products, [slot - nb][T][T]
    int tc;            // FP32 products on the tensor cores (the handle's set-up choice)
};

// Out[r0+i][c] (=, -=) sum_e M[r0+i][uq[c][e]] uv[c][e] for a chunk of FROWS rows.
// A thread takes CPT columns at once, so the coupling loads of all of them are in
// flight together (each column's terms are still summed in entry order).
template <typename AT>
__device__ void rows_times_up(AT *rows, const AT *M, AT *Out, const int *uq, const AT *uv,
                              const int *un, int T, int r0, bool subtract) {
    {
        // FROWS x T contiguous values, 16-byte loads in batches of 8 per thread
        constexpr int VEC = 16 / sizeof(AT);
        using V16 = typename std::conditional<sizeof(AT) == 4, float4, double2>::type;
        const V16 *src = reinterpret_cast<const V16 *>(M + (long long)r0 * T);
        V16 *dst = reinterpret_cast<V16 *>(rows);
        const int nv = FROWS * T / VEC;
        for (int base = 0; base < nv; base += 8 * 256) {
            V16 buf[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int e = base + threadIdx.x + 256 * m;
                if (e < nv) buf[m] = __ldcg(src + e);
            }
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int e = base + threadIdx.x + 256 * m;
                if (e < nv) dst[e] = buf[m];
            }
        }
    }
    __syncthreads();
    constexpr int CPT = sizeof(AT) == 4 ? 4 : 2;   // register budget
    const int nb = blockDim.x;
    for (int c0 = threadIdx.x; c0 < T; c0 += CPT * nb) {
        AT acc[CPT][FROWS];
        int ne[CPT], nmax = 0;
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
            const int c = c0 + j * nb;
            ne[j] = c < T ? un[c] : 0;
            nmax = max(nmax, ne[j]);
#pragma unroll
            for (int i = 0; i < FROWS; ++i) acc[j][i] = (AT)0;
        }
        // transposed ELL: entry e of column c at [e * T + c] (coalesced)
        for (int e0 = 0; e0 < nmax; e0 += 4) {
            int qb[CPT][4];
            AT vb[CPT][4];
#pragma unroll
            for (int j = 0; j < CPT; ++j)
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const bool ok = e0 + m < ne[j];
                    const long long at = (long long)(e0 + m) * T + c0 + j * nb;
                    qb[j][m] = ok ? uq[at] : 0;
                    vb[j][m] = ok ? uv[at] : (AT)0;
                }
#pragma unroll
            for (int j = 0; j < CPT; ++j)
#pragma unroll
                for (int m = 0; m < 4; ++m)
#pragma unroll
                    for (int i = 0; i < FROWS; ++i) acc[j][i] += rows[i * T + qb[j][m]] * vb[j][m];
        }
        AT prev[CPT][FROWS];
#pragma unroll
        for (int j = 0; j < CPT; ++j)
#pragma unroll
            for (int i = 0; i < FROWS; ++i) {
                const int c = c0 + j * nb;
                prev[j][i] = subtract && c < T ? __ldcg(Out + (long long)(r0 + i) * T + c) : (AT)0;
            }
#pragma unroll
        for (int j = 0; j < CPT; ++j)
#pragma unroll
            for (int i = 0; i < FROWS; ++i) {
                const int c = c0 + j * nb;
                if (c < T) Out[(long long)(r0 + i) * T + c] = subtract ? prev[j][i] - acc[j][i] : acc[j][i];
            }
    }
    __syncthreads();
}

constexpr int ERG = 8;     // rows of C_e per item of the gathered sparse product

// Shared memory of sparse_rows_times for block size T.
__host__ __device__ constexpr size_t edge_rows_smem(int T, size_t esz) {
    return (size_t)(T / 32 + 32) * sizeof(int) + (size_t)ERG * ELLW * sizeof(int) +
           (size_t)ERG * ERG * ELLW * esz + 16;
}

// out[r][c] = sum_e lv[r][e] Inv[lq[r][e]][c] for the ERG consecutive rows r of one
// item (row-wise ELL, ELLW entries per row, ln[r] used): the rows' coupled
// positions are merged into one sorted list U (a bitmap and its ranks), their
// values scattered into a dense ERG x |U| block in shared memory, and every row of
// Inv in U is read once per item for all ERG outputs (neighbouring rows couple to
// nearly the same cells), with NB 16-byte loads in flight per thread. Terms are
// summed in the order of U.
template <typename AT>
__device__ void sparse_rows_times(const AT *Inv, const int *lq, const AT *lv, const int *ln, AT *out, int T,
                                  unsigned char *smem) {
    constexpr int VEC = 16 / sizeof(AT), NB = 8;
    using V16 = typename std::conditional<sizeof(AT) == 4, float4, double2>::type;
    const int nw = T / 32;
    unsigned *bits = reinterpret_cast<unsigned *>(smem);               // [nw]
    int *wpre = reinterpret_cast<int *>(bits + nw);                     // [32] per-lane prefix scratch
    int *U = wpre + 32;                                                 // [ERG * ELLW]
    AT *coef = reinterpret_cast<AT *>(                                  // [ERG][ERG * ELLW]
        (reinterpret_cast<uintptr_t>(U + ERG * ELLW) + 15) & ~(uintptr_t)15);
    __shared__ int s_k;
    __syncthreads();                      // the shared memory of the previous item is free
    for (int w = threadIdx.x; w < nw; w += blockDim.x) bits[w] = 0u;
    __syncthreads();
    for (int t = threadIdx.x; t < ERG * ELLW; t += blockDim.x) {
        const int r = t / ELLW, e = t % ELLW;
        if (e < ln[r]) {
            const int q = lq[(long long)r * ELLW + e];
            atomicOr(&bits[q >> 5], 1u << (q & 31));
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {               // exclusive prefix of the words' bit counts
        const int lane = threadIdx.x, per = (nw + 31) / 32;
        int c = 0;
        for (int w = lane * per; w < min(nw, lane * per + per); ++w) c += __popc(bits[w]);
        int inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        wpre[lane] = inc - c;
        if (lane == 31) s_k = inc;
    }
    __syncthreads();
    const int K = s_k, per = (nw + 31) / 32;
    auto rank = [&](int q) {              // position of q in U
        const int w = q >> 5, l = w / per;
        int rk = wpre[l];
        for (int x = l * per; x < w; ++x) rk += __popc(bits[x]);
        return rk + __popc(bits[w] & ((1u << (q & 31)) - 1u));
    };
    for (int w = threadIdx.x; w < nw; w += blockDim.x) {
        unsigned m = bits[w];
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            const int q = 32 * w + b;
            U[rank(q)] = q;
        }
    }
    for (int t = threadIdx.x; t < ERG * K; t += blockDim.x) coef[t] = (AT)0;
    __syncthreads();
    for (int t = threadIdx.x; t < ERG * ELLW; t += blockDim.x) {
        const int r = t / ELLW, e = t % ELLW;
        if (e < ln[r]) coef[r * K + rank(lq[(long long)r * ELLW + e])] = lv[(long long)r * ELLW + e];
    }
    __syncthreads();
    const int ng = T / VEC;
    for (int g = threadIdx.x; g < ng; g += blockDim.x) {
        AT acc[ERG][VEC];
#pragma unroll
        for (int r = 0; r < ERG; ++r)
#pragma unroll
            for (int q = 0; q < VEC; ++q) acc[r][q] = (AT)0;
        for (int k0 = 0; k0 < K; k0 += NB) {
            V16 buf[NB];
#pragma unroll
            for (int m = 0; m < NB; ++m)
                if (k0 + m < K) buf[m] = __ldcg(reinterpret_cast<const V16 *>(Inv + (long long)U[k0 + m] * T) + g);
#pragma unroll
            for (int m = 0; m < NB; ++m)
                if (k0 + m < K) {
                    const AT *v = reinterpret_cast<const AT *>(&buf[m]);
#pragma unroll
                    for (int r = 0; r < ERG; ++r) {
                        const AT w = coef[r * K + k0 + m];
#pragma unroll
                        for (int q = 0; q < VEC; ++q) acc[r][q] += w * v[q];
                    }
                }
        }
#pragma unroll
        for (int r = 0; r < ERG; ++r) {
            V16 o;
            AT *ov = reinterpret_cast<AT *>(&o);
#pragma unroll
            for (int q = 0; q < VEC; ++q) ov[q] = acc[r][q];
            reinterpret_cast<V16 *>(out + (long long)r * T)[g] = o;
        }
    }
    __syncthreads();                      // the next item may overwrite the staged couplings
}

// In-place inverses of the blocks blk[0..nblk) (one chain each), panel by
// panel; the pivot tile of the next panel of each block is updated and
// inverted by a CTA of its own (when the grid has more CTAs than chains).
template <typename AT>
__device__ __forceinline__ bool invert_blocks(const FacArgs<AT> &a, TileSmem<AT> &ts, const int *blk, int nblk,
                              unsigned &epoch, int b, int G, TcState &tcs) {
    const int T = a.T, nt = a.nt;
    const long long bsz = (long long)T * T;
    // prologue: pivot tile 0 and the row panel of step 0
    for (int c = b; c < nblk; c += G) tile_invert(ts, a.D + blk[c] * bsz, T, 0, a.err);
    if (!grid_barrier(a.bar, a.err, epoch, G)) return false;
    {
        const int n0 = 4 * (nt - 1);
        for (int it = b; it < nblk * n0; it += G) {
            AT *Dk = a.D + blk[it / n0] * bsz;
            const int j = ((it % n0) >> 2) + 1, q = it & 3;
            subtile_product<AT, 64, 16, 2, 2>(ts, Dk, Dk, Dk, T, 0, 0, 0, j, 0, j, 0, 16 * q, (AT)1, false);
        }
    }
    if (!grid_barrier(a.bar, a.err, epoch, G)) return false;
    const bool own = G > nblk;              // CTAs 0..nblk-1 do only the pivot tiles
    for (int p = 0; p < nt; ++p) {
        const bool nxt = p + 1 < nt;
        // phase A: trailing update D_ij -= D_ip D_pj (i, j != p); the next
        // pivot tile is updated and inverted by one CTA per chain
        const int nu = (nt - 1) * (nt - 1);
        const int nz = nxt ? 4 : 0;           // Z = -D_{p+1,p} P_p into the chain's scratch strip
        const int dpiv = p * (nt - 1) + p;    // update item of tile (p+1, p+1)
        const int nreg = nu - (nxt ? 1 : 0) + nz;
        auto update = [&](int c, int t) {     // update item t (in 0..nu) of chain c
            AT *Dk = a.D + blk[c] * bsz;
            const int bi = t / (nt - 1), bj = t % (nt - 1);
            const int i = bi < p ? bi : bi + 1, j = bj < p ? bj : bj + 1;
            subtile_product<AT, 64, 64, 4, 4>(ts, Dk, Dk, Dk, T, i, p, p, j, i, j, 0, 0, (AT)-1, true);
        };
        // FP32 with the tensor path: the items are pairs of vertically adjacent tiles
        // (rows 2 pb, 2 pb + 1) of a tile column j != p, one MMA group per pair; a pair
        // with the pivot row or the next pivot tile (updated by its own CTA) in it
        // keeps its other tile on the CUDA-core product
        const bool tcp = sizeof(AT) == 4 && tcs.on;
        const int npair = (nt + 1) / 2, npi = (nt - 1) * npair;
        const int nitem = tcp ? npi + nz : nreg;
        auto z_item = [&](int c, int z) {
            AT *Dk = a.D + blk[c] * bsz;
            subtile_product<AT, 16, 64, 2, 2>(ts, Dk, Dk, a.Z + (long long)c * TILE * T, T, p + 1, p,
                                              p, p, 0, 0, 16 * z, 0, (AT)-1, false);
        };
        auto regular = [&](int q) {            // q in 0..nblk*nitem
            const int c = q / nitem, r = q % nitem;
            if (r >= nitem - nz) {
                z_item(c, r - (nitem - nz));
                return;
            }
            if (!tcp) {
                update(c, nxt && r >= dpiv ? r + 1 : r);
                return;
            }
            if constexpr (sizeof(AT) == 4) {
                AT *Dk = a.D + blk[c] * bsz;
                const int bj = r / npair, pb = r % npair;
                const int j = bj < p ? bj : bj + 1;
                auto ok = [&](int i) { return i < nt && i != p && !(nxt && i == p + 1 && j == p + 1); };
                const int i0 = 2 * pb, i1 = 2 * pb + 1;
                const bool o0 = ok(i0), o1 = ok(i1);
                if (o0 && o1) {
                    tc_pair_update(*reinterpret_cast<TcSmem *>(&ts), tcs, Dk, T, i0, p, j, a.err);
                } else if (o0 || o1) {
                    const int i = o0 ? i0 : i1;
                    subtile_product<AT, 64, 64, 4, 4>(ts, Dk, Dk, Dk, T, i, p, p, j, i, j, 0, 0, (AT)-1, true);
                }
            }
        };
        auto special = [&](int c) {         // tile (p+1, p+1) -= D_{p+1,p} D_{p,p+1}, then inverted
            AT *Dk = a.D + blk[c] * bsz;
            tile_invert(ts, Dk, T, p + 1, a.err, Dk + (long long)(p + 1) * TILE * T + p * TILE,
                        Dk + (long long)p * TILE * T + (p + 1) * TILE);
        };
        if (nxt && own) {
            if (b < nblk) special(b);
            else
                for (int q = b - nblk; q < nblk * nitem; q += G - nblk) regular(q);
        } else {
            const int ns = nxt ? nblk : 0;
            for (int it = b; it < ns + nblk * nitem; it += G) {
                if (it < ns) special(it);
                else regular(it - ns);
            }
        }
        if (!grid_barrier(a.bar, a.err, epoch, G)) return false;
        // phase B: column panel of step p (D_ip = -D_ip P_p, i != p, p+1),
        // row panel of step p+1 (D_{p+1,j} = P_{p+1} D_{p+1,j}, j != p, p+1),
        // and tile (p+1, p) = P_{p+1} (-D_{p+1,p} P_p)
        const int ncol = nt - 1 - (nxt ? 1 : 0);
        const int nrow = nxt ? nt - 2 : 0;
        const int nB = 4 * ncol + 4 * nrow + (nxt ? 4 : 0);
        for (int it2 = b; it2 < nblk * nB; it2 += G) {
            const int c = it2 / nB, it = it2 % nB;
            AT *Dk = a.D + blk[c] * bsz;
            if (it < 4 * ncol) {
                const int t = it >> 2, q = it & 3;
                const int i = t < p ? t : t + 2;      // skip p and p + 1
                subtile_product<AT, 16, 64, 2, 2>(ts, Dk, Dk, Dk, T, i, p, p, p, i, p, 16 * q, 0,
                                                  (AT)-1, false);
            } else if (it < 4 * ncol + 4 * nrow) {
                const int e = it - 4 * ncol;
                const int t = e >> 2, q = e & 3;
                const int j = t < p ? t : t + 2;      // skip p and p + 1
                subtile_product<AT, 64, 16, 2, 2>(ts, Dk, Dk, Dk, T, p + 1, p + 1, p + 1, j, p + 1, j,
                                                  0, 16 * q, (AT)1, false);
            } else {                                  // D_{p+1,p} = P_{p+1} Z (column strips)
                const int q = it - 4 * ncol - 4 * nrow;
                subtile_product<AT, 64, 16, 2, 2>(ts, Dk, a.Z + (long long)c * TILE * T, Dk, T, p + 1,
                                                  p + 1, 0, 0, p + 1, p, 0, 16 * q, (AT)1, false);
            }
        }
        if (!grid_barrier(a.bar, a.err, epoch, G)) return false;
    }
    return true;
}

// Two-ended block elimination (see the header): at step s the top chain
// inverts block s and the bottom chain block nb-1-s, then both form C_e, F_e
// of their edge and update their target block; the middle block is inverted
// last.
// The factorisation of one handle by a group of G co-resident CTAs (b: this CTA's
// index in the group).
// ---------------------------------------------------------------------------
// cyclic reduction of the block tridiagonal system (FP32 on the tensor cores)
// ---------------------------------------------------------------------------
//
// Round r takes the active blocks L_r (initially all, in order) and eliminates
// those at odd positions; their inverses are computed concurrently (the same
// in-place Gauss-Jordan as above, one chain per block). With L(k), U(k) the
// couplings of active block k to its previous / next active block (the
// off-diagonal blocks of the operator in the first round), every kept block e
// between eliminated neighbours om, op receives
//     X_e = L(e) Inv_om,  Y_e = U(e) Inv_op,
//     D_e -= X_e U(om) + Y_e L(op),  L(e) <- -X_e L(om),  U(e) <- -Y_e U(op),
// and every eliminated block o keeps V_o = Inv_o L(o), W_o = Inv_o U(o). The last
// active block is inverted at the end. Solve: per round, x_o = Inv_o g_o and
// g_e -= X_e g_om + Y_e g_op; x_last = Inv_last g_last; then back through the
// rounds, x_o -= V_o x_prev + W_o x_next. The depth is ceil(log2(nb)) + 1 block
// inversions instead of about nb / 2 + 1, at the price of dense T x T products
// (all of them on tcgen05), which is why only the FP32 form with the tensor path
// takes it. Every product is one task of the schedule, computed as items of a
// 128-row pair of tiles and a tile column.
//
// Schedule (ints): nround, last; per round: nE, E[nE]; then two phases of
// products, each ntask followed by ntask records CrTask. A block slot s < nb is
// diagonal block s (D, inverted in place when eliminated), s >= nb is
// W + (s - nb) T^2: the dense couplings L(k) at slot nb + k, U(k) at 2 nb + k,
// then the products.
struct CrTask {
    int out, acc, sign, a1, b1, a2, b2, pad;   // Out (=, +=) sign (A1 B1 [+ A2 B2]); a2 < 0: one term
};

template <typename AT>
__device__ __forceinline__ AT *cr_slot(const FacArgs<AT> &a, int s) {
    const long long bsz = (long long)a.T * a.T;
    return s < a.nb ? a.D + s * bsz : a.W + (long long)(s - a.nb) * bsz;
}

template <typename AT>
__device__ void cr_factor_body(const FacArgs<AT> &a, int b, int G, TcState &tcs) {
    if constexpr (sizeof(AT) == 4) {
        extern __shared__ __align__(16) unsigned char smem_raw[];
        TileSmem<AT> &ts = *reinterpret_cast<TileSmem<AT> *>(smem_raw);
        TcSmem &tsm = *reinterpret_cast<TcSmem *>(smem_raw);
        const int nt = a.nt, per = ((nt + 1) / 2) * nt;   // items of one product
        if (!tcs.on) {                     // the reduction needs the tensor path
            if (threadIdx.x == 0) atomicExch(a.err, ERR_ELL);
            return;
        }
        const int *s = a.crs;
        const int nround = s[0];
        const int *last = s + 1;
        s += 2;
        unsigned epoch = 0;
        for (int r = 0; r < nround; ++r) {
            const int nE = s[0];
            if (!invert_blocks(a, ts, s + 1, nE, epoch, b, G, tcs)) return;
            s += 1 + nE;
            for (int ph = 0; ph < 2; ++ph) {
                const int n = s[0];
                const CrTask *tk = reinterpret_cast<const CrTask *>(s + 1);
                for (int it = b; it < n * per; it += G) {
                    const CrTask t = tk[it / per];
                    const int q = it % per, pr = q / nt, j = q % nt;
                    tc_gemm_pair(tsm, tcs, cr_slot(a, t.out), a.T, pr, j, cr_slot(a, t.a1), cr_slot(a, t.b1),
                                 t.a2 >= 0 ? cr_slot(a, t.a2) : nullptr, t.a2 >= 0 ? cr_slot(a, t.b2) : nullptr,
                                 t.acc != 0, (float)t.sign, a.err);
                }
                s += 1 + 8 * n;
                if (!grid_barrier(a.bar, a.err, epoch, G)) return;
            }
        }
        invert_blocks(a, ts, last, 1, epoch, b, G, tcs);
    }
}

template <typename AT>
__device__ __forceinline__ void coarse_factor_body(const FacArgs<AT> &a, int b, int G, TcState &tcs) {
    if (a.cr) {
        cr_factor_body(a, b, G, tcs);
        return;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem<AT> &ts = *reinterpret_cast<TileSmem<AT> *>(smem_raw);
    AT *rows = reinterpret_cast<AT *>(smem_raw);
    const int T = a.T, nb = a.nb, mid = a.mid;
    const long long bsz = (long long)T * T;
    const int ntop = mid, nbot = nb - 1 - mid;
    const int nsteps = max(ntop, nbot);
    unsigned epoch = 0;
    for (int s = 0; s <= nsteps; ++s) {
        int blk[2], edg[2], nblk = 0, ne = 0;
        if (s < nsteps) {
            if (s < ntop) { blk[nblk++] = s; edg[ne++] = s; }
            if (s < nbot) { blk[nblk++] = nb - 1 - s; edg[ne++] = nb - 2 - s; }
        } else {
            blk[nblk++] = mid;
        }
        if (!invert_blocks(a, ts, blk, nblk, epoch, b, G, tcs)) return;
        if (s == nsteps) break;
        const long long ell = (long long)T * ELLW;
        const int nchunk = T / FROWS;
        const int nC = T / ERG;                             // C_e: ERG rows per item
        const int nE = nC + nchunk;
        for (int it2 = b; it2 < ne * nE; it2 += G) {
            const int e = edg[it2 / nE], it = it2 % nE;
            const AT *Inv = a.D + edge_pivot(e, mid) * bsz;
            if (it < nC) {                                  // C_e rows = A(target, pivot) rows * Inv
                const int r0 = it * ERG;
                const long long at = e * ell + (long long)r0 * ELLW;
                sparse_rows_times(Inv, a.lo_q + at, a.lo_v + at, a.lo_n + (long long)e * T + r0,
                                  a.C + e * bsz + (long long)r0 * T, T, smem_raw);
            } else {                                        // F_e = Inv A(pivot, target)
                rows_times_up(rows, Inv, a.F + e * bsz, a.up_q + e * ell, a.up_v + e * ell,
                              a.up_n + (long long)e * T, T, (it - nC) * FROWS, false);
            }
        }
        if (!grid_barrier(a.bar, a.err, epoch, G)) return;
        for (int it2 = b; it2 < ne * nchunk; it2 += G) {    // S_target -= C_e A(pivot, target)
            const int e = edg[it2 / nchunk], it = it2 % nchunk;
            rows_times_up(rows, a.C + e * bsz, a.D + edge_target(e, mid) * bsz, a.up_q + e * ell,
                          a.up_v + e * ell, a.up_n + (long long)e * T, T, it * FROWS, true);
        }
        if (!grid_barrier(a.bar, a.err, epoch, G)) return;
    }
}

// Tensor memory and the MMA mbarrier of a factorisation CTA (FP32 with the tensor
// path): allocated before the body, freed after it on every return path.
template <typename AT>
__device__ __forceinline__ void tc_begin(TcState &tcs, unsigned *slot, unsigned long long *mbar, bool want) {
    tcs.on = false;
    tcs.tmem = 0;
    tcs.mbar = mbar;
    tcs.phase = 0;
    if (sizeof(AT) != 4 || !want) return;
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;"
                     ::"r"((unsigned)__cvta_generic_to_shared(slot)) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;"
                     ::"r"((unsigned)__cvta_generic_to_shared(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tcs.tmem = *slot;
    tcs.on = true;
}
template <typename AT>
__device__ __forceinline__ void tc_end(const TcState &tcs) {
    if (sizeof(AT) != 4 || !tcs.on) return;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tcs.tmem) : "memory");
}

template <typename AT>
__global__ void __launch_bounds__(256) k_coarse_factor(FacArgs<AT> a, int use_tc) {
    __shared__ unsigned tmem_slot;
    __shared__ unsigned long long mbar;
    TcState tcs;
    tc_begin<AT>(tcs, &tmem_slot, &mbar, use_tc != 0);
    coarse_factor_body(a, blockIdx.x, gridDim.x, tcs);
    tc_end<AT>(tcs);
}

// The factorisations of several handles in one cooperative launch: handle h takes
// CTAs first[h] .. first[h] + size[h] - 1 and its own barrier word; handles off in
// `active` return at once.
template <typename AT>
__global__ void __launch_bounds__(256) k_coarse_factor_batch(const FacArgs<AT> *args, const int *cta_inst,
                                                             const int *first, const int *size,
                                                             const unsigned char *active) {
    const int h = cta_inst[blockIdx.x];
    if (!active[h]) return;
    // the handle's products on the tensor cores when its set-up chose them (FP32),
    // as in its single factorisation
    __shared__ unsigned tmem_slot;
    __shared__ unsigned long long mbar;
    TcState tcs;
    tc_begin<AT>(tcs, &tmem_slot, &mbar, args[h].tc != 0 || args[h].cr != 0);
    coarse_factor_body(args[h], blockIdx.x - first[h], size[h], tcs);
    tc_end<AT>(tcs);
}

// ---------------------------------------------------------------------------
// cooperative solve: restriction, block forward / backward sweeps, prolongation
// ---------------------------------------------------------------------------

template <typename AT>
struct SolArgs {
    const double *t;
    double *z;
    int accumulate;
    Interp P;
    CGeom G;
    const int *pos;
    const AT *E, *C, *F;
    AT *g, *x;
    AT *rx, *ry;
    GridBar *bar;
    int *err;
    int npf;   // matrix rows per warp prefetched into shared memory per stage (0..2)
    int cr;            // cyclic reduction: the block sweeps follow its solve schedule
    const int *crs;
    const AT *W;
    AT *xn;            // the coarse solution in natural order (written with its final values)
    const int *cell;   // block position -> natural coarse index or -1
    int prolong;       // 1: the cooperative kernel ends with z (+)= P x; 0: k_coarse_prolong does it
};

__device__ __forceinline__ void cp_async16_cg(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit_all() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// dot of a shared-memory matrix row with a shared-memory vector; lane l reads the
// 16-byte pieces l, l + 32, ... (the pieces it copied itself)
template <typename AT>
__device__ __forceinline__ AT row_dot_s(const AT *row, const AT *xs, int T, int lane) {
    constexpr int VEC = 16 / sizeof(AT);
    using V16 = typename std::conditional<sizeof(AT) == 4, float4, double2>::type;
    const V16 *rv = reinterpret_cast<const V16 *>(row);
    const V16 *xv = reinterpret_cast<const V16 *>(xs);   // 16-byte reads: no bank conflicts
    AT acc = 0;
    for (int v = lane; v < T / VEC; v += 32) {
        const V16 b = rv[v], x = xv[v];
        const AT *w = reinterpret_cast<const AT *>(&b);
        const AT *y = reinterpret_cast<const AT *>(&x);
#pragma unroll
        for (int q = 0; q < VEC; ++q) acc += w[q] * y[q];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    return acc;
}

// dot of a matrix row with a shared-memory vector, 16-byte loads (T is a
// multiple of 64 and rows start 16-byte aligned)
// (GX: the vector is in global memory and read through L2 only)
template <typename AT, bool GX = false>
__device__ __forceinline__ AT row_dot(const AT *row, const AT *xs, int T, int lane) {
    AT acc = 0;
    constexpr int VEC = 16 / sizeof(AT);
    using V16 = typename std::conditional<sizeof(AT) == 4, float4, double2>::type;
    const V16 *rv = reinterpret_cast<const V16 *>(row), *xv = reinterpret_cast<const V16 *>(xs);
    auto X = [&](int i) { return GX ? __ldcg(xv + i) : xv[i]; };   // 16-byte reads
    const int nv = T / VEC;
    for (int base = lane; base < nv; base += 32 * 8) {
        V16 buf[8];
#pragma unroll
        for (int m = 0; m < 8; ++m)
            if (base + 32 * m < nv) buf[m] = __ldcg(rv + base + 32 * m);
#pragma unroll
        for (int m = 0; m < 8; ++m)
            if (base + 32 * m < nv) {
                const V16 xq = X(base + 32 * m);
                const AT *v = reinterpret_cast<const AT *>(&buf[m]);
                const AT *y = reinterpret_cast<const AT *>(&xq);
#pragma unroll
                for (int q = 0; q < VEC; ++q) acc += v[q] * y[q];
            }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    return acc;
}

// xs <- xsrc (T values, 16-byte loads, read through L2 only)
template <typename AT>
__device__ void stage_vector(const AT *xsrc, AT *xs, int T) {
    using V16 = typename std::conditional<sizeof(AT) == 4, float4, double2>::type;
    const int nv = T / (16 / (int)sizeof(AT));
    const V16 *src = reinterpret_cast<const V16 *>(xsrc);
    V16 *dst = reinterpret_cast<V16 *>(xs);
    for (int base = threadIdx.x; base < nv; base += 4 * blockDim.x) {
        V16 buf[4];
#pragma unroll
        for (int m = 0; m < 4; ++m)
            if (base + m * (int)blockDim.x < nv) buf[m] = __ldcg(src + base + m * blockDim.x);
#pragma unroll
        for (int m = 0; m < 4; ++m)
            if (base + m * (int)blockDim.x < nv) dst[base + m * blockDim.x] = buf[m];
    }
    __syncthreads();
}

// The coarse correction of one handle by a group of ng co-resident CTAs (b: this
// CTA's index in the group); t: fine residual, z: fine correction.
// Block sweeps of the cyclic reduction: phases separated by grid barriers, each a
// list of tasks out (=, -=) M1 v1 [+ M2 v2] over the T rows of a block, one warp
// per row (matrix rows from HBM, vectors through L2). Schedule: nphase, then per
// phase ntask and ntask records {out, 0, sub, m1, v1, m2, v2, 0}; a vector is
// (0 for g, 1 for x) << 16 | block, a matrix a block slot as in the factorisation
// (m2 < 0: one term).
template <typename AT>
__device__ bool cr_sweeps(const SolArgs<AT> &a, int b, int ng, unsigned &epoch) {
    const int T = a.G.T, nb = a.G.nb, lane = threadIdx.x & 31, wpb = blockDim.x / 32;
    const int wg = b * wpb + (threadIdx.x >> 5), nwt = ng * wpb;
    const long long bsz = (long long)T * T;
    auto mat = [&](int q) -> const AT * { return q < nb ? a.E + q * bsz : a.W + (long long)(q - nb) * bsz; };
    auto vec = [&](int v) -> AT * { return ((v >> 16) ? a.x : a.g) + (long long)(v & 0xffff) * T; };
    const int *s = a.crs;
    const int nph = *s++;
    for (int ph = 0; ph < nph; ++ph) {
        const int n = *s++;
        const int *tk = s;
        s += 8 * n;
        for (int r = wg; r < n * T; r += nwt) {
            const int *t = tk + 8 * (r / T);
            const int i = r % T;
            AT acc = 0;
#pragma unroll 1
            for (int m = 0; m < 2 && t[3 + 2 * m] >= 0; ++m)
                acc += row_dot<AT, true>(mat(t[3 + 2 * m]) + (long long)i * T, vec(t[4 + 2 * m]), T, lane);
            if (lane == 0) {
                AT *y = vec(t[0]) + i;
                *y = t[2] ? __ldcg(y) - acc : acc;
            }
        }
        if (!grid_barrier(a.bar, a.err, epoch, ng)) return false;
    }
    return true;
}

// z (+)= P x for the fine cells p0, p0 + stride, ..., four at a time with their loads
// in flight together; the coarse values from the natural-order copy (the cyclic
// reduction's sweeps leave x in block order only)
template <typename AT>
__device__ __forceinline__ void coarse_prolong_range(const SolArgs<AT> &a, double *z, long long start,
                                                     long long stride) {
    const CGeom &G = a.G;
    const Interp &P = a.P;
    const long long N = (long long)G.nx * G.ny * G.nz;
    for (long long p0 = start; p0 < N; p0 += 4 * stride) {
        AT sv[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const long long p = p0 + m * stride;
            sv[m] = 0;
            if (p >= N) continue;
            const int ax = (int)(p % G.nx), ay = (int)((p / G.nx) % G.ny),
                      az = (int)(p / ((long long)G.nx * G.ny));
            const int Ix[2] = {P.ia[0][ax], P.ib[0][ax]};
            const int Iy[2] = {P.ia[1][ay], P.ib[1][ay]};
            const int Iz[2] = {P.ia[2][az], P.ib[2][az]};
            const AT Wx[2] = {(AT)P.wa[0][ax], (AT)P.wb[0][ax]};
            const AT Wy[2] = {(AT)P.wa[1][ay], (AT)P.wb[1][ay]};
            const AT Wz[2] = {(AT)P.wa[2][az], (AT)P.wb[2][az]};
            AT s = 0;
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int v = 0; v < 2; ++v)
#pragma unroll
                    for (int w = 0; w < 2; ++w) {
                        const AT wt = Wx[w] * Wy[v] * Wz[u];
                        const int I = Ix[w] + G.cx * (Iy[v] + G.cy * Iz[u]);
                        if (wt != (AT)0) s += wt * (a.cr ? __ldcg(a.x + a.pos[I]) : __ldcg(a.xn + I));
                    }
            sv[m] = s;
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const long long p = p0 + m * stride;
            if (p < N) { if (a.accumulate) z[p] += (double)sv[m]; else z[p] = (double)sv[m]; }
        }
    }
}

template <typename AT>
__device__ __forceinline__ void coarse_solve_body(const SolArgs<AT> &a, int b, int ng, const double *t, double *z) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AT *xs = reinterpret_cast<AT *>(smem_raw);
    const CGeom &G = a.G;
    const Interp &P = a.P;
    const int T = G.T;
    const long long bsz = (long long)T * T;
    const int lane = threadIdx.x & 31, wpb = blockDim.x / 32;
    unsigned epoch = 0;
    // Block sweeps as 2 nsteps + 1 stages separated by grid barriers: forward along
    // both chains (g_target -= C_e g_pivot, and x_pivot = Inv_pivot g_pivot), the
    // middle block (x_mid = Inv_mid g_mid), back along both chains
    // (x_pivot -= F_e x_target). The matrix rows of a stage do not depend on the
    // vectors, so each warp copies its first npf rows of the next stage into shared
    // memory before the barrier (the copies overlap the barrier and the next
    // vector staging); further rows are read directly.
    const int nb = G.nb, mid = G.mid, ntop = mid, nbot = nb - 1 - mid;
    const int nsteps = max(ntop, nbot), nstage = 2 * nsteps + 1;
    const int wg = b * wpb + (threadIdx.x >> 5), nwt = ng * wpb;
    AT *rbuf = xs + 2 * (long long)T + (long long)(threadIdx.x >> 5) * a.npf * T;
    constexpr int VEC = 16 / sizeof(AT);
    auto edges_of = [&](int st, int *edg) {
        int ne = 0;
        if (st < nsteps) {
            if (st < ntop) edg[ne++] = st;
            if (st < nbot) edg[ne++] = nb - 2 - st;
        } else if (st > nsteps) {
            const int q = st - nsteps - 1;
            if (q < ntop) edg[ne++] = ntop - 1 - q;
            if (q < nbot) edg[ne++] = mid + q;
        }
        return ne;
    };
    auto nrows_of = [&](int st, int ne) { return st < nsteps ? ne * 2 * T : (st == nsteps ? T : ne * T); };
    auto row_ptr = [&](int st, const int *edg, int r) -> const AT * {
        if (st < nsteps) {
            const int c = r / (2 * T), rr = r % (2 * T), e = edg[c];
            return rr < T ? a.E + edge_pivot(e, mid) * bsz + (long long)rr * T
                          : a.C + e * bsz + (long long)(rr - T) * T;
        }
        if (st == nsteps) return a.E + mid * bsz + (long long)r * T;
        return a.F + edg[r / T] * bsz + (long long)(r % T) * T;
    };
    auto prefetch = [&](int st) {
        if (st < nstage) {
            int edg[2];
            const int nr = nrows_of(st, edges_of(st, edg));
            for (int k = 0; k < a.npf; ++k) {
                const int r = wg + k * nwt;
                if (r >= nr) break;
                const AT *src = row_ptr(st, edg, r);
                for (int v = lane; v < T / VEC; v += 32) cp_async16_cg(rbuf + (long long)k * T + v * VEC, src + v * VEC);
            }
        }
        cp_async_commit_all();
    };
    prefetch(0);   // lands during the restriction
    // g = R t with R = P^T = Pz^T Py^T Px^T, one axis per pass
    const long long gtid = b * (long long)blockDim.x + threadIdx.x;
    const long long gstride = (long long)ng * blockDim.x;
    const long long n1 = (long long)G.cx * G.ny * G.nz;
    // (each pass: the support's weights from the per-axis table and its values
    // loaded in batches of 8 before any is used; terms summed in index order)
    for (long long e = gtid; e < n1; e += gstride) {          // x pass
        const int Ix = (int)(e % G.cx);
        const long long yz = e / G.cx;
        const int x0 = P.lo[0][Ix], nw = P.hi[0][Ix] - x0;
        const double *src = t + yz * G.nx + x0, *wt = P.wt[0] + (long long)Ix * P.W[0];
        AT acc = 0;
        for (int m0 = 0; m0 < nw; m0 += 8) {
            double tv[8], wv[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                tv[m] = m0 + m < nw ? __ldg(src + m0 + m) : 0.0;
                wv[m] = m0 + m < nw ? __ldg(wt + m0 + m) : 0.0;
            }
#pragma unroll
            for (int m = 0; m < 8; ++m)
                if (m0 + m < nw) acc += (AT)wv[m] * (AT)tv[m];
        }
        a.rx[e] = acc;
    }
    if (!grid_barrier(a.bar, a.err, epoch, ng)) { cp_async_wait_all(); return; }
    const long long n2 = (long long)G.cx * G.cy * G.nz;
    for (long long e = gtid; e < n2; e += gstride) {          // y pass
        const int Ix = (int)(e % G.cx), Iy = (int)((e / G.cx) % G.cy);
        const long long az = e / ((long long)G.cx * G.cy);
        const int y0 = P.lo[1][Iy], nw = P.hi[1][Iy] - y0;
        const AT *src = a.rx + Ix + (long long)G.cx * (y0 + (long long)G.ny * az);
        const double *wt = P.wt[1] + (long long)Iy * P.W[1];
        AT acc = 0;
        for (int m0 = 0; m0 < nw; m0 += 8) {
            AT v[8];
            double wv[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                v[m] = m0 + m < nw ? __ldcg(src + (long long)G.cx * (m0 + m)) : (AT)0;
                wv[m] = m0 + m < nw ? __ldg(wt + m0 + m) : 0.0;
            }
#pragma unroll
            for (int m = 0; m < 8; ++m)
                if (m0 + m < nw) acc += (AT)wv[m] * v[m];
        }
        a.ry[e] = acc;
    }
    if (!grid_barrier(a.bar, a.err, epoch, ng)) { cp_async_wait_all(); return; }
    for (long long I = gtid; I < G.Nc; I += gstride) {         // z pass
        const int Ix = (int)(I % G.cx), Iy = (int)((I / G.cx) % G.cy), Iz = (int)(I / ((long long)G.cx * G.cy));
        const int z0 = P.lo[2][Iz], nw = P.hi[2][Iz] - z0;
        const long long cxy = (long long)G.cx * G.cy;
        const AT *src = a.ry + Ix + (long long)G.cx * Iy + cxy * z0;
        const double *wt = P.wt[2] + (long long)Iz * P.W[2];
        const int dst = a.pos[I];
        AT acc = 0;
        for (int m0 = 0; m0 < nw; m0 += 8) {
            AT v[8];
            double wv[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                v[m] = m0 + m < nw ? __ldcg(src + cxy * (m0 + m)) : (AT)0;
                wv[m] = m0 + m < nw ? __ldg(wt + m0 + m) : 0.0;
            }
#pragma unroll
            for (int m = 0; m < 8; ++m)
                if (m0 + m < nw) acc += (AT)wv[m] * v[m];
        }
        a.g[dst] = acc;
    }
    if (!grid_barrier(a.bar, a.err, epoch, ng)) { cp_async_wait_all(); return; }
    if (a.cr && !cr_sweeps(a, b, ng, epoch)) { cp_async_wait_all(); return; }
    for (int st = 0; st < (a.cr ? 0 : nstage); ++st) {
        int edg[2];
        const int ne = edges_of(st, edg);
        if (st < nsteps)
            for (int c = 0; c < ne; ++c)
                stage_vector(a.g + (long long)edge_pivot(edg[c], mid) * T, xs + (long long)c * T, T);
        else if (st == nsteps)
            stage_vector(a.g + (long long)mid * T, xs, T);
        else
            for (int c = 0; c < ne; ++c)
                stage_vector(a.x + (long long)edge_target(edg[c], mid) * T, xs + (long long)c * T, T);
        cp_async_wait_all();
        __syncwarp();
        const int nr = nrows_of(st, ne);
        int k = 0;
        for (int r = wg; r < nr; r += nwt, ++k) {
            // lane 0 first reads what the row updates (the target entry of g, or the
            // pivot entry of x on the way back) and the natural index of a row whose x
            // value becomes final in this stage (the middle block, and the pivot blocks
            // on the way back), so that those loads overlap the dot product
            AT *y = nullptr;
            long long qf = -1;
            if (st < nsteps) {
                const int c = r / (2 * T), rr = r % (2 * T), e = edg[c];
                y = rr < T ? a.x + (long long)edge_pivot(e, mid) * T + rr
                           : a.g + (long long)edge_target(e, mid) * T + (rr - T);
            } else if (st == nsteps) {
                qf = (long long)mid * T + r;
                y = a.x + qf;
            } else {
                qf = (long long)edge_pivot(edg[r / T], mid) * T + (r % T);
                y = a.x + qf;
            }
            const bool rmw = st > nsteps || (st < nsteps && r % (2 * T) >= T);   // y -= acc
            const AT prev = lane == 0 && rmw ? __ldcg(y) : (AT)0;
            const int cf = lane == 0 && qf >= 0 ? a.cell[qf] : -1;
            const AT *xv = xs + (long long)(st < nsteps ? r / (2 * T) : (st == nsteps ? 0 : r / T)) * T;
            const AT acc = k < a.npf ? row_dot_s(rbuf + (long long)k * T, xv, T, lane)
                                     : row_dot(row_ptr(st, edg, r), xv, T, lane);
            if (lane == 0) {
                const AT v = rmw ? prev - acc : acc;
                *y = v;
                if (cf >= 0) a.xn[cf] = v;
            }
        }
        __syncwarp();                      // this warp's reads of its row buffer are done
        prefetch(st + 1);
        if (!grid_barrier(a.bar, a.err, epoch, ng)) { cp_async_wait_all(); return; }
    }
    if (a.prolong) coarse_prolong_range(a, z, gtid, gstride);
}

template <typename AT>
__global__ void __launch_bounds__(256, 2) k_coarse_solve(SolArgs<AT> a) {
    coarse_solve_body(a, blockIdx.x, gridDim.x, a.t, a.z);
}

// The prolongation of a single coarse correction as a kernel of its own (full
// occupancy: the loop is bound by the latency of its table and coarse loads, which
// the cooperative kernel's two CTAs per SM do not hide)
template <typename AT>
__global__ void __launch_bounds__(256) k_coarse_prolong(SolArgs<AT> a) {
    coarse_prolong_range(a, a.z, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                         (long long)gridDim.x * blockDim.x);
}

// The coarse corrections of several handles in one cooperative launch: handle h
// takes CTAs first[h] .. first[h] + size[h] - 1 and its own barrier word; t and z
// are the handles' fine vectors concatenated at off[h]; a handle switched off in
// `active` returns at once (all its CTAs).
template <typename AT>
__global__ void __launch_bounds__(256, 2) k_coarse_solve_batch(const SolArgs<AT> *args, const int *cta_inst,
                                                            const int *first, const int *size,
                                                            const long long *off, const unsigned char *active,
                                                            const double *t, double *z) {
    const int h = cta_inst[blockIdx.x];
    if (!active[h]) return;
    coarse_solve_body(args[h], blockIdx.x - first[h], size[h], t + off[h], z + off[h]);
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------

static int grid_of(long long n, int threads = 256) {
    long long g = (n + threads - 1) / threads;
    return (int)std::max(1LL, std::min(g, 152LL * 16));
}

// One axis of I_{j-1}^j: order 2, tensor-product linear between the bracketing
// coarse centres (Eq. equ:inter-second), constant beyond the outermost ones;
// order 1, the nearest coarse centre (Eq. equ:inter-frist), the lower on ties.
static void interp_axis(int n, int r, std::vector<int> &ia, std::vector<int> &ib,
                        std::vector<double> &wa, std::vector<double> &wb, std::vector<int> &lo,
                        std::vector<int> &hi, int &nc, int order) {
    nc = n > 1 ? (n + r - 1) / r : 1;
    ia.assign(n, 0); ib.assign(n, 0); wa.assign(n, 1.0); wb.assign(n, 0.0);
    std::vector<double> xc(nc);
    for (int I = 0; I < nc; ++I) xc[I] = (r * I + std::min(r * I + r, n)) / 2.0;
    if (n > 1) {
        for (int i = 0; i < n; ++i) {
            const double x = i + 0.5;
            if (order == 1) {
                int best = 0;
                for (int I = 1; I < nc; ++I)
                    if (std::fabs(xc[I] - x) < std::fabs(xc[best] - x)) best = I;
                ia[i] = ib[i] = best; wa[i] = 1.0; wb[i] = 0.0;
                continue;
            }
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

// Zero the grid barriers of a cooperative launch (the arrival counters of n
// barrier words) and set their poll limit, by a kernel rather than a host copy so
// that the reset can be captured in a graph. RAS_BARRIER_POLLS (environment, read
// at every launch) shortens the bounded wait, so that a test can make it run out
// and check the RAS_ETIMEOUT path.
__global__ void k_reset_bars(GridBar *bars, int n, long long polls) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        bars[i].count = 0;
        bars[i].polls = polls;
    }
}

static long long barrier_polls() {
    long long polls = 0;
    if (const char *e = getenv("RAS_BARRIER_POLLS")) polls = atoll(e);
    return polls;
}

long long coarse_barrier_polls() { return barrier_polls(); }

static int reset_bar(Coarse *c, cudaStream_t st) {
    k_reset_bars<<<1, 32, 0, st>>>(c->d_bar, 1, barrier_polls());
    RAS_LAUNCHED();
    return RAS_OK;
}

static Interp interp_of(const Coarse *c) {
    Interp P;
    for (int a = 0; a < 3; ++a) {
        P.ia[a] = c->d_ia[a]; P.ib[a] = c->d_ib[a];
        P.wa[a] = c->d_wa[a]; P.wb[a] = c->d_wb[a];
        P.lo[a] = c->d_lo[a]; P.hi[a] = c->d_hi[a];
        P.wt[a] = c->d_wt[a]; P.W[a] = c->wmax[a];
    }
    return P;
}

static CGeom geom_of(const Coarse *c) {
    CGeom G;
    G.nx = c->nx; G.ny = c->ny; G.nz = c->nz;
    G.cx = c->c[0]; G.cy = c->c[1]; G.cz = c->c[2]; G.Nc = c->Nc;
    G.T = c->T; G.nb = c->nb; G.mid = c->mid;
    return G;
}

// Schedules of the cyclic reduction of nb blocks (layout at cr_factor_body and
// cr_sweeps).
struct CrPlan {
    std::vector<int> fac, sol;
    int nslot = 0;        // W slots: the dense couplings (2 nb) and the products
    int maxE = 1;         // most blocks inverted concurrently
    long long mats = 0;   // T x T matrices one solve reads
};
static void cr_plan(int nb, CrPlan &P) {
    const int LC = nb, UC = 2 * nb, GV = 0, XV = 1 << 16;
    int next = 3 * nb;
    std::vector<int> L(nb);
    std::iota(L.begin(), L.end(), 0);
    P.fac = {0, 0};
    std::vector<std::vector<int>> fwd, bwd;
    auto task = [](std::vector<int> &v, int out, int acc, int sign, int a1, int b1, int a2, int b2) {
        v.insert(v.end(), {out, acc, sign, a1, b1, a2, b2, 0});
    };
    auto stask = [&](std::vector<int> &v, int out, int sub, int m1, int v1, int m2, int v2) {
        v.insert(v.end(), {out, 0, sub, m1, v1, m2, v2, 0});
        P.mats += m2 >= 0 ? 2 : 1;
    };
    int nround = 0;
    while (L.size() > 1) {
        const int n = (int)L.size();
        std::vector<int> E, K, f2, f3, sf, sb;
        for (int i = 1; i < n; i += 2) E.push_back(L[i]);
        P.maxE = std::max(P.maxE, (int)E.size());
        for (int i = 0; i < n; ++i) {
            const int k = L[i];
            const int prev = i > 0 ? L[i - 1] : -1, nxt = i + 1 < n ? L[i + 1] : -1;
            if (i & 1) {                       // eliminated: V = Inv L(k), W = Inv U(k)
                const int vs = next++;
                task(f2, vs, 0, 1, k, LC + k, -1, -1);
                int ws = -1;
                if (nxt >= 0) {
                    ws = next++;
                    task(f2, ws, 0, 1, k, UC + k, -1, -1);
                }
                stask(sf, XV | k, 0, k, GV | k, -1, 0);                            // x_k = Inv g_k
                stask(sb, XV | k, 1, vs, XV | prev, ws, ws >= 0 ? (XV | nxt) : 0);  // x_k -= V x_prev + W x_next
            } else {                           // kept: X = L(k) Inv_prev, Y = U(k) Inv_next
                int xs = -1, ys = -1;
                if (prev >= 0) {
                    xs = next++;
                    task(f2, xs, 0, 1, LC + k, prev, -1, -1);
                }
                if (nxt >= 0) {
                    ys = next++;
                    task(f2, ys, 0, 1, UC + k, nxt, -1, -1);
                }
                if (xs >= 0 || ys >= 0) {      // D_k -= X U(prev) + Y L(next); g_k -= X g_prev + Y g_next
                    const int a1 = xs >= 0 ? xs : ys, b1 = xs >= 0 ? UC + prev : LC + nxt;
                    const int a2 = xs >= 0 && ys >= 0 ? ys : -1, b2 = a2 >= 0 ? LC + nxt : -1;
                    task(f3, k, 1, -1, a1, b1, a2, b2);
                    stask(sf, GV | k, 1, a1, GV | (xs >= 0 ? prev : nxt), a2, a2 >= 0 ? (GV | nxt) : 0);
                }
                if (xs >= 0 && i >= 2) task(f3, LC + k, 0, -1, xs, LC + prev, -1, -1);    // L(k) <- -X L(prev)
                if (ys >= 0 && i + 2 < n) task(f3, UC + k, 0, -1, ys, UC + nxt, -1, -1);  // U(k) <- -Y U(next)
                K.push_back(k);
            }
        }
        P.fac.push_back((int)E.size());
        P.fac.insert(P.fac.end(), E.begin(), E.end());
        P.fac.push_back((int)f2.size() / 8);
        P.fac.insert(P.fac.end(), f2.begin(), f2.end());
        P.fac.push_back((int)f3.size() / 8);
        P.fac.insert(P.fac.end(), f3.begin(), f3.end());
        fwd.push_back(sf);
        bwd.push_back(sb);
        L = K;
        ++nround;
    }
    P.fac[0] = nround;
    P.fac[1] = L[0];
    std::vector<int> fin;
    stask(fin, XV | L[0], 0, L[0], GV | L[0], -1, 0);                              // x_last = Inv g_last
    std::vector<std::vector<int>> phases(fwd.begin(), fwd.end());
    phases.push_back(fin);
    for (int r = nround - 1; r >= 0; --r) phases.push_back(bwd[r]);
    P.sol = {(int)phases.size()};
    for (const auto &ph : phases) {
        P.sol.push_back((int)ph.size() / 8);
        P.sol.insert(P.sol.end(), ph.begin(), ph.end());
    }
    P.nslot = next - nb;
}

template <typename AT>
static int configure_t(Coarse *c) {
    // dynamic opt-in well above any need here and below the per-block limit
    // minus the kernels' static shared memory
    const int big = 200 * 1024;
    RAS_CK(cudaFuncSetAttribute(k_rap<AT>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    RAS_CK(cudaFuncSetAttribute(k_rap_slab<AT>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    RAS_CK(cudaFuncSetAttribute(k_rap125<AT>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    RAS_CK(cudaFuncSetAttribute(k_coarse_factor<AT>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    RAS_CK(cudaFuncSetAttribute(k_coarse_factor_batch<AT>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    RAS_CK(cudaFuncSetAttribute(k_coarse_solve<AT>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    RAS_CK(cudaFuncSetAttribute(k_coarse_solve_batch<AT>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    const int WX = c->wmax[0], WY = c->wmax[1], WZ = c->wmax[2];
    const int WM = std::max(WX, std::max(WY, WZ));
    const size_t tables = sizeof(int) * (size_t)(5 * WY * WX + 25 * WX);
    if (rap_plan(c->wmax, sizeof(AT), big, c->rap_zs, c->rap_smem)) return RAS_EINVAL;
    // offsets staged per round: 25 (one plane of offsets) when it fits, else fewer
    for (c->rap125_ng = 25;; c->rap125_ng = c->rap125_ng > 5 ? 5 : 1) {
        c->rap125_smem = sizeof(AT) * (size_t)(c->rap125_ng * WX * WY * WZ + 75 * WM + 5 * WY * WX +
                                               25 * WX + 128) + 32 * sizeof(int) + tables;
        if (c->rap125_smem <= (size_t)big || c->rap125_ng == 1) break;
    }
    c->fac_smem = std::max(sizeof(TileSmem<AT>), sizeof(AT) * (size_t)FROWS * c->T);
    c->fac_smem = std::max(c->fac_smem, edge_rows_smem(c->T, sizeof(AT)));
    // FP32: trailing updates of the inverses on the tensor cores (RAS_COARSE_TC=0: CUDA cores)
    c->use_tc = sizeof(AT) == 4 ? 1 : 0;
    if (const char *e = getenv("RAS_COARSE_TC")) c->use_tc = c->use_tc && atoi(e) != 0;
    if (c->use_tc) c->fac_smem = std::max(c->fac_smem, sizeof(TcSmem));
    // RAS_COARSE_CR=1 at set-up (FP32 with the tensor path, at least three
    // blocks): cyclic reduction instead of the two-ended elimination. Not the
    // default: on the 1M-cell workload it takes 9.8 ms per factorisation against
    // 5.3 ms and its solve reads half as many bytes again (the dense products of
    // its rounds outweigh the shorter chain of inversions).
    c->cr = 0;
    if (const char *e = getenv("RAS_COARSE_CR"))
        c->cr = sizeof(AT) == 4 && c->use_tc && c->nb >= 3 && atoi(e) != 0 ? 1 : 0;
    // the solve prefetches up to two (FP32) or one (FP64) matrix rows per warp
    // (the reduction's sweeps read theirs directly)
    c->sol_npf = c->cr ? 0 : (sizeof(AT) == 4 ? 2 : 1);
    while (c->sol_npf > 0 && sizeof(AT) * (size_t)(2 + 8 * c->sol_npf) * c->T > (size_t)big) --c->sol_npf;
    c->sol_smem = sizeof(AT) * (size_t)(2 + 8 * c->sol_npf) * c->T;
    if (c->rap_smem > (size_t)big || (c->need125 && c->rap125_smem > (size_t)big) || c->fac_smem > (size_t)big ||
        c->sol_smem > (size_t)big)
        return RAS_EINVAL;
    int dev = 0, sms = 0, bf = 0, bs = 0;
    RAS_CK(cudaGetDevice(&dev));
    RAS_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    RAS_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bf, k_coarse_factor<AT>, 256, c->fac_smem));
    RAS_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, k_coarse_solve<AT>, 256, c->sol_smem));
    if (bf < 1 || bs < 1) return RAS_EINVAL;
    c->fac_grid = sms * std::min(bf, 2);
    c->sol_grid = sms * std::min(bs, 2);
    // tuning knobs: fewer CTAs make the grid barrier cheaper (clamped to the
    // co-resident maximum, which the cooperative launch requires)
    if (const char *e = getenv("RAS_COARSE_FACTOR_CTAS")) {
        const int v = atoi(e);
        if (v >= 1) c->fac_grid = std::min(v, sms * bf);
    }
    if (const char *e = getenv("RAS_COARSE_SOLVE_CTAS")) {
        const int v = atoi(e);
        if (v >= 1) c->sol_grid = std::min(v, sms * bs);
    }
    return RAS_OK;
}

// interpolation tables of one axis on the device
static int upload_axis(int n, int r, int order, int *&d_ia, int *&d_ib, double *&d_wa, double *&d_wb, int *&d_lo,
                       int *&d_hi, double *&d_wt, int &nc, int &wmax) {
    std::vector<int> ia, ib, lo, hi;
    std::vector<double> wa, wb;
    interp_axis(n, r, ia, ib, wa, wb, lo, hi, nc, order);
    wmax = 1;
    for (size_t I = 0; I < lo.size(); ++I) wmax = std::max(wmax, hi[I] - lo[I]);
    // wt[I][m] = P(lo[I] + m, I) by w1's selection (zero past hi[I])
    std::vector<double> wt((size_t)nc * wmax, 0.0);
    for (int I = 0; I < nc; ++I)
        for (int a = lo[I]; a < hi[I]; ++a)
            wt[(size_t)I * wmax + (a - lo[I])] = ia[a] == I ? wa[a] : (ib[a] == I ? wb[a] : 0.0);
    RAS_TRY(dalloc(&d_wt, wt.size()));
    RAS_CK(cudaMemcpy(d_wt, wt.data(), wt.size() * 8, cudaMemcpyHostToDevice));
    RAS_TRY(dalloc(&d_ia, ia.size()));
    RAS_TRY(dalloc(&d_ib, ib.size()));
    RAS_TRY(dalloc(&d_wa, wa.size()));
    RAS_TRY(dalloc(&d_wb, wb.size()));
    RAS_TRY(dalloc(&d_lo, lo.size()));
    RAS_TRY(dalloc(&d_hi, hi.size()));
    RAS_CK(cudaMemcpy(d_ia, ia.data(), ia.size() * 4, cudaMemcpyHostToDevice));
    RAS_CK(cudaMemcpy(d_ib, ib.data(), ib.size() * 4, cudaMemcpyHostToDevice));
    RAS_CK(cudaMemcpy(d_wa, wa.data(), wa.size() * 8, cudaMemcpyHostToDevice));
    RAS_CK(cudaMemcpy(d_wb, wb.data(), wb.size() * 8, cudaMemcpyHostToDevice));
    RAS_CK(cudaMemcpy(d_lo, lo.data(), lo.size() * 4, cudaMemcpyHostToDevice));
    RAS_CK(cudaMemcpy(d_hi, hi.data(), hi.size() * 4, cudaMemcpyHostToDevice));
    return RAS_OK;
}

int coarse_setup(Coarse **out, const ras_problem *Pb, const ras_opts &o) {
    return coarse_setup_grid(out, Pb->nx, Pb->ny, Pb->nz, o);
}

int coarse_setup_grid(Coarse **out, int fnx, int fny, int fnz, const ras_opts &o) {
    *out = nullptr;
    if (o.interp_order != 1 && o.interp_order != 2) return RAS_EINVAL;
    if (o.coarse_prec != 64 && o.coarse_prec != 32) return RAS_EINVAL;
    for (int a = 0; a < 3; ++a) if (o.coarsen[a] < 1) return RAS_EINVAL;
    int dev = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop)
        return RAS_EINVAL;
    Coarse *c = new Coarse();
    auto fail = [&](int s) { coarse_free(c); return s; };
    c->prec = o.coarse_prec;
    c->esz = c->prec == 64 ? 8 : 4;
    if (fnx < 1 || fny < 1 || fnz < 1) return fail(RAS_EINVAL);
    c->nx = fnx; c->ny = fny; c->nz = fnz; c->N = fnx * fny * fnz;
    c->n[0] = fnx; c->n[1] = fny; c->n[2] = fnz;
    for (int a = 0; a < 3; ++a) {
        c->r[a] = o.coarsen[a];
        const int rc = upload_axis(c->n[a], c->r[a], o.interp_order, c->d_ia[a], c->d_ib[a], c->d_wa[a], c->d_wb[a],
                                   c->d_lo[a], c->d_hi[a], c->d_wt[a], c->c[a], c->wmax[a]);
        if (rc) return fail(rc);
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
    c->mid = c->nb == 1 ? 0 : (c->nb + 1) / 2;   // the two chains differ in length
    if ((long long)c->T * c->T * c->nb * c->esz > (8LL << 30)) return fail(RAS_EINVAL);
    c->need125 = o.nlevels == 3 ? 1 : 0;
    int rc = c->prec == 64 ? configure_t<double>(c) : configure_t<float>(c);
    if (rc) return fail(rc);
    CrPlan plan;
    if (c->cr) {
        c->mid = c->nb - 1;              // every edge oriented pivot e -> target e + 1
        cr_plan(c->nb, plan);
        c->cr_maxE = plan.maxE;
        c->cr_mats = plan.mats;
        if ((long long)c->T * c->T * (plan.nslot + c->nb) * c->esz > (16LL << 30)) return fail(RAS_EINVAL);
    }
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
    if ((rc = dalloc(&c->d_pos, pos.size())) || (rc = dalloc(&c->d_cell, cell.size())) ||
        (rc = dalloc(&c->d_err, 1)) || (rc = dalloc(&c->d_bar, 1)))
        return fail(rc);
    unsigned char *p_ac, *p_d, *p_c = nullptr, *p_f = nullptr, *p_lv, *p_uv, *p_g, *p_x;
    const size_t nbm1 = (size_t)std::max(c->nb - 1, 1);
    if (c->cr) {                         // the reduction's buffers instead of C and F
        unsigned char *p_w = nullptr;
        if ((rc = dalloc(&p_w, (size_t)plan.nslot * bsz * c->esz)) ||
            (rc = dalloc(&c->d_crf, plan.fac.size())) || (rc = dalloc(&c->d_crs, plan.sol.size())))
            return fail(rc);
        c->W = p_w;
        if (cudaMemcpy(c->d_crf, plan.fac.data(), plan.fac.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(c->d_crs, plan.sol.data(), plan.sol.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(RAS_ECUDA);
    } else if ((rc = dalloc(&p_c, nbm1 * bsz * c->esz)) || (rc = dalloc(&p_f, nbm1 * bsz * c->esz))) {
        return fail(rc);
    }
    if ((rc = dalloc(&p_ac, (size_t)125 * c->Nc * c->esz)) || (rc = dalloc(&p_d, c->nb * bsz * c->esz)) ||
        (rc = dalloc(&c->lo_q, nbm1 * c->T * ELLW)) || (rc = dalloc(&c->up_q, nbm1 * c->T * ELLW)) ||
        (rc = dalloc(&c->lo_n, nbm1 * c->T)) || (rc = dalloc(&c->up_n, nbm1 * c->T)) ||
        (rc = dalloc(&p_lv, nbm1 * c->T * ELLW * c->esz)) ||
        (rc = dalloc(&p_uv, nbm1 * c->T * ELLW * c->esz)) ||
        (rc = dalloc(&p_g, (size_t)c->nb * c->T * c->esz)) ||
        (rc = dalloc(&p_x, (size_t)c->nb * c->T * c->esz)))
        return fail(rc);
    {
        unsigned char *p_z = nullptr, *p_rx = nullptr, *p_ry = nullptr;
        const size_t nz = (size_t)std::max(2, c->cr_maxE);   // one scratch strip per concurrent inversion
        if ((rc = dalloc(&p_z, nz * TILE * c->T * c->esz))) return fail(rc);
        c->Zs = p_z;
        if ((rc = dalloc(&p_rx, (size_t)c->c[0] * c->n[1] * c->n[2] * c->esz))) return fail(rc);
        c->rx = p_rx;
        if ((rc = dalloc(&p_ry, (size_t)c->c[0] * c->c[1] * c->n[2] * c->esz))) return fail(rc);
        c->ry = p_ry;
        unsigned char *p_xn = nullptr;
        if ((rc = dalloc(&p_xn, (size_t)c->Nc * c->esz))) return fail(rc);
        c->xn = p_xn;
    }
    c->Ac = p_ac; c->D = p_d; c->C = p_c; c->F = p_f; c->lo_v = p_lv; c->up_v = p_uv;
    c->g = p_g; c->x = p_x;
    if (cudaMemcpy(c->d_pos, pos.data(), pos.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_cell, cell.data(), cell.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(c->d_err, 0, 4) != cudaSuccess ||
        cudaMemset(c->d_bar, 0, sizeof(GridBar)) != cudaSuccess ||
        cudaMemset(c->g, 0, (size_t)c->nb * c->T * c->esz) != cudaSuccess ||
        cudaMemset(c->x, 0, (size_t)c->nb * c->T * c->esz) != cudaSuccess ||
        cudaMemset(c->lo_q, 0, nbm1 * c->T * ELLW * sizeof(int)) != cudaSuccess ||
        cudaMemset(c->up_q, 0, nbm1 * c->T * ELLW * sizeof(int)) != cudaSuccess ||
        cudaMemset(c->lo_n, 0, nbm1 * c->T * sizeof(int)) != cudaSuccess ||
        cudaMemset(c->up_n, 0, nbm1 * c->T * sizeof(int)) != cudaSuccess)
        return fail(RAS_ECUDA);
    *out = c;
    return RAS_OK;
}

void coarse_free(Coarse *c) {
    if (!c) return;
    for (int a = 0; a < 3; ++a) {
        dfree(c->d_ia[a]); dfree(c->d_ib[a]); dfree(c->d_wa[a]); dfree(c->d_wb[a]);
        dfree(c->d_lo[a]); dfree(c->d_hi[a]); dfree(c->d_wt[a]);
    }
    dfree(c->d_pos); dfree(c->d_cell); dfree(c->d_err); dfree(c->d_bar);
    dfree(c->lo_q); dfree(c->up_q); dfree(c->lo_n); dfree(c->up_n); dfree(c->d_crf); dfree(c->d_crs);
    for (void *p : {c->Ac, c->D, c->C, c->F, c->lo_v, c->up_v, c->g, c->x, c->Zs, c->rx, c->ry, c->W, c->xn})
        if (p) cudaFree(p);
    delete c;
}

// dense block factorisation of the Galerkin operator already in c->Ac
template <typename AT>
static int assemble_blocks_t(Coarse *c, cudaStream_t st) {
    const CGeom G = geom_of(c);
    AT *Ac = (AT *)c->Ac, *D = (AT *)c->D;
    const size_t bsz = (size_t)c->T * c->T;
    RAS_CK(cudaMemsetAsync(D, 0, c->nb * bsz * sizeof(AT), st));
    k_assemble<AT><<<grid_of((long long)c->nb * c->T), 256, 0, st>>>(Ac, c->d_pos, c->d_cell, G, D);
    RAS_LAUNCHED();
    if (c->nb > 1) {
        k_ell<AT><<<grid_of((long long)(c->nb - 1) * c->T), 256, 0, st>>>(
            Ac, c->d_pos, c->d_cell, G, c->lo_q, (AT *)c->lo_v, c->up_q, (AT *)c->up_v, c->lo_n,
            c->up_n, c->d_err);
        RAS_LAUNCHED();
    }
    if (c->cr) {   // the first round's couplings, dense (slots nb + k and 2 nb + k)
        AT *Lc = (AT *)c->W, *Uc = Lc + c->nb * bsz;
        RAS_CK(cudaMemsetAsync(Lc, 0, 2 * c->nb * bsz * sizeof(AT), st));
        k_cr_couplings<AT><<<grid_of((long long)(c->nb - 1) * c->T), 256, 0, st>>>(
            c->lo_q, (const AT *)c->lo_v, c->lo_n, c->up_q, (const AT *)c->up_v, c->up_n, c->T, c->nb, Lc, Uc);
        RAS_LAUNCHED();
    }
    return RAS_OK;
}

template <typename AT>
static FacArgs<AT> fac_args(Coarse *c, GridBar *bar) {
    return FacArgs<AT>{(AT *)c->D, (AT *)c->C, (AT *)c->F, (AT *)c->Zs, c->lo_q, c->up_q, c->lo_n, c->up_n,
                       (const AT *)c->lo_v, (const AT *)c->up_v, c->T, c->T / TILE, c->nb, c->mid, bar, c->d_err,
                       c->cr, c->d_crf, (AT *)c->W, c->use_tc};
}

template <typename AT>
static SolArgs<AT> sol_args(Coarse *c, GridBar *bar, const double *t, double *z, int accumulate) {
    return SolArgs<AT>{t, z, accumulate, interp_of(c), geom_of(c), c->d_pos, (const AT *)c->D,
                       (const AT *)c->C, (const AT *)c->F, (AT *)c->g, (AT *)c->x, (AT *)c->rx,
                       (AT *)c->ry, bar, c->d_err, c->sol_npf, c->cr, c->d_crs, (const AT *)c->W,
                       (AT *)c->xn, c->d_cell, 1};
}

template <typename AT>
static int eliminate_t(Coarse *c, cudaStream_t st);

template <typename AT>
static int factor_blocks_t(Coarse *c, cudaStream_t st) {
    RAS_TRY(assemble_blocks_t<AT>(c, st));
    return eliminate_t<AT>(c, st);
}

// the block elimination of the assembled blocks (one cooperative launch)
template <typename AT>
static int eliminate_t(Coarse *c, cudaStream_t st) {
    RAS_TRY(reset_bar(c, st));
    FacArgs<AT> fa = fac_args<AT>(c, c->d_bar);
    int use_tc = c->use_tc;
    void *args[] = {&fa, &use_tc};
    RAS_CK(cudaLaunchCooperativeKernel((const void *)k_coarse_factor<AT>, dim3(c->fac_grid),
                                       dim3(256), args, c->fac_smem, st));
    RAS_LAUNCHED();
    return RAS_OK;
}

// the Galerkin product of the 7-point operator in the form of the handle's plan
template <typename AT>
static void rap_launch(const Coarse *c, int zs, size_t smem, const Stencil7 &A, AT *Ac, cudaStream_t st) {
    RapDims W{c->wmax[0], c->wmax[1], c->wmax[2]};
    if (zs == 0) k_rap<AT><<<c->Nc, 256, smem, st>>>(A, interp_of(c), geom_of(c), W, Ac);
    else k_rap_slab<AT><<<c->Nc, 256, smem, st>>>(A, interp_of(c), geom_of(c), W, zs, Ac);
}

template <typename AT>
static int factor_t(Coarse *c, const Stencil7 &A, cudaStream_t st) {
    rap_launch<AT>(c, c->rap_zs, c->rap_smem, A, (AT *)c->Ac, st);
    RAS_LAUNCHED();
    return factor_blocks_t<AT>(c, st);
}

template <typename AT>
static int factor125_t(Coarse *c, const double *Af, cudaStream_t st) {
    RapDims W{c->wmax[0], c->wmax[1], c->wmax[2]};
    k_rap125<AT><<<c->Nc, 256, c->rap125_smem, st>>>(Af, interp_of(c), geom_of(c), W, c->rap125_ng,
                                                      (AT *)c->Ac);
    RAS_LAUNCHED();
    return factor_blocks_t<AT>(c, st);
}

int coarse_factor(Coarse *c, const Stencil7 &A, cudaStream_t st) {
    return c->prec == 64 ? factor_t<double>(c, A, st) : factor_t<float>(c, A, st);
}

template <typename AT>
static int prepare_t(Coarse *c, const Stencil7 &A, cudaStream_t st) {
    rap_launch<AT>(c, c->rap_zs, c->rap_smem, A, (AT *)c->Ac, st);
    RAS_LAUNCHED();
    return assemble_blocks_t<AT>(c, st);
}

int coarse_factor_blocks(Coarse *c, cudaStream_t st) {
    return c->prec == 64 ? eliminate_t<double>(c, st) : eliminate_t<float>(c, st);
}

int coarse_factor_prepare(Coarse *c, const Stencil7 &A, cudaStream_t st) {
    return c->prec == 64 ? prepare_t<double>(c, A, st) : prepare_t<float>(c, A, st);
}

int coarse_factor125(Coarse *c, const double *Af, cudaStream_t st) {
    return c->prec == 64 ? factor125_t<double>(c, Af, st) : factor125_t<float>(c, Af, st);
}

int coarse_check(Coarse *c, cudaStream_t st) {
    int h = 0;
    RAS_CK(cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    RAS_CK(cudaStreamSynchronize(st));
    if (h) {
        RAS_CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), st));
        return h == ERR_TIMEOUT ? RAS_ETIMEOUT : (h == ERR_ELL ? RAS_EINVAL : RAS_EZEROPIVOT);
    }
    return RAS_OK;
}

template <typename AT>
static int correct_t(Coarse *c, const double *t, double *z, int accumulate, cudaStream_t st) {
    RAS_TRY(reset_bar(c, st));
    SolArgs<AT> sa = sol_args<AT>(c, c->d_bar, t, z, accumulate);
    sa.prolong = 0;
    void *args[] = {&sa};
    RAS_CK(cudaLaunchCooperativeKernel((const void *)k_coarse_solve<AT>, dim3(c->sol_grid),
                                       dim3(256), args, c->sol_smem, st));
    RAS_LAUNCHED();
    k_coarse_prolong<AT><<<grid_of((long long)c->N), 256, 0, st>>>(sa);
    RAS_LAUNCHED();
    return RAS_OK;
}

// ---------------------------------------------------------------------------
// coarse corrections of many handles in one cooperative launch
// ---------------------------------------------------------------------------

struct CoarseBatch {
    int n = 0, prec = 32, grid = 0, fgrid = 0;
    size_t smem = 0, fsmem = 0;
    void *d_args = nullptr;                 // SolArgs<AT>[n]
    int *d_cta_inst = nullptr, *d_first = nullptr, *d_size = nullptr;
    void *d_fargs = nullptr;                // FacArgs<AT>[n]
    int *d_fcta_inst = nullptr, *d_ffirst = nullptr, *d_fsize = nullptr;
    std::vector<int> fwave0, fwaven;        // factorisation waves: CTA range in d_fcta_inst
    GridBar *d_bars = nullptr;              // [n], one barrier word per handle
};

void coarse_batch_free(CoarseBatch *cb) {
    if (!cb) return;
    if (cb->d_args) cudaFree(cb->d_args);
    if (cb->d_fargs) cudaFree(cb->d_fargs);
    dfree(cb->d_cta_inst); dfree(cb->d_first); dfree(cb->d_size); dfree(cb->d_bars);
    dfree(cb->d_fcta_inst); dfree(cb->d_ffirst); dfree(cb->d_fsize);
    delete cb;
}

// CTA groups of a batched cooperative launch: `total` CTAs split over n handles in
// proportion to w (at least one each); cta[k] = handle of CTA k.
static int partition(const std::vector<double> &w, int total, std::vector<int> &cta, std::vector<int> &first,
                     std::vector<int> &size) {
    const int n = (int)w.size();
    if (n > total) return RAS_EINVAL;
    double wsum = 0.0;
    for (double v : w) wsum += v;
    size.assign(n, 1);
    first.assign(n, 0);
    int used = 0;
    for (int i = 0; i < n; ++i) {
        size[i] = std::max(1, (int)((total - n) * (wsum > 0 ? w[i] / wsum : 0.0)) + 1);
        used += size[i];
    }
    while (used > total) {                  // rounding: take from the largest groups
        const int j = (int)(std::max_element(size.begin(), size.end()) - size.begin());
        --size[j];
        --used;
    }
    cta.clear();
    for (int i = 0; i < n; ++i) {
        first[i] = (int)cta.size();
        for (int q = 0; q < size[i]; ++q) cta.push_back(i);
    }
    return RAS_OK;
}

template <typename AT>
static int batch_setup_t(Coarse *const *cs, int n, CoarseBatch *cb) {
    int dev = 0, sms = 0, bs = 0, bf = 0;
    size_t smem = 0, fsmem = 0;
    for (int i = 0; i < n; ++i) {
        smem = std::max(smem, cs[i]->sol_smem);
        fsmem = std::max(fsmem, cs[i]->fac_smem);
    }
    RAS_CK(cudaGetDevice(&dev));
    RAS_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    RAS_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, k_coarse_solve_batch<AT>, 256, smem));
    RAS_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bf, k_coarse_factor_batch<AT>, 256, fsmem));
    if (bs < 1 || bf < 1) return RAS_EINVAL;
    // solve: CTAs in proportion to the fine cells (the restriction and prolongation
    // scale with them, the block sweeps' latency-bound rows with the coarse cells);
    // factorisation: in proportion to the block elimination's work T^3 nb
    std::vector<double> ws(n), wf(n);
    for (int i = 0; i < n; ++i) {
        ws[i] = (double)cs[i]->N;
        wf[i] = (double)cs[i]->T * cs[i]->T * cs[i]->T * cs[i]->nb;
    }
    std::vector<int> cta, first, size, fcta, ffirst(n, 0), fsize(n, 1);
    RAS_TRY(partition(ws, sms * std::min(bs, 2), cta, first, size));
    // The block elimination is a chain of latency-bound panel steps whose trailing
    // work needs CTAs: handles are factored in waves (largest first) of at most
    // total / FWAVE_CTAS handles, so every handle gets at least FWAVE_CTAS CTAs.
    // On 64 reservoirs of 32^3 to 96^3 cells 16 is the best of 1 to 48: fewer
    // leave each handle's trailing updates too few CTAs, more make more waves,
    // each paying its handles' pivot chains.
    const int ftotal = sms * std::min(bf, 2);
    int wave_ctas = FWAVE_CTAS;
    if (const char *e = getenv("RAS_COARSE_WAVE_CTAS")) {   // tuning knob
        const int v = atoi(e);
        if (v >= 1) wave_ctas = v;
    }
    const int per = std::max(1, ftotal / wave_ctas);
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return wf[x] > wf[y]; });
    for (int w0 = 0; w0 < n; w0 += per) {
        const int m = std::min(per, n - w0);
        std::vector<double> ww(m);
        for (int q = 0; q < m; ++q) ww[q] = wf[order[w0 + q]];
        std::vector<int> wc, wfirst, wsize;
        RAS_TRY(partition(ww, ftotal, wc, wfirst, wsize));
        cb->fwave0.push_back((int)fcta.size());
        cb->fwaven.push_back((int)wc.size());
        for (int q = 0; q < m; ++q) {
            ffirst[order[w0 + q]] = wfirst[q];
            fsize[order[w0 + q]] = wsize[q];
        }
        for (int k : wc) fcta.push_back(order[w0 + k]);
    }
    std::vector<SolArgs<AT>> args(n);
    std::vector<FacArgs<AT>> fargs(n);
    RAS_TRY(dalloc(&cb->d_bars, n));
    for (int i = 0; i < n; ++i) {
        Coarse *c = cs[i];
        args[i] = sol_args<AT>(c, cb->d_bars + i, nullptr, nullptr, 1);
        fargs[i] = fac_args<AT>(c, cb->d_bars + i);
    }
    RAS_CK(cudaMalloc(&cb->d_args, n * sizeof(SolArgs<AT>)));
    RAS_CK(cudaMalloc(&cb->d_fargs, n * sizeof(FacArgs<AT>)));
    RAS_TRY(dalloc(&cb->d_cta_inst, cta.size()));
    RAS_TRY(dalloc(&cb->d_first, n));
    RAS_TRY(dalloc(&cb->d_size, n));
    RAS_TRY(dalloc(&cb->d_fcta_inst, fcta.size()));
    RAS_TRY(dalloc(&cb->d_ffirst, n));
    RAS_TRY(dalloc(&cb->d_fsize, n));
    RAS_CK(cudaMemcpy(cb->d_args, args.data(), n * sizeof(SolArgs<AT>), cudaMemcpyHostToDevice));
    RAS_CK(cudaMemcpy(cb->d_fargs, fargs.data(), n * sizeof(FacArgs<AT>), cudaMemcpyHostToDevice));
    RAS_CK(cudaMemcpy(cb->d_cta_inst, cta.data(), cta.size() * sizeof(int), cudaMemcpyHostToDevice));
    RAS_CK(cudaMemcpy(cb->d_first, first.data(), n * sizeof(int), cudaMemcpyHostToDevice));
    RAS_CK(cudaMemcpy(cb->d_size, size.data(), n * sizeof(int), cudaMemcpyHostToDevice));
    RAS_CK(cudaMemcpy(cb->d_fcta_inst, fcta.data(), fcta.size() * sizeof(int), cudaMemcpyHostToDevice));
    RAS_CK(cudaMemcpy(cb->d_ffirst, ffirst.data(), n * sizeof(int), cudaMemcpyHostToDevice));
    RAS_CK(cudaMemcpy(cb->d_fsize, fsize.data(), n * sizeof(int), cudaMemcpyHostToDevice));
    RAS_CK(cudaMemset(cb->d_bars, 0, n * sizeof(GridBar)));
    cb->grid = (int)cta.size();
    cb->smem = smem;
    cb->fgrid = (int)fcta.size();   // all waves
    cb->fsmem = fsmem;
    return RAS_OK;
}

int coarse_batch_setup(Coarse *const *cs, int n, CoarseBatch **out) {
    *out = nullptr;
    if (n < 1) return RAS_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!cs[i] || cs[i]->prec != cs[0]->prec) return RAS_EINVAL;
    CoarseBatch *cb = new CoarseBatch();
    cb->n = n;
    cb->prec = cs[0]->prec;
    const int rc = cb->prec == 64 ? batch_setup_t<double>(cs, n, cb) : batch_setup_t<float>(cs, n, cb);
    if (rc) { coarse_batch_free(cb); return rc; }
    *out = cb;
    return RAS_OK;
}

int coarse_factor_batch(CoarseBatch *cb, const unsigned char *d_active, cudaStream_t st) {
    k_reset_bars<<<(cb->n + 127) / 128, 128, 0, st>>>(cb->d_bars, cb->n, barrier_polls());
    RAS_LAUNCHED();
    for (size_t w = 0; w < cb->fwave0.size(); ++w) {
        const int *cta = cb->d_fcta_inst + cb->fwave0[w];
        const dim3 grid(cb->fwaven[w]);
        if (cb->prec == 64) {
            const FacArgs<double> *a = (const FacArgs<double> *)cb->d_fargs;
            void *args[] = {&a, &cta, &cb->d_ffirst, &cb->d_fsize, &d_active};
            RAS_CK(cudaLaunchCooperativeKernel((const void *)k_coarse_factor_batch<double>, grid, dim3(256), args,
                                               cb->fsmem, st));
        } else {
            const FacArgs<float> *a = (const FacArgs<float> *)cb->d_fargs;
            void *args[] = {&a, &cta, &cb->d_ffirst, &cb->d_fsize, &d_active};
            RAS_CK(cudaLaunchCooperativeKernel((const void *)k_coarse_factor_batch<float>, grid, dim3(256), args,
                                               cb->fsmem, st));
        }
        RAS_LAUNCHED();
    }
    return RAS_OK;
}

int coarse_correct_batch(CoarseBatch *cb, const long long *d_off, const unsigned char *d_active, const double *t,
                         double *z, cudaStream_t st) {
    k_reset_bars<<<(cb->n + 127) / 128, 128, 0, st>>>(cb->d_bars, cb->n, barrier_polls());
    RAS_LAUNCHED();
    if (cb->prec == 64) {
        const SolArgs<double> *a = (const SolArgs<double> *)cb->d_args;
        void *args[] = {&a, &cb->d_cta_inst, &cb->d_first, &cb->d_size, &d_off, &d_active, &t, &z};
        RAS_CK(cudaLaunchCooperativeKernel((const void *)k_coarse_solve_batch<double>, dim3(cb->grid), dim3(256),
                                           args, cb->smem, st));
    } else {
        const SolArgs<float> *a = (const SolArgs<float> *)cb->d_args;
        void *args[] = {&a, &cb->d_cta_inst, &cb->d_first, &cb->d_size, &d_off, &d_active, &t, &z};
        RAS_CK(cudaLaunchCooperativeKernel((const void *)k_coarse_solve_batch<float>, dim3(cb->grid), dim3(256),
                                           args, cb->smem, st));
    }
    RAS_LAUNCHED();
    return RAS_OK;
}

int coarse_correct(Coarse *c, const double *t, double *z, int accumulate, cudaStream_t st) {
    return c->prec == 64 ? correct_t<double>(c, t, z, accumulate, st)
                         : correct_t<float>(c, t, z, accumulate, st);
}

double coarse_bytes(const Coarse *c) {
    // E, C, F read once per solve; the reduction's matrices as its schedule reads them
    if (c->cr) return (double)c->esz * c->T * c->T * c->cr_mats;
    return (double)c->esz * c->T * c->T * (c->nb + 2.0 * (c->nb - 1));
}


// ---------------------------------------------------------------------------
// transfer between a level and the next coarser one (Algorithm 1): the
// Galerkin operator of a 7-point operator, restriction R = P^T, prolongation
// ---------------------------------------------------------------------------

struct Transfer {
    Coarse geo;        // interpolation tables and grid sizes only (no factors)
    int zs32 = 0;      // the FP32 Galerkin kernel's form and shared memory (geo holds FP64's)
    size_t smem32 = 0;
};

// tc[I] = sum_a P(a, I) t[a] over the fine support box of I (FP64)
__global__ void __launch_bounds__(256) k_restrict(Interp P, CGeom G, const double *__restrict__ t,
                                                  double *__restrict__ tc) {
    const long long nxy = (long long)G.nx * G.ny;
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < G.Nc; I += gridDim.x * blockDim.x) {
        const int Ix = I % G.cx, Iy = (I / G.cx) % G.cy, Iz = I / (G.cx * G.cy);
        double acc = 0.0;
        for (int az = P.lo[2][Iz]; az < P.hi[2][Iz]; ++az) {
            const double wz = w1(P, 2, az, Iz);
            for (int ay = P.lo[1][Iy]; ay < P.hi[1][Iy]; ++ay) {
                const double wyz = wz * w1(P, 1, ay, Iy);
                const double *row = t + G.nx * (long long)ay + nxy * az;
                for (int ax = P.lo[0][Ix]; ax < P.hi[0][Ix]; ++ax)
                    acc += wyz * w1(P, 0, ax, Ix) * __ldg(row + ax);
            }
        }
        tc[I] = acc;
    }
}

// x[a] += sum_I P(a, I) xc[I] (eight coarse cells per fine cell, FP64)
__global__ void __launch_bounds__(256) k_prolong(Interp P, CGeom G, const double *__restrict__ xc,
                                                 double *__restrict__ x) {
    const long long N = (long long)G.nx * G.ny * G.nz;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x) {
        const int ax = (int)(p % G.nx), ay = (int)((p / G.nx) % G.ny),
                  az = (int)(p / ((long long)G.nx * G.ny));
        const int Ix[2] = {P.ia[0][ax], P.ib[0][ax]};
        const int Iy[2] = {P.ia[1][ay], P.ib[1][ay]};
        const int Iz[2] = {P.ia[2][az], P.ib[2][az]};
        const double Wx[2] = {P.wa[0][ax], P.wb[0][ax]};
        const double Wy[2] = {P.wa[1][ay], P.wb[1][ay]};
        const double Wz[2] = {P.wa[2][az], P.wb[2][az]};
        double s = 0.0;
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int v = 0; v < 2; ++v)
#pragma unroll
                for (int w = 0; w < 2; ++w) {
                    const double wt = Wx[w] * Wy[v] * Wz[u];
                    if (wt != 0.0) s += wt * __ldg(xc + Ix[w] + G.cx * (Iy[v] + G.cy * Iz[u]));
                }
        x[p] += s;
    }
}

int transfer_setup(Transfer **out, int nx, int ny, int nz, const int ratio[3], int order) {
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return RAS_EINVAL;
    for (int a = 0; a < 3; ++a) if (ratio[a] < 1) return RAS_EINVAL;
    Transfer *t = new Transfer();
    Coarse *c = &t->geo;
    c->nx = nx; c->ny = ny; c->nz = nz; c->N = nx * ny * nz;
    c->n[0] = nx; c->n[1] = ny; c->n[2] = nz;
    for (int a = 0; a < 3; ++a) {
        c->r[a] = ratio[a];
        const int rc = upload_axis(c->n[a], c->r[a], order, c->d_ia[a], c->d_ib[a], c->d_wa[a], c->d_wb[a],
                                   c->d_lo[a], c->d_hi[a], c->d_wt[a], c->c[a], c->wmax[a]);
        if (rc) { transfer_free(t); return rc; }
    }
    c->Nc = c->c[0] * c->c[1] * c->c[2];
    if (rap_plan(c->wmax, sizeof(double), 200 * 1024, c->rap_zs, c->rap_smem) ||
        rap_plan(c->wmax, sizeof(float), 200 * 1024, t->zs32, t->smem32)) {
        transfer_free(t);
        return RAS_EINVAL;
    }
    if (cudaFuncSetAttribute(k_rap<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_rap<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_rap_slab<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_rap_slab<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
            cudaSuccess) {
        transfer_free(t);
        return RAS_ECUDA;
    }
    *out = t;
    return RAS_OK;
}

void transfer_free(Transfer *t) {
    if (!t) return;
    Coarse *c = &t->geo;
    for (int a = 0; a < 3; ++a) {
        dfree(c->d_ia[a]); dfree(c->d_ib[a]); dfree(c->d_wa[a]); dfree(c->d_wb[a]);
        dfree(c->d_lo[a]); dfree(c->d_hi[a]); dfree(c->d_wt[a]);
    }
    delete t;
}

void transfer_dims(const Transfer *t, int c[3]) {
    for (int a = 0; a < 3; ++a) c[a] = t->geo.c[a];
}

int transfer_galerkin7(Transfer *t, const Stencil7 &A, double *Ac, float *scratch, cudaStream_t st) {
    const Coarse *c = &t->geo;
    if (!scratch) {
        rap_launch<double>(c, c->rap_zs, c->rap_smem, A, Ac, st);
        RAS_LAUNCHED();
        return RAS_OK;
    }
    rap_launch<float>(c, t->zs32, t->smem32, A, scratch, st);
    RAS_LAUNCHED();
    k_widen<<<grid_of(125LL * c->Nc), 256, 0, st>>>(scratch, Ac, 125LL * c->Nc);
    RAS_LAUNCHED();
    return RAS_OK;
}

int transfer_restrict(Transfer *t, const double *x, double *xc, cudaStream_t st) {
    const Coarse *c = &t->geo;
    k_restrict<<<grid_of(c->Nc), 256, 0, st>>>(interp_of(c), geom_of(c), x, xc);
    RAS_LAUNCHED();
    return RAS_OK;
}

int transfer_prolong(Transfer *t, const double *xc, double *x, cudaStream_t st) {
    const Coarse *c = &t->geo;
    k_prolong<<<grid_of(c->N), 256, 0, st>>>(interp_of(c), geom_of(c), xc, x);
    RAS_LAUNCHED();
    return RAS_OK;
}

}  // namespace ras

// The cyclic-reduction schedule for nb blocks, copied out for inspection (host
// only: the plan is the one coarse set-up builds).
extern "C" int ras_coarse_cr_schedule(int nb, int *fac, int fac_cap, int *sol, int sol_cap, int *fac_len,
                                      int *sol_len, int *nslot) {
    if (nb < 1 || nb > 0xffff || !fac_len || !sol_len || !nslot) return RAS_EINVAL;
    ras::CrPlan P;
    ras::cr_plan(nb, P);
    *fac_len = (int)P.fac.size();
    *sol_len = (int)P.sol.size();
    *nslot = P.nslot;
    if (!fac || !sol || fac_cap < *fac_len || sol_cap < *sol_len) return RAS_EINVAL;
    std::copy(P.fac.begin(), P.fac.end(), fac);
    std::copy(P.sol.begin(), P.sol.end(), sol);
    return RAS_OK;
}
