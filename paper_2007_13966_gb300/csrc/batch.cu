// Many independent reservoirs advanced together on one GPU: a batched inexact
// Newton step (Section 2) whose FGMRES iterations run each operation for every
// reservoir in one launch -- the left-RAS subdomain solves of all reservoirs'
// boxes (Eq. equ:as-left; a persistent kernel over a largest-first work queue),
// their 7-point operators, the Arnoldi dot products and updates. Each reservoir's
// Arnoldi scalars (Hessenberg column, Givens rotations, residual estimate, stop
// test) are updated on the device, so a restart cycle replays as CUDA graphs of a
// few Arnoldi steps with the host reading the mask only between them; the cubic
// backtracking stays on the host. With two-level V-cycle preconditioners
// (Eq. equ:v-cycle) the fine-level solves and residuals are batched the same way,
// the exact coarse corrections of all reservoirs run in one cooperative launch (a
// group of CTAs and a barrier word per reservoir), and their coarse block
// eliminations in a few such launches (waves of reservoirs).
//
// Vectors of the batch are the reservoirs' vectors concatenated (each starting
// at a multiple of 32 cells). The vector kernels run on chunks of BCH cells of
// one reservoir each, so every reduction is a fixed per-chunk partial followed
// by a fixed-order sum over that reservoir's chunks (deterministic). A reservoir
// whose solve has finished is switched off in a device mask; its chunks and
// boxes return at once.
#include "precond.cuh"

#include <algorithm>
#include <cstring>

namespace ras {

constexpr int BCH = 2048;               // cells per CTA of the batched vector kernels
constexpr int OST = 2 * MAX_MDOT + 8;   // device results per reservoir
constexpr int CYC_CHUNK = 2;            // Arnoldi steps per replayed graph (mask read between chunks)
constexpr int NPOOL = 8;                // streams for independent per-reservoir launches

struct BOp {                    // one reservoir's 7-point operator
    const double *c[7];
    int nx, ny, nz;
    unsigned long long mx, my;  // ceil(2^64 / nx), ceil(2^64 / ny) (0 for 1)
};

struct BChunk {
    int inst, start, count;
};

// q / d as a 64-bit multiply-high by ceil(2^64 / d): exact for 0 <= q < 2^32 and
// 1 <= d < 2^31 (q times the multiplier's excess over 2^64 / d stays below 2^64)
__device__ __forceinline__ int bdiv(int q, int d, unsigned long long m) {
    return d == 1 ? q : (int)__umul64hi((unsigned long long)q, m);
}
static unsigned long long bmagic(int d) { return d == 1 ? 0ull : (~0ull / (unsigned long long)d) + 1ull; }

// y = A x, or y = b - A x, per reservoir (the arithmetic of the single-reservoir
// operator)
template <bool RESID>
__global__ void __launch_bounds__(256) k_bstencil(const BOp *__restrict__ ops, const BChunk *__restrict__ ch,
                                                  const long long *__restrict__ off,
                                                  const unsigned char *__restrict__ active,
                                                  const double *__restrict__ b, const double *__restrict__ x,
                                                  double *__restrict__ y) {
    const BChunk c = ch[blockIdx.x];
    if (!active[c.inst]) return;
    const BOp A = ops[c.inst];
    const int nx = A.nx, ny = A.ny, nz = A.nz, nxy = nx * ny;
    const long long o = off[c.inst];
    const double *xi = x + o;
    double *yi = y + o;
    for (int q = threadIdx.x; q < c.count; q += blockDim.x) {
        const int n = c.start + q;
        const int row = bdiv(n, nx, A.mx), k = bdiv(row, ny, A.my);
        const int i = n - row * nx, j = row - k * ny;
        double s = A.c[0][n] * xi[n];
        if (i > 0) s = fma(A.c[1][n], xi[n - 1], s);
        if (i < nx - 1) s = fma(A.c[2][n], xi[n + 1], s);
        if (j > 0) s = fma(A.c[3][n], xi[n - nx], s);
        if (j < ny - 1) s = fma(A.c[4][n], xi[n + nx], s);
        if (k > 0) s = fma(A.c[5][n], xi[n - nxy], s);
        if (k < nz - 1) s = fma(A.c[6][n], xi[n + nxy], s);
        yi[n] = RESID ? b[o + n] - s : s;
    }
}

// block sum of `acc` -> partials[slot * nch + blockIdx.x] (RED_THREADS threads)
__device__ __forceinline__ void block_partial(double acc, double *sh, double *partials, long long at) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __syncthreads();
    if (lane == 0) sh[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < RED_THREADS / 32; ++q) s += sh[q];
        partials[at] = s;
    }
}

// partials[v][chunk] = sum over the chunk of V[v] w (v < k); row KM: w . w if self
template <int KM>
__global__ void __launch_bounds__(RED_THREADS) k_bmdot(const double *__restrict__ V, long long ldv, int k,
                                                       int self, const double *__restrict__ w,
                                                       const BChunk *__restrict__ ch,
                                                       const long long *__restrict__ off,
                                                       const unsigned char *__restrict__ active,
                                                       double *__restrict__ partials, int nch) {
    const BChunk c = ch[blockIdx.x];
    if (!active[c.inst]) return;
    const long long base = off[c.inst] + c.start;
    double acc[KM + 1];
#pragma unroll
    for (int v = 0; v <= KM; ++v) acc[v] = 0.0;
    for (int q = threadIdx.x; q < c.count; q += blockDim.x) {
        const double wi = w[base + q];
#pragma unroll
        for (int v = 0; v < KM; ++v)
            if (v < k) acc[v] = fma(V[v * ldv + base + q], wi, acc[v]);
        if (self) acc[KM] = fma(wi, wi, acc[KM]);
    }
    __shared__ double sh[RED_THREADS / 32];
    for (int v = 0; v < k; ++v) block_partial(acc[v], sh, partials, (long long)v * nch + blockIdx.x);
    if (self) block_partial(acc[KM], sh, partials, (long long)k * nch + blockIdx.x);
}

// out[inst][slot0 + v] = sum of the reservoir's chunk partials of row v, in chunk
// order (one warp per reservoir); the last row's square root if sqrt_last
__global__ void k_bfinalize(const double *__restrict__ partials, int nch, int nvec,
                            const int *__restrict__ ch0, const int *__restrict__ chn,
                            const unsigned char *__restrict__ active, double *__restrict__ out, int slot0,
                            int sqrt_last, int ninst) {
    const int inst = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (inst >= ninst || !active[inst]) return;
    const int lane = threadIdx.x & 31, a = ch0[inst], cnt = chn[inst];
    for (int v = 0; v < nvec; ++v) {
        double acc = 0.0;
        for (int q = lane; q < cnt; q += 32) acc += partials[(long long)v * nch + a + q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) out[(long long)inst * OST + slot0 + v] = (sqrt_last && v == nvec - 1) ? sqrt(acc) : acc;
    }
}

// w -= sum_v h[v] V[v] with the reservoir's coefficients h = out[inst][hslot ..];
// partial sums of the new w . w if NORM
template <bool NORM, int KM>
__global__ void __launch_bounds__(RED_THREADS) k_bupdate(const double *__restrict__ V, long long ldv, int k,
                                                         const double *__restrict__ out, int hslot,
                                                         double *__restrict__ w, const BChunk *__restrict__ ch,
                                                         const long long *__restrict__ off,
                                                         const unsigned char *__restrict__ active,
                                                         double *__restrict__ partials) {
    const BChunk c = ch[blockIdx.x];
    if (!active[c.inst]) return;
    const long long base = off[c.inst] + c.start;
    const double *h = out + (long long)c.inst * OST + hslot;
    double hv[KM];
#pragma unroll
    for (int v = 0; v < KM; ++v) hv[v] = v < k ? h[v] : 0.0;
    double acc = 0.0;
    for (int q = threadIdx.x; q < c.count; q += blockDim.x) {
        double s = w[base + q];
#pragma unroll
        for (int v = 0; v < KM; ++v)
            if (v < k) s = fma(-hv[v], V[v * ldv + base + q], s);
        w[base + q] = s;
        if (NORM) acc = fma(s, s, acc);
    }
    if (NORM) {
        __shared__ double sh[RED_THREADS / 32];
        block_partial(acc, sh, partials, blockIdx.x);
    }
}

// y = x / s[inst * stride] per reservoir
__global__ void __launch_bounds__(256) k_bscale(double *__restrict__ y, const double *__restrict__ x,
                                                const double *__restrict__ s, int stride,
                                                const BChunk *__restrict__ ch, const long long *__restrict__ off,
                                                const unsigned char *__restrict__ active) {
    const BChunk c = ch[blockIdx.x];
    if (!active[c.inst]) return;
    const long long base = off[c.inst] + c.start;
    const double d = s[(long long)c.inst * stride];
    for (int q = threadIdx.x; q < c.count; q += blockDim.x) y[base + q] = x[base + q] / d;
}

// x += sum_{v < kk[inst]} y[inst][v] Z[v] per reservoir
__global__ void __launch_bounds__(256) k_bcombine(double *__restrict__ x, const double *__restrict__ Z,
                                                  long long ldz, const double *__restrict__ y,
                                                  const int *__restrict__ kk, const BChunk *__restrict__ ch,
                                                  const long long *__restrict__ off,
                                                  const unsigned char *__restrict__ active) {
    const BChunk c = ch[blockIdx.x];
    if (!active[c.inst]) return;
    const long long base = off[c.inst] + c.start;
    const int k = kk[c.inst];
    const double *yc = y + (long long)c.inst * MAX_MDOT;
    for (int q = threadIdx.x; q < c.count; q += blockDim.x) {
        double s = x[base + q];
        for (int v = 0; v < k; ++v) s = fma(yc[v], Z[v * ldz + base + q], s);
        x[base + q] = s;
    }
}

// Per-reservoir FGMRES scalars of one restart cycle, on the device: the Hessenberg
// matrix, the Givens rotations, the rotated right-hand side g, the stop tolerance,
// the residual estimate after each Arnoldi step, the iteration counts.
struct BKrylov {
    double *H;       // [n][(m+1) m]
    double *cs, *sn; // [n][m]
    double *g;       // [n][m+1]
    double *tol;     // [n]
    double *res;     // [n][m]
    int *it;         // [n] Arnoldi steps so far (all cycles)
    int *jend;       // [n] Arnoldi steps of this cycle
    int *bad;        // [n] NaN / Inf met
    int m, maxit;
};

// start of a cycle: H = 0, g = beta e_1 for the reservoirs of the cycle
__global__ void k_bcycle_init(BKrylov K, const double *__restrict__ beta, const unsigned char *__restrict__ cyc,
                              int n) {
    const int i = blockIdx.x;
    if (i >= n || !cyc[i]) return;
    const int m = K.m;
    for (int q = threadIdx.x; q < (m + 1) * m; q += blockDim.x) K.H[(long long)i * (m + 1) * m + q] = 0.0;
    for (int q = threadIdx.x; q <= m; q += blockDim.x) K.g[(long long)i * (m + 1) + q] = q == 0 ? beta[i] : 0.0;
    if (threadIdx.x == 0) K.jend[i] = 0;
}

// Arnoldi step j, one thread per reservoir (the arithmetic of the single-reservoir
// routine, in its order): the column of H from the two CGS passes, the earlier
// rotations applied to it, a new rotation, the residual estimate |g_{j+1}| and the
// stop test; a reservoir that stops (converged, breakdown, iteration limit, NaN) is
// switched off in the mask, so the remaining steps of the cycle skip it.
__global__ void k_bgivens(BKrylov K, const double *__restrict__ out, unsigned char *__restrict__ act, int j, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !act[i]) return;
    const int m = K.m, k = j + 1;
    const double *hh = out + (long long)i * OST;
    double *Hi = K.H + (long long)i * (m + 1) * m;
    double *csi = K.cs + (long long)i * m, *sni = K.sn + (long long)i * m, *gi = K.g + (long long)i * (m + 1);
    for (int a = 0; a < k; ++a) Hi[(long long)a * m + j] = hh[a] + hh[k + 1 + a];
    const double wnorm0 = sqrt(hh[k]);
    const double hn = hh[2 * k + 1];
    Hi[(long long)(j + 1) * m + j] = hn;
    if (!isfinite(hn) || !isfinite(wnorm0)) {
        K.bad[i] = 1;
        act[i] = 0;
        return;
    }
    const bool breakdown = hn <= 1e-14 * wnorm0;
    for (int a = 0; a < j; ++a) {
        const double t = csi[a] * Hi[(long long)a * m + j] + sni[a] * Hi[(long long)(a + 1) * m + j];
        Hi[(long long)(a + 1) * m + j] = -sni[a] * Hi[(long long)a * m + j] + csi[a] * Hi[(long long)(a + 1) * m + j];
        Hi[(long long)a * m + j] = t;
    }
    const double hjj = Hi[(long long)j * m + j], hj1 = Hi[(long long)(j + 1) * m + j];
    const double den = hypot(hjj, hj1);
    csi[j] = hjj / den;
    sni[j] = hj1 / den;
    Hi[(long long)j * m + j] = den;
    Hi[(long long)(j + 1) * m + j] = 0.0;
    gi[j + 1] = -sni[j] * gi[j];
    gi[j] = csi[j] * gi[j];
    const int itn = ++K.it[i];
    const double r = fabs(gi[j + 1]);
    K.res[(long long)i * m + j] = r;
    K.jend[i] = j + 1;
    if (r <= K.tol[i] || breakdown || itn >= K.maxit) act[i] = 0;
}

// end of a cycle: y = H^{-1} g on the cycle's Krylov dimension, per reservoir
__global__ void k_btrisolve(BKrylov K, const unsigned char *__restrict__ cyc, double *__restrict__ y,
                            int *__restrict__ kk, double *__restrict__ lastg, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    kk[i] = 0;
    if (!cyc[i]) return;
    const int m = K.m, kq = K.jend[i];
    const double *Hi = K.H + (long long)i * (m + 1) * m, *gi = K.g + (long long)i * (m + 1);
    double *yi = y + (long long)i * MAX_MDOT;
    for (int a = kq - 1; a >= 0; --a) {
        double s = gi[a];
        for (int l = a + 1; l < kq; ++l) s -= Hi[(long long)a * m + l] * yi[l];
        yi[a] = s / Hi[(long long)a * m + a];
    }
    kk[i] = kq;
    lastg[i] = gi[kq];
}

}  // namespace ras

using namespace ras;

struct ras_batch {
    int n = 0;
    std::vector<ras_problem *> P;
    std::vector<ras_precond *> pc;
    std::vector<long long> off;              // cell offset of each reservoir
    long long Ntot = 0;
    int nch = 0, nbox = 0, qgrid = 0;       // chunks; boxes in the work queue; persistent CTAs
    int *d_qcount = nullptr;                 // work counter of the batched subdomain solves
    FactorParams *d_fp = nullptr;            // [n] the reservoirs' factorisation parameters
    std::vector<int> ch0, chn;               // per reservoir: first chunk, chunks
    int prec = 32, block = 0;
    size_t smem = 0;
    bool twolevel = false;                   // two-level V-cycle preconditioners
    CoarseBatch *cb = nullptr;               // their coarse corrections in one launch (or null: one each)
    std::vector<BOp> ops, opsM;              // host copies: FGMRES operators, V-cycle operators
    std::vector<unsigned char> act;          // host copy of the mask
    // device tables
    BOp *d_ops = nullptr, *d_opsM = nullptr;
    BChunk *d_ch = nullptr;
    long long *d_off = nullptr;
    int *d_ch0 = nullptr, *d_chn = nullptr, *d_kk = nullptr;
    unsigned char *d_act = nullptr;
    ApplyParams *d_ap = nullptr;
    int *d_box_inst = nullptr, *d_box_local = nullptr;
    double *partials = nullptr, *out = nullptr, *h_out = nullptr, *d_y = nullptr, *d_beta = nullptr;
    // per-reservoir FGMRES scalars on the device, and the restart cycle as a CUDA graph
    BKrylov K{};
    int Km = 0;                              // m the device scalars were sized for
    unsigned char *d_cyc = nullptr;          // reservoirs of the current cycle
    double *d_lastg = nullptr;
    std::vector<cudaGraphExec_t> cycle_exec; // the cycle's Arnoldi steps, CYC_CHUNK per graph
    std::vector<long long> cycle_launches;   // kernels in each (counted at every replay)
    int cycle_m = 0;                         // m of the captured cycle
    long long cycle_polls = 0;               // coarse barrier poll limit captured in it
    unsigned char *h_act = nullptr;          // pinned host copy of the mask (between chunks)
    bool graph_off = false;                  // capture failed or disabled: direct launches
    cudaStream_t gstream = nullptr;          // the graph's own stream (joined to the caller's by events)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // streams for the independent per-reservoir launches (Galerkin products and
    // block assembly, residual evaluations), forked from and joined to the caller's
    cudaStream_t pool[NPOOL] = {};
    cudaEvent_t pool_fork_ev = nullptr, pool_join_ev[NPOOL] = {};
    // Krylov and batch vectors
    int m = 0;
    double *V = nullptr, *Z = nullptr, *w = nullptr, *r = nullptr, *b = nullptr, *x = nullptr,
           *tmp = nullptr, *t = nullptr;
};

namespace ras {

static void batch_free(ras_batch *B) {
    if (!B) return;
    coarse_batch_free(B->cb);
    dfree(B->d_ops); dfree(B->d_opsM); dfree(B->t); dfree(B->d_ch); dfree(B->d_off); dfree(B->d_ch0); dfree(B->d_chn); dfree(B->d_kk);
    dfree(B->d_act); dfree(B->d_ap); dfree(B->d_box_inst); dfree(B->d_box_local); dfree(B->d_qcount); dfree(B->d_fp);
    dfree(B->partials); dfree(B->out); dfree(B->d_y); dfree(B->d_beta);
    if (B->h_out) cudaFreeHost(B->h_out);
    dfree(B->V); dfree(B->Z); dfree(B->w); dfree(B->r); dfree(B->b); dfree(B->x); dfree(B->tmp);
    dfree(B->K.H); dfree(B->K.cs); dfree(B->K.sn); dfree(B->K.g); dfree(B->K.tol); dfree(B->K.res);
    dfree(B->K.it); dfree(B->K.jend); dfree(B->K.bad); dfree(B->d_cyc); dfree(B->d_lastg);
    for (auto g : B->cycle_exec)
        if (g) cudaGraphExecDestroy(g);
    if (B->h_act) cudaFreeHost(B->h_act);
    if (B->ev_fork) cudaEventDestroy(B->ev_fork);
    if (B->ev_join) cudaEventDestroy(B->ev_join);
    if (B->gstream) cudaStreamDestroy(B->gstream);
    if (B->pool_fork_ev) cudaEventDestroy(B->pool_fork_ev);
    for (int k = 0; k < NPOOL; ++k) {
        if (B->pool_join_ev[k]) cudaEventDestroy(B->pool_join_ev[k]);
        if (B->pool[k]) cudaStreamDestroy(B->pool[k]);
    }
    delete B;
}

// Fork: every pool stream waits for the work issued so far on st (streams and
// events made on first use). pool_stream(B, q) is the stream of the q-th
// reservoir's launches; join: st waits for everything issued on the pool.
static int pool_fork(ras_batch *B, cudaStream_t st) {
    if (!B->pool_fork_ev) {
        if (cudaEventCreateWithFlags(&B->pool_fork_ev, cudaEventDisableTiming) != cudaSuccess) return RAS_ECUDA;
        for (int k = 0; k < NPOOL; ++k)
            if (cudaStreamCreateWithFlags(&B->pool[k], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&B->pool_join_ev[k], cudaEventDisableTiming) != cudaSuccess)
                return RAS_ECUDA;
    }
    RAS_CK(cudaEventRecord(B->pool_fork_ev, st));
    for (int k = 0; k < NPOOL; ++k) RAS_CK(cudaStreamWaitEvent(B->pool[k], B->pool_fork_ev, 0));
    return RAS_OK;
}
static cudaStream_t pool_stream(ras_batch *B, int q) { return B->pool[q % NPOOL]; }
static int pool_join(ras_batch *B, cudaStream_t st) {
    for (int k = 0; k < NPOOL; ++k) {
        RAS_CK(cudaEventRecord(B->pool_join_ev[k], B->pool[k]));
        RAS_CK(cudaStreamWaitEvent(st, B->pool_join_ev[k], 0));
    }
    return RAS_OK;
}

static int upload_mask(ras_batch *B, cudaStream_t st) {
    RAS_CK(cudaMemcpyAsync(B->d_act, B->act.data(), B->n, cudaMemcpyHostToDevice, st));
    return RAS_OK;
}

static int ensure_krylov_b(ras_batch *B, int m) {
    if (B->m >= m) return RAS_OK;
    dfree(B->V); dfree(B->Z);
    B->m = 0;
    RAS_TRY(dalloc(&B->V, (size_t)(m + 1) * B->Ntot));
    RAS_TRY(dalloc(&B->Z, (size_t)m * B->Ntot));
    B->m = m;
    return RAS_OK;
}

// launches over the batch's chunks
static int b_mdot(ras_batch *B, const double *V, int k, int self, const double *w, cudaStream_t st) {
#define RAS_BMDOT(KM) k_bmdot<KM><<<B->nch, RED_THREADS, 0, st>>>(V, B->Ntot, k, self, w, B->d_ch, B->d_off, \
                                                                   B->d_act, B->partials, B->nch)
    if (k <= 1) RAS_BMDOT(1);
    else if (k <= 2) RAS_BMDOT(2);
    else if (k <= 4) RAS_BMDOT(4);
    else if (k <= 8) RAS_BMDOT(8);
    else if (k <= 16) RAS_BMDOT(16);
    else RAS_BMDOT(32);
#undef RAS_BMDOT
    RAS_LAUNCHED();
    return RAS_OK;
}

static int b_finalize(ras_batch *B, int nvec, int slot0, int sqrt_last, cudaStream_t st) {
    const int wpb = 4;
    k_bfinalize<<<(B->n + wpb - 1) / wpb, 32 * wpb, 0, st>>>(B->partials, B->nch, nvec, B->d_ch0, B->d_chn,
                                                             B->d_act, B->out, slot0, sqrt_last, B->n);
    RAS_LAUNCHED();
    return RAS_OK;
}

template <bool NORM>
static int b_update(ras_batch *B, int k, int hslot, double *w, cudaStream_t st) {
#define RAS_BUPD(KM) k_bupdate<NORM, KM><<<B->nch, RED_THREADS, 0, st>>>(B->V, B->Ntot, k, B->out, hslot, w, \
                                                                         B->d_ch, B->d_off, B->d_act, B->partials)
    if (k <= 1) RAS_BUPD(1);
    else if (k <= 2) RAS_BUPD(2);
    else if (k <= 4) RAS_BUPD(4);
    else if (k <= 8) RAS_BUPD(8);
    else if (k <= 16) RAS_BUPD(16);
    else RAS_BUPD(32);
#undef RAS_BUPD
    RAS_LAUNCHED();
    return RAS_OK;
}

template <bool RESID>
static int b_stencil(ras_batch *B, const double *b, const double *x, double *y, cudaStream_t st,
                     const BOp *ops = nullptr) {
    k_bstencil<RESID><<<B->nch, 256, 0, st>>>(ops ? ops : B->d_ops, B->d_ch, B->d_off, B->d_act, b, x, y);
    RAS_LAUNCHED();
    return RAS_OK;
}

static int b_scale(ras_batch *B, double *y, const double *x, const double *s, int stride, cudaStream_t st) {
    k_bscale<<<B->nch, 256, 0, st>>>(y, x, s, stride, B->d_ch, B->d_off, B->d_act);
    RAS_LAUNCHED();
    return RAS_OK;
}

// z = M^{-1} v for the reservoirs in the mask: left-RAS, or the two-level V-cycle
//   z = M v;  t = v - A z;  z += P A_c^{-1} R t;  t = v - A z;  z += M t
// (A: the operator of each reservoir's last factorisation)
static int b_precond(ras_batch *B, const double *v, double *z, cudaStream_t st) {
    BatchApply A{B->d_ap, B->d_box_inst, B->d_box_local, B->d_off, B->d_act, v, z, 0, B->nbox, B->d_qcount};
    RAS_TRY(ras1_apply_batch(A, B->qgrid, B->prec, B->block, B->smem, st));
    if (!B->twolevel) return RAS_OK;
    RAS_TRY(b_stencil<true>(B, v, z, B->t, st, B->d_opsM));
    if (B->cb) {
        RAS_TRY(coarse_correct_batch(B->cb, B->d_off, B->d_act, B->t, z, st));
    } else {
        for (int i = 0; i < B->n; ++i)
            if (B->act[i]) RAS_TRY(coarse_correct(B->pc[i]->coarse, B->t + B->off[i], z + B->off[i], 1, st));
    }
    RAS_TRY(b_stencil<true>(B, v, z, B->t, st, B->d_opsM));
    A.r = B->t;
    A.accumulate = 1;
    return ras1_apply_batch(A, B->qgrid, B->prec, B->block, B->smem, st);
}

// the V-cycle operators of the reservoirs factored since the last upload
static int refresh_opsM(ras_batch *B, cudaStream_t st) {
    if (!B->twolevel) return RAS_OK;
    for (int i = 0; i < B->n; ++i)
        for (int s = 0; s < 7; ++s) B->opsM[i].c[s] = B->pc[i]->A.c[s];
    RAS_CK(cudaMemcpyAsync(B->d_opsM, B->opsM.data(), B->n * sizeof(BOp), cudaMemcpyHostToDevice, st));
    return RAS_OK;
}

// out[inst][0] = ||vec of inst|| for the reservoirs in the mask (synchronises)
static int b_norms(ras_batch *B, const double *v, std::vector<double> &res, cudaStream_t st) {
    RAS_TRY(b_mdot(B, nullptr, 0, 1, v, st));
    RAS_TRY(b_finalize(B, 1, 0, 1, st));
    RAS_CK(cudaMemcpyAsync(B->h_out, B->out, (size_t)B->n * OST * sizeof(double), cudaMemcpyDeviceToHost, st));
    RAS_CK(cudaStreamSynchronize(st));
    for (int i = 0; i < B->n; ++i) res[i] = B->h_out[(size_t)i * OST];
    return RAS_OK;
}

static int ensure_krylov_dev(ras_batch *B, int m) {
    if (B->Km == m) return RAS_OK;
    BKrylov &K = B->K;
    dfree(K.H); dfree(K.cs); dfree(K.sn); dfree(K.g); dfree(K.tol); dfree(K.res);
    dfree(K.it); dfree(K.jend); dfree(K.bad);
    B->Km = 0;
    const int n = B->n;
    RAS_TRY(dalloc(&K.H, (size_t)n * (m + 1) * m));
    RAS_TRY(dalloc(&K.cs, (size_t)n * m));
    RAS_TRY(dalloc(&K.sn, (size_t)n * m));
    RAS_TRY(dalloc(&K.g, (size_t)n * (m + 1)));
    RAS_TRY(dalloc(&K.tol, n));
    RAS_TRY(dalloc(&K.res, (size_t)n * m));
    RAS_TRY(dalloc(&K.it, n));
    RAS_TRY(dalloc(&K.jend, n));
    RAS_TRY(dalloc(&K.bad, n));
    if (!B->d_cyc) RAS_TRY(dalloc(&B->d_cyc, n));
    if (!B->d_lastg) RAS_TRY(dalloc(&B->d_lastg, n));
    K.m = m;
    B->Km = m;
    for (auto &g : B->cycle_exec) {   // a captured cycle of another m is stale
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
    B->cycle_m = 0;
    return RAS_OK;
}

// The m Arnoldi steps of one restart cycle for every reservoir in the device mask:
// preconditioner, operator, two CGS passes with their norms, the next basis vector,
// and the device-side Hessenberg / Givens step that switches a stopping reservoir off.
// No host data enters: the same launches serve every cycle.
static int b_cycle(ras_batch *B, int j0, int j1, cudaStream_t st) {
    const long long Nt = B->Ntot;
    for (int j = j0; j < j1; ++j) {
        const int k = j + 1;
        double *Vj = B->V + (size_t)j * Nt, *Zj = B->Z + (size_t)j * Nt;
        RAS_TRY(b_precond(B, Vj, Zj, st));
        RAS_TRY(b_stencil<false>(B, nullptr, Zj, B->w, st));
        RAS_TRY(b_mdot(B, B->V, k, 1, B->w, st));
        RAS_TRY(b_finalize(B, k + 1, 0, 0, st));
        RAS_TRY(b_update<false>(B, k, 0, B->w, st));
        RAS_TRY(b_mdot(B, B->V, k, 0, B->w, st));
        RAS_TRY(b_finalize(B, k, k + 1, 0, st));
        RAS_TRY(b_update<true>(B, k, k + 1, B->w, st));
        RAS_TRY(b_finalize(B, 1, 2 * k + 1, 1, st));
        RAS_TRY(b_scale(B, B->V + (size_t)(j + 1) * Nt, B->w, B->out + 2 * k + 1, OST, st));
        k_bgivens<<<(B->n + 63) / 64, 64, 0, st>>>(B->K, B->out, B->d_act, j, B->n);
        RAS_LAUNCHED();
    }
    return RAS_OK;
}

// Runs the cycle in chunks of CYC_CHUNK Arnoldi steps: each chunk's launches are
// captured once (per m and coarse poll limit) as a CUDA graph on the batch's own
// stream, joined to the caller's stream by events, and replayed; between chunks the
// host reads the device mask and ends the cycle once no reservoir is active (the
// remaining steps would change nothing). With RAS_BATCH_GRAPH=0, for a batch whose
// coarse corrections are launched per reservoir from host state, or after a capture
// failed, the same chunks are launched directly.
static int b_run_cycle(ras_batch *B, int m, cudaStream_t st) {
    bool use_graph = !B->graph_off && (!B->twolevel || B->cb);
    if (const char *e = getenv("RAS_BATCH_GRAPH")) use_graph = use_graph && atoi(e) != 0;
    if (use_graph && !B->gstream) {
        if (cudaStreamCreateWithFlags(&B->gstream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&B->ev_join, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            B->graph_off = true;
            use_graph = false;
        }
    }
    const int nchk = (m + CYC_CHUNK - 1) / CYC_CHUNK;
    const long long polls = B->twolevel ? coarse_barrier_polls() : 0;
    if (use_graph && (B->cycle_m != m || B->cycle_polls != polls || (int)B->cycle_exec.size() != nchk)) {
        for (auto &g : B->cycle_exec)
            if (g) cudaGraphExecDestroy(g);
        B->cycle_exec.assign(nchk, nullptr);
        B->cycle_launches.assign(nchk, 0);
        B->cycle_m = m;
        B->cycle_polls = polls;
    }
    for (int c = 0; c < nchk; ++c) {
        const int j0 = c * CYC_CHUNK, j1 = std::min(m, j0 + CYC_CHUNK);
        if (use_graph && !B->cycle_exec[c]) {
            const long long n0 = g_launches.load();
            cudaGraph_t graph = nullptr;
            bool ok = cudaStreamBeginCapture(B->gstream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            long long cnt = 0;
            if (ok) {
                const int rc = b_cycle(B, j0, j1, B->gstream);
                cnt = g_launches.load() - n0;
                const cudaError_t ec = cudaStreamEndCapture(B->gstream, &graph);
                ok = rc >= 0 && ec == cudaSuccess && graph &&
                     cudaGraphInstantiate(&B->cycle_exec[c], graph, 0) == cudaSuccess;
            }
            if (graph) cudaGraphDestroy(graph);
            g_launches.store(n0);
            if (!ok) {                   // nothing ran during the capture: launch directly from now on
                cudaGetLastError();
                B->cycle_exec[c] = nullptr;
                B->graph_off = true;
                use_graph = false;
            } else {
                B->cycle_launches[c] = cnt;
            }
        }
        if (use_graph) {
            RAS_CK(cudaEventRecord(B->ev_fork, st));
            RAS_CK(cudaStreamWaitEvent(B->gstream, B->ev_fork, 0));
            RAS_CK(cudaGraphLaunch(B->cycle_exec[c], B->gstream));
            RAS_CK(cudaEventRecord(B->ev_join, B->gstream));
            RAS_CK(cudaStreamWaitEvent(st, B->ev_join, 0));
            g_launches.fetch_add(B->cycle_launches[c], std::memory_order_relaxed);
        } else {
            RAS_TRY(b_cycle(B, j0, j1, st));
        }
        if (j1 < m) {                    // any reservoir still active in this cycle?
            RAS_CK(cudaMemcpyAsync(B->h_act, B->d_act, (size_t)B->n, cudaMemcpyDeviceToHost, st));
            RAS_CK(cudaStreamSynchronize(st));
            bool any = false;
            for (int i = 0; i < B->n && !any; ++i) any = B->h_act[i] != 0;
            if (!any) break;
        }
    }
    return RAS_OK;
}

// Reads and clears the deferred error words of every selected reservoir (the
// fine factors' and the coarse level's after a factorisation, the
// preconditioner's after a solve), so that an error of one launch is not left
// set for a later call; returns the first error found.
static int drain_checks(ras_batch *B, const std::vector<unsigned char> &sel, bool factor, cudaStream_t st) {
    int first = RAS_OK;
    auto keep = [&](int rc) { if (rc != RAS_OK && first == RAS_OK) first = rc; };
    for (int i = 0; i < B->n; ++i) {
        if (!sel[i]) continue;
        if (factor) {
            keep(ras1_check(B->pc[i]->fine, st));
            if (B->twolevel) keep(coarse_check(B->pc[i]->coarse, st));
        } else {
            keep(precond_check(B->pc[i], st));
        }
    }
    return first;
}

// Batched right-preconditioned FGMRES(m) (the steps of the single-reservoir
// routine, per reservoir) on B->b -> B->x for the reservoirs with want[i];
// operators in B->ops (uploaded by the caller). The Arnoldi scalars of every
// reservoir are updated on the device, so a restart cycle runs without the host
// (one CUDA graph); the host reads the cycle's outcome once per restart.
static int bfgmres_run(ras_batch *B, const std::vector<unsigned char> &want, const ras_krylov_opts &o,
                       ras_krylov_stats *stats, cudaStream_t st) {
    const int n = B->n, m = o.restart;
    if (m < 1 || m > MAX_MDOT - 1 || o.maxit < 1) return RAS_EINVAL;
    RAS_TRY(ensure_krylov_b(B, m));
    RAS_TRY(ensure_krylov_dev(B, m));
    const long long Nt = B->Ntot;
    auto push = [&](int i, double v) {
        if (!stats) return;
        ras_krylov_stats &S = stats[i];
        if (S.history && S.history_len < S.history_cap) S.history[S.history_len++] = v;
    };
    if (stats)
        for (int i = 0; i < n; ++i)
            if (want[i]) { stats[i].history_len = 0; stats[i].iters = 0; stats[i].converged = 0; }
    B->act = want;
    RAS_TRY(upload_mask(B, st));
    std::vector<double> bnorm(n, 0.0), beta(n, 0.0), tol(n, 0.0);
    RAS_TRY(b_norms(B, B->b, bnorm, st));
    for (int i = 0; i < n; ++i) {
        if (!want[i]) continue;
        if (!std::isfinite(bnorm[i])) return RAS_ENAN;
        tol[i] = std::max(o.rtol * bnorm[i], o.atol);
        beta[i] = bnorm[i];
        push(i, beta[i]);
    }
    BKrylov &K = B->K;
    K.maxit = o.maxit;
    RAS_CK(cudaMemcpyAsync(K.tol, tol.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
    RAS_CK(cudaMemsetAsync(K.it, 0, n * sizeof(int), st));
    RAS_CK(cudaMemsetAsync(K.bad, 0, n * sizeof(int), st));
    RAS_TRY(vec_set(B->x, 0.0, (int)Nt, st));
    RAS_TRY(vec_copy(B->r, B->b, (int)Nt, st));
    std::vector<int> it(n, 0), jend(n, 0), bad(n, 0);
    std::vector<unsigned char> conv(n, 0), cyc(n, 0);
    for (int i = 0; i < n; ++i) conv[i] = want[i] && beta[i] <= tol[i];
    std::vector<double> res((size_t)n * m), lastg(n, 0.0);
    for (;;) {
        bool any = false;
        for (int i = 0; i < n; ++i) {
            cyc[i] = want[i] && !conv[i] && it[i] < o.maxit;
            any = any || cyc[i];
        }
        if (!any) break;
        // V_0 = r / beta; g = beta e_1
        RAS_CK(cudaMemcpyAsync(B->d_beta, beta.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
        B->act = cyc;
        RAS_TRY(upload_mask(B, st));
        RAS_CK(cudaMemcpyAsync(B->d_cyc, cyc.data(), n, cudaMemcpyHostToDevice, st));
        RAS_TRY(b_scale(B, B->V, B->r, B->d_beta, 1, st));
        k_bcycle_init<<<n, 64, 0, st>>>(K, B->d_beta, B->d_cyc, n);
        RAS_LAUNCHED();
        RAS_TRY(b_run_cycle(B, m, st));
        // x += Z y per reservoir (its own Krylov dimension); mask back to the cycle's reservoirs
        k_btrisolve<<<(n + 63) / 64, 64, 0, st>>>(K, B->d_cyc, B->d_y, B->d_kk, B->d_lastg, n);
        RAS_LAUNCHED();
        RAS_CK(cudaMemcpyAsync(B->d_act, B->d_cyc, n, cudaMemcpyDeviceToDevice, st));
        B->act = cyc;
        k_bcombine<<<B->nch, 256, 0, st>>>(B->x, B->Z, Nt, B->d_y, B->d_kk, B->d_ch, B->d_off, B->d_act);
        RAS_LAUNCHED();
        RAS_TRY(b_stencil<true>(B, B->b, B->x, B->r, st));
        // the cycle's outcome: iteration counts, steps, residual estimates, NaN flags
        RAS_CK(cudaMemcpyAsync(it.data(), K.it, n * sizeof(int), cudaMemcpyDeviceToHost, st));
        RAS_CK(cudaMemcpyAsync(jend.data(), K.jend, n * sizeof(int), cudaMemcpyDeviceToHost, st));
        RAS_CK(cudaMemcpyAsync(bad.data(), K.bad, n * sizeof(int), cudaMemcpyDeviceToHost, st));
        RAS_CK(cudaMemcpyAsync(res.data(), K.res, res.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        RAS_CK(cudaMemcpyAsync(lastg.data(), B->d_lastg, n * sizeof(double), cudaMemcpyDeviceToHost, st));
        std::vector<double> nb(n, 0.0);
        RAS_TRY(b_norms(B, B->r, nb, st));   // synchronises
        for (int i = 0; i < n; ++i) {
            if (!cyc[i]) continue;
            if (bad[i]) return RAS_ENAN;
            for (int j = 0; j < jend[i]; ++j) push(i, res[(size_t)i * m + j]);
            beta[i] = nb[i];
            if (!std::isfinite(beta[i])) return RAS_ENAN;
            conv[i] = beta[i] <= tol[i] || std::fabs(lastg[i]) <= tol[i];
            if (!conv[i] && it[i] < o.maxit) push(i, beta[i]);
        }
    }
    RAS_TRY(drain_checks(B, want, false, st));
    int status = RAS_OK;
    for (int i = 0; i < n; ++i) {
        if (!want[i]) continue;
        if (stats) {
            stats[i].iters = it[i];
            stats[i].converged = conv[i] ? 1 : 0;
            stats[i].r0 = bnorm[i];
            stats[i].rfinal = beta[i];
        }
        if (!conv[i]) status = RAS_GMRES_MAXIT;
    }
    return status;
}

// The batched FGMRES; on an early error return (a non-finite value after a coarse
// solve whose barrier wait ran out, say) the deferred error words are still read
// and cleared, and the device error, which explains the other, is reported.
static int bfgmres(ras_batch *B, const std::vector<unsigned char> &want, const ras_krylov_opts &o,
                   ras_krylov_stats *stats, cudaStream_t st) {
    const int rc = bfgmres_run(B, want, o, stats, st);
    if (rc >= 0) return rc;
    const int d = drain_checks(B, want, false, st);
    return d != RAS_OK ? d : rc;
}

static void set_ops(ras_batch *B, int i, double *const *J) {
    for (int s = 0; s < 7; ++s) B->ops[i].c[s] = J[s];
}

static int upload_ops(ras_batch *B, cudaStream_t st) {
    RAS_CK(cudaMemcpyAsync(B->d_ops, B->ops.data(), B->ops.size() * sizeof(BOp), cudaMemcpyHostToDevice, st));
    return RAS_OK;
}

// norms of per-reservoir vectors vecs[i] (gathered into B->tmp) for want[i]
static int b_norms_of(ras_batch *B, const std::vector<const double *> &vecs, const std::vector<unsigned char> &want,
                      std::vector<double> &res, cudaStream_t st) {
    for (int i = 0; i < B->n; ++i)
        if (want[i]) RAS_TRY(vec_copy(B->tmp + B->off[i], vecs[i], B->P[i]->N, st));
    B->act = want;
    RAS_TRY(upload_mask(B, st));
    return b_norms(B, B->tmp, res, st);
}

// ras_factor of the live reservoirs on their current Jacobians: the subdomain
// ILU(0) factorisations of all of them in one launch (a CTA per (reservoir, box)).
// Two-level batches also take, per reservoir, the operator copy (the V-cycle's
// operator) and the Galerkin coarse operator with its blocks, then all block
// eliminations in a few cooperative launches; then each reservoir's checks (the
// steps of precond_factor).
static int b_factor(ras_batch *B, const std::vector<int> &cur, const std::vector<unsigned char> &live,
                    cudaStream_t st) {
    const int n = B->n;
    std::vector<FactorParams> fp(n);
    int fblock = 32;
    size_t fsmem = 0;
    for (int i = 0; i < n; ++i) {
        ras_precond *pc = B->pc[i];
        const ras_problem *P = B->P[i];
        Stencil7 A;
        for (int s = 0; s < 7; ++s) A.c[s] = P->nJ[cur[i]][s];
        if (live[i] && B->twolevel) {
            for (int s = 0; s < 7; ++s) {
                RAS_CK(cudaMemcpyAsync(pc->Acopy[s], A.c[s], (size_t)P->N * sizeof(double),
                                       cudaMemcpyDeviceToDevice, st));
                pc->A.c[s] = pc->Acopy[s];
                A.c[s] = pc->Acopy[s];
            }
        }
        ras1_factor_params(pc->fine, A, fp[i]);
        fblock = std::max(fblock, std::min(pc->fine.block, 256));
        fsmem = std::max(fsmem, pc->fine.smem_factor);
    }
    RAS_CK(cudaMemcpyAsync(B->d_fp, fp.data(), n * sizeof(FactorParams), cudaMemcpyHostToDevice, st));
    B->act = live;
    RAS_TRY(upload_mask(B, st));
    RAS_TRY(ras1_factor_batch(B->d_fp, B->d_box_inst, B->d_box_local, B->d_act, B->nbox, B->prec, fblock, fsmem,
                              st));
    if (B->twolevel) {   // each reservoir's Galerkin product and block assembly on a pool stream
        RAS_TRY(pool_fork(B, st));
        for (int i = 0, q = 0; i < n; ++i)
            if (live[i]) RAS_TRY(coarse_factor_prepare(B->pc[i]->coarse, B->pc[i]->A, pool_stream(B, q++)));
        RAS_TRY(pool_join(B, st));
        if (B->cb) {
            RAS_TRY(coarse_factor_batch(B->cb, B->d_act, st));
        } else {
            for (int i = 0; i < n; ++i)
                if (live[i]) RAS_TRY(coarse_factor_blocks(B->pc[i]->coarse, st));
        }
    }
    return drain_checks(B, live, true, st);
}

// One implicit step of every reservoir (the single-reservoir Newton driver's
// steps, per reservoir, with the linear solves batched).
static int bnewton(ras_batch *B, double *const *p, const double *const *pl, const double *const *plm1,
                   const double *dt, int order, const ras_newton_opts &o, ras_newton_stats *stats,
                   cudaStream_t st) {
    const int n = B->n;
    std::vector<int> cur(n, 0), k(n, 0), nres(n, 0), lin_total(n, 0), status(n, RAS_OK);
    RAS_TRY(pool_fork(B, st));   // the reservoirs' residual evaluations on the pool streams
    for (int i = 0; i < n; ++i) {
        ras_problem *P = B->P[i];
        const cudaStream_t sq = pool_stream(B, i);
        RAS_TRY(ensure_newton(P));
        RAS_TRY(vec_copy(P->nX[0], p[i], P->N, sq));
        RAS_TRY(residual_eval_impl(P, P->nX[0], pl[i], order == 2 ? plm1[i] : nullptr, dt[i], order, P->nF[0],
                                   P->nJ[0], sq));
        ++nres[i];
    }
    RAS_TRY(pool_join(B, st));
    std::vector<unsigned char> all(n, 1), live(n, 0);
    std::vector<const double *> vecs(n);
    std::vector<double> fnorm(n, 0.0), f0(n, 0.0), tol(n, 0.0), ft(n, 0.0);
    for (int i = 0; i < n; ++i) vecs[i] = B->P[i]->nF[0];
    RAS_TRY(b_norms_of(B, vecs, all, fnorm, st));
    for (int i = 0; i < n; ++i) {
        if (noroot_take(B->P[i])) return RAS_ENOROOT;
        if (!std::isfinite(fnorm[i])) return RAS_ENAN;
        f0[i] = fnorm[i];
        tol[i] = std::max(o.rtol * f0[i], o.atol);
        live[i] = fnorm[i] > tol[i];
        if (stats) {
            ras_newton_stats &S = stats[i];
            S.fhistory_len = 0; S.iters = 0; S.lin_iters = 0;
            if (S.fhistory && S.fhistory_cap > 0) S.fhistory[S.fhistory_len++] = f0[i];
        }
    }
    std::vector<ras_krylov_stats> ks(n);
    for (;;) {
        bool any = false;
        for (int i = 0; i < n; ++i) {
            if (live[i] && k[i] >= o.maxit) { status[i] = RAS_NEWTON_MAXIT; live[i] = 0; }
            any = any || live[i];
        }
        if (!any) break;
        RAS_TRY(b_factor(B, cur, live, st));
        for (int i = 0; i < n; ++i) {
            if (!live[i]) continue;
            ras_problem *P = B->P[i];
            RAS_TRY(vec_axpby(B->b + B->off[i], -1.0, P->nF[cur[i]], 0.0, P->N, st));
            set_ops(B, i, P->nJ[cur[i]]);
        }
        RAS_TRY(upload_ops(B, st));
        RAS_TRY(refresh_opsM(B, st));
        std::memset(ks.data(), 0, ks.size() * sizeof(ras_krylov_stats));
        const int ls = bfgmres(B, live, o.lin, ks.data(), st);
        if (ls < 0) return ls;
        for (int i = 0; i < n; ++i) {
            if (!live[i]) continue;
            lin_total[i] += ks[i].iters;
            if (stats && stats[i].lin_history && k[i] < stats[i].lin_history_cap) stats[i].lin_history[k[i]] = ks[i].iters;
        }
        // slope_i = F_i^T J_i s_i = -(b_i . J_i s_i)
        B->act = live;
        RAS_TRY(upload_mask(B, st));
        RAS_TRY(b_stencil<false>(B, nullptr, B->x, B->tmp, st));
        RAS_TRY(b_mdot(B, B->b, 1, 0, B->tmp, st));
        RAS_TRY(b_finalize(B, 1, 0, 0, st));
        RAS_CK(cudaMemcpyAsync(B->h_out, B->out, (size_t)n * OST * sizeof(double), cudaMemcpyDeviceToHost, st));
        RAS_CK(cudaStreamSynchronize(st));
        std::vector<double> slope(n, 0.0), phi0(n, 0.0), lam(n, 1.0), lam_prev(n, 0.0), phi_prev(n, 0.0);
        std::vector<unsigned char> first(n, 1), search = live;
        for (int i = 0; i < n; ++i) {
            if (!live[i]) continue;
            slope[i] = -B->h_out[(size_t)i * OST];
            if (!(slope[i] < 0.0)) slope[i] = -fnorm[i] * fnorm[i];
            phi0[i] = 0.5 * fnorm[i] * fnorm[i];
        }
        // line search, all searching reservoirs' trials evaluated together
        for (;;) {
            bool anys = false;
            for (int i = 0; i < n; ++i) anys = anys || search[i];
            if (!anys) break;
            RAS_TRY(pool_fork(B, st));   // the trial residuals on the pool streams
            for (int i = 0, q = 0; i < n; ++i) {
                if (!search[i]) continue;
                ras_problem *P = B->P[i];
                const int nxt = 1 - cur[i];
                const cudaStream_t sq = pool_stream(B, q++);
                RAS_TRY(vec_copy(P->nX[nxt], P->nX[cur[i]], P->N, sq));
                RAS_TRY(vec_axpby(P->nX[nxt], lam[i], B->x + B->off[i], 1.0, P->N, sq));
                RAS_TRY(residual_eval_impl(P, P->nX[nxt], pl[i], order == 2 ? plm1[i] : nullptr, dt[i], order,
                                           P->nF[nxt], P->nJ[nxt], sq));
                ++nres[i];
                vecs[i] = P->nF[nxt];
            }
            RAS_TRY(pool_join(B, st));
            RAS_TRY(b_norms_of(B, vecs, search, ft, st));
            for (int i = 0; i < n; ++i) {
                if (!search[i]) continue;
                if (noroot_take(B->P[i])) ft[i] = NAN;
                if (std::isfinite(ft[i]) && ft[i] <= (1.0 - o.ls_alpha * lam[i]) * fnorm[i]) {
                    search[i] = 0;
                    if (stats && stats[i].lambdas && k[i] < stats[i].lin_history_cap) stats[i].lambdas[k[i]] = lam[i];
                    cur[i] = 1 - cur[i];
                    fnorm[i] = ft[i];
                    ++k[i];
                    if (stats && stats[i].fhistory && stats[i].fhistory_len < stats[i].fhistory_cap)
                        stats[i].fhistory[stats[i].fhistory_len++] = fnorm[i];
                    if (fnorm[i] <= tol[i]) live[i] = 0;
                    continue;
                }
                const double phit = std::isfinite(ft[i]) ? 0.5 * ft[i] * ft[i] : 1e300;
                const double nl = backtrack(lam[i], lam_prev[i], phi0[i], slope[i], phit, phi_prev[i], first[i] != 0);
                first[i] = 0;
                lam_prev[i] = lam[i];
                phi_prev[i] = phit;
                lam[i] = nl;
                if (lam[i] < o.ls_min_lambda) { status[i] = RAS_LINESEARCH_FAIL; search[i] = 0; live[i] = 0; }
            }
        }
    }
    int ret = RAS_OK;
    for (int i = 0; i < n; ++i) {
        ras_problem *P = B->P[i];
        RAS_TRY(vec_copy(p[i], P->nX[cur[i]], P->N, st));
        if (stats) {
            stats[i].iters = k[i];
            stats[i].lin_iters = lin_total[i];
            stats[i].residual_evals = nres[i];
            stats[i].f0 = f0[i];
            stats[i].ffinal = fnorm[i];
        }
        if (ret == RAS_OK && status[i] != RAS_OK) ret = status[i];
    }
    RAS_CK(cudaStreamSynchronize(st));
    return ret;
}

static int batch_create(int n, ras_problem *const *probs, ras_precond *const *pcs, ras_batch **out) {
    ras_batch *B = new ras_batch();
    auto fail = [&](int s) { batch_free(B); return s; };
    B->n = n;
    B->P.assign(probs, probs + n);
    B->pc.assign(pcs, pcs + n);
    std::vector<BChunk> ch;
    std::vector<ApplyParams> ap(n);
    std::vector<int> box_inst, box_local, box_cells;
    long long off = 0;
    for (int i = 0; i < n; ++i) {
        ras_problem *P = probs[i];
        ras_precond *pc = pcs[i];
        if (!P || !pc || pc->prob != P) return fail(RAS_EINVAL);
        for (int q = 0; q < i; ++q)
            if (probs[q] == P) return fail(RAS_EINVAL);   // every reservoir its own handle
        // left-RAS with ILU(0) subdomain solves, one level or the two-level V-cycle with
        // the exact coarse solve; one factor precision and one kind for the batch
        const bool two = pc->coarse != nullptr;
        if (pc->icoarse || pc->xfer || pc->use125 || pc->fine.kind != 1) return fail(RAS_EINVAL);
        if (two && pc->opts.mlevel_type != 0) return fail(RAS_EINVAL);
        if (i == 0) { B->prec = pc->fine.prec; B->twolevel = two; }
        else if (pc->fine.prec != B->prec || two != B->twolevel) return fail(RAS_EINVAL);
        B->off.push_back(off);
        B->ch0.push_back((int)ch.size());
        for (int s = 0; s < P->N; s += BCH) ch.push_back(BChunk{i, s, std::min(BCH, P->N - s)});
        B->chn.push_back((int)ch.size() - B->ch0.back());
        off += ((long long)P->N + 31) / 32 * 32;
        BOp op{};
        op.nx = P->nx; op.ny = P->ny; op.nz = P->nz;
        op.mx = bmagic(P->nx); op.my = bmagic(P->ny);
        B->ops.push_back(op);
        ras1_apply_params(pc->fine, ap[i]);
        for (int q = 0; q < pc->fine.nsub; ++q) {
            box_inst.push_back(i);
            box_local.push_back(q);
            box_cells.push_back(pc->fine.shapes[pc->fine.subs[q].shape].ncell);
        }
        B->block = std::max(B->block, pc->fine.block);
        B->smem = std::max(B->smem, pc->fine.smem_apply);
    }
    if (off > 0x7fffffffLL) return fail(RAS_EINVAL);   // the flat vector kernels take int counts
    {
        const int rq = ras1_batch_grid(B->prec, B->block, B->smem, (int)box_inst.size(), &B->qgrid);
        if (rq < 0) return fail(rq);
    }
    B->Ntot = off;
    B->nch = (int)ch.size();
    B->nbox = (int)box_inst.size();
    {   // the work queue of the batched subdomain solves: largest box first
        std::vector<int> ord(B->nbox);
        for (int q = 0; q < B->nbox; ++q) ord[q] = q;
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return box_cells[a] > box_cells[b]; });
        std::vector<int> bi(B->nbox), bl(B->nbox);
        for (int q = 0; q < B->nbox; ++q) { bi[q] = box_inst[ord[q]]; bl[q] = box_local[ord[q]]; }
        box_inst.swap(bi);
        box_local.swap(bl);
    }
    B->act.assign(n, 1);
    const size_t Nt = (size_t)B->Ntot;
    int rc = 0;
    B->opsM = B->ops;
    if ((rc = dalloc(&B->d_ops, n)) || (rc = dalloc(&B->d_opsM, n)) || (rc = dalloc(&B->t, Nt)) ||
        (rc = dalloc(&B->d_ch, ch.size())) || (rc = dalloc(&B->d_off, n)) ||
        (rc = dalloc(&B->d_ch0, n)) || (rc = dalloc(&B->d_chn, n)) || (rc = dalloc(&B->d_kk, n)) ||
        (rc = dalloc(&B->d_act, n)) || (rc = dalloc(&B->d_ap, n)) || (rc = dalloc(&B->d_box_inst, box_inst.size())) ||
        (rc = dalloc(&B->d_box_local, box_local.size())) || (rc = dalloc(&B->d_qcount, 1)) || (rc = dalloc(&B->d_fp, n)) ||
        (rc = dalloc(&B->partials, (size_t)(MAX_MDOT + 1) * B->nch)) || (rc = dalloc(&B->out, (size_t)n * OST)) ||
        (rc = dalloc(&B->d_y, (size_t)n * MAX_MDOT)) || (rc = dalloc(&B->d_beta, n)) || (rc = dalloc(&B->w, Nt)) ||
        (rc = dalloc(&B->r, Nt)) || (rc = dalloc(&B->b, Nt)) || (rc = dalloc(&B->x, Nt)) || (rc = dalloc(&B->tmp, Nt)))
        return fail(rc);
    if (cudaMallocHost((void **)&B->h_out, (size_t)n * OST * sizeof(double)) != cudaSuccess) {
        B->h_out = nullptr;
        return fail(RAS_ENOMEM);
    }
    if (cudaMallocHost((void **)&B->h_act, (size_t)n) != cudaSuccess) {
        B->h_act = nullptr;
        return fail(RAS_ENOMEM);
    }
    auto up = [&](void *d, const void *h, size_t bytes) {
        return cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    if (!up(B->d_ops, B->ops.data(), n * sizeof(BOp)) || !up(B->d_ch, ch.data(), ch.size() * sizeof(BChunk)) ||
        !up(B->d_off, B->off.data(), n * sizeof(long long)) || !up(B->d_ch0, B->ch0.data(), n * sizeof(int)) ||
        !up(B->d_chn, B->chn.data(), n * sizeof(int)) || !up(B->d_act, B->act.data(), n) ||
        !up(B->d_ap, ap.data(), n * sizeof(ApplyParams)) ||
        !up(B->d_box_inst, box_inst.data(), box_inst.size() * sizeof(int)) ||
        !up(B->d_box_local, box_local.data(), box_local.size() * sizeof(int)))
        return fail(RAS_ECUDA);
    // the padding between reservoirs stays zero in every vector
    if (cudaMemset(B->w, 0, Nt * sizeof(double)) != cudaSuccess || cudaMemset(B->r, 0, Nt * sizeof(double)) ||
        cudaMemset(B->b, 0, Nt * sizeof(double)) || cudaMemset(B->x, 0, Nt * sizeof(double)) ||
        cudaMemset(B->tmp, 0, Nt * sizeof(double)) || cudaMemset(B->t, 0, Nt * sizeof(double)))
        return fail(RAS_ECUDA);
    if (B->twolevel) {
        // one cooperative launch for all coarse corrections when the handles fit in one
        // co-resident grid; otherwise one launch per handle
        std::vector<Coarse *> cs(n);
        for (int i = 0; i < n; ++i) cs[i] = B->pc[i]->coarse;
        if (coarse_batch_setup(cs.data(), n, &B->cb) != RAS_OK) B->cb = nullptr;
        cudaGetLastError();
    }
    *out = B;
    return RAS_OK;
}

}  // namespace ras

extern "C" int ras_batch_create(int n, ras_problem *const *problems, ras_precond *const *preconds,
                                ras_batch **out) {
    if (!out) return RAS_EINVAL;
    *out = nullptr;
    if (n < 1 || !problems || !preconds) return RAS_EINVAL;
    return batch_create(n, problems, preconds, out);
}

extern "C" void ras_batch_destroy(ras_batch *b) { batch_free(b); }

extern "C" int ras_batch_gmres(ras_batch *b, const ras_stencil *J, const double *const *rhs, double *const *x,
                               const ras_krylov_opts *opts, ras_krylov_stats *stats, void *stream) {
    if (!b || !J || !rhs || !x || !opts) return RAS_EINVAL;
    const cudaStream_t st = S(stream);
    for (int i = 0; i < b->n; ++i) {
        if (!rhs[i] || !x[i]) return RAS_EINVAL;
        for (int s = 0; s < 7; ++s)
            if (!J[i].c[s]) return RAS_EINVAL;
        set_ops(b, i, J[i].c);
        RAS_TRY(vec_copy(b->b + b->off[i], rhs[i], b->P[i]->N, st));
    }
    RAS_TRY(upload_ops(b, st));
    RAS_TRY(refresh_opsM(b, st));
    std::vector<unsigned char> all(b->n, 1);
    const int status = bfgmres(b, all, *opts, stats, st);
    if (status < 0) return status;
    for (int i = 0; i < b->n; ++i) RAS_TRY(vec_copy(x[i], b->x + b->off[i], b->P[i]->N, st));
    RAS_CK(cudaStreamSynchronize(st));
    return status;
}

extern "C" int ras_batch_newton_step(ras_batch *b, double *const *p, const double *const *p_l,
                                     const double *const *p_lm1, const double *dt, int bdf_order,
                                     const ras_newton_opts *opts, ras_newton_stats *stats, void *stream) {
    if (!b || !p || !p_l || !dt || !opts) return RAS_EINVAL;
    if (bdf_order != 1 && bdf_order != 2) return RAS_EINVAL;
    if (bdf_order == 2 && !p_lm1) return RAS_EINVAL;
    for (int i = 0; i < b->n; ++i) {
        if (!p[i] || !p_l[i] || !(dt[i] > 0)) return RAS_EINVAL;
        if (bdf_order == 2 && !p_lm1[i]) return RAS_EINVAL;
    }
    return bnewton(b, p, p_l, p_lm1, dt, bdf_order, *opts, stats, S(stream));
}
