// Preconditioner handle, right-preconditioned flexible GMRES(m) with CGS2 and
// the inexact Newton driver with cubic backtracking (Sections 2-3).
//
// Vectors, the Krylov basis and every reduction stay on the device; the host
// sees the Hessenberg column (2j + 3 scalars) once per Arnoldi step and keeps
// the Givens rotations, exactly as the scalar logic of the method requires.
#include "precond.cuh"

#include <algorithm>
#include <cstring>

namespace ras {

// ---------------------------------------------------------------------------
// Krylov kernels
// ---------------------------------------------------------------------------


// partials[v][block] = sum_i V[v][i] w[i]  (v < k);  row k: sum_i w[i]^2 if self.
// KM is the compile-time bound on k (the host picks the next power of two).
template <int KM>
__global__ void __launch_bounds__(RED_THREADS) k_mdot(const double *__restrict__ V, long long ldv,
                                                      int k, int self, const double *__restrict__ w,
                                                      int n, double *__restrict__ partials) {
    double acc[KM + 1];
#pragma unroll
    for (int v = 0; v <= KM; ++v) acc[v] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double wi = w[i];
#pragma unroll
        for (int v = 0; v < KM; ++v)
            if (v < k) acc[v] = fma(V[v * ldv + i], wi, acc[v]);
        if (self) acc[KM] = fma(wi, wi, acc[KM]);
    }
    __shared__ double sh[RED_THREADS / 32][KM + 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v <= KM; ++v) {
        double s = acc[v];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) sh[wid][v] = s;
    }
    __syncthreads();
    const int nv = k + (self ? 1 : 0);
    for (int t = threadIdx.x; t < nv; t += blockDim.x) {
        const int v = t < k ? t : KM;
        double s = 0.0;
        for (int q = 0; q < RED_THREADS / 32; ++q) s += sh[q][v];
        partials[(long long)t * RED_BLOCKS + blockIdx.x] = s;
    }
}

// Sums the per-block partials of nvec reductions, one CTA per reduction (grid =
// nvec), each in a fixed order: strided per thread, a warp tree, then the warps in
// order; the square root of the last when sqrt_last.
__global__ void k_finalize_rows(const double *__restrict__ partials, int nvec,
                                double *__restrict__ out, int slot0, int sqrt_last) {
    __shared__ double sh[RED_THREADS / 32];
    const int v = blockIdx.x;
    double acc = 0.0;
    for (int i = threadIdx.x; i < RED_BLOCKS; i += blockDim.x) acc += partials[v * RED_BLOCKS + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < RED_THREADS / 32; ++q) s += sh[q];
        out[slot0 + v] = (sqrt_last && v == nvec - 1) ? sqrt(s) : s;
    }
}

// w -= sum_v h[v] V[v]; optionally partial sums of the new w^2
template <bool NORM, int KM>
__global__ void __launch_bounds__(RED_THREADS) k_update(const double *__restrict__ V, long long ldv,
                                                        int k, const double *__restrict__ h,
                                                        double *__restrict__ w, int n,
                                                        double *__restrict__ partials) {
    double hv[KM];
#pragma unroll
    for (int v = 0; v < KM; ++v) hv[v] = v < k ? h[v] : 0.0;
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = w[i];
#pragma unroll
        for (int v = 0; v < KM; ++v)
            if (v < k) s = fma(-hv[v], V[v * ldv + i], s);
        w[i] = s;
        if (NORM) acc = fma(s, s, acc);
    }
    if (NORM) {
        __shared__ double sh[RED_THREADS / 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int q = 0; q < RED_THREADS / 32; ++q) s += sh[q];
            partials[blockIdx.x] = s;
        }
    }
}

// host dispatch on the next power of two >= k
static int launch_mdot(const double *V, long long ld, int k, int self, const double *w, int n,
                       double *partials, cudaStream_t st) {
#define RAS_MDOT(KM) k_mdot<KM><<<RED_BLOCKS, RED_THREADS, 0, st>>>(V, ld, k, self, w, n, partials)
    if (k <= 1) RAS_MDOT(1);
    else if (k <= 2) RAS_MDOT(2);
    else if (k <= 4) RAS_MDOT(4);
    else if (k <= 8) RAS_MDOT(8);
    else if (k <= 16) RAS_MDOT(16);
    else RAS_MDOT(32);
#undef RAS_MDOT
    RAS_LAUNCHED();
    return RAS_OK;
}

template <bool NORM>
static int launch_update(const double *V, long long ld, int k, const double *h, double *w, int n,
                         double *partials, cudaStream_t st) {
#define RAS_UPD(KM) k_update<NORM, KM><<<RED_BLOCKS, RED_THREADS, 0, st>>>(V, ld, k, h, w, n, partials)
    if (k <= 1) RAS_UPD(1);
    else if (k <= 2) RAS_UPD(2);
    else if (k <= 4) RAS_UPD(4);
    else if (k <= 8) RAS_UPD(8);
    else if (k <= 16) RAS_UPD(16);
    else RAS_UPD(32);
#undef RAS_UPD
    RAS_LAUNCHED();
    return RAS_OK;
}

struct Coefs {
    double y[MAX_MDOT];
};

// x += sum_v y[v] Z[v]
__global__ void k_combine(double *__restrict__ x, const double *__restrict__ Z, long long ldz, int k,
                          Coefs c, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = x[i];
        for (int v = 0; v < k; ++v) s = fma(c.y[v], Z[v * ldz + i], s);
        x[i] = s;
    }
}

static int ensure_krylov(ras_problem *P, int m) {
    if (P->kr_m >= m) return RAS_OK;
    dfree(P->kV); dfree(P->kZ); dfree(P->kw); dfree(P->kr);
    P->kr_m = 0;
    RAS_TRY(dalloc(&P->kV, (size_t)(m + 1) * P->N));
    RAS_TRY(dalloc(&P->kZ, (size_t)m * P->N));
    RAS_TRY(dalloc(&P->kw, P->N));
    RAS_TRY(dalloc(&P->kr, P->N));
    P->kr_m = m;
    return RAS_OK;
}

static inline int gridn(int n) {
    int g = (n + 255) / 256;
    return std::max(1, std::min(g, 152 * 8));
}

// Flexible GMRES(m) on any operator: apply_M(v, z) (z = M^{-1} v), apply_A(z, w)
// (w = A z), resid(b, x, r) (r = b - A x), finish() after the last iteration.
// V [(m+1) N], Z [m N], w, r [N] are the caller's workspace.
template <class ApplyM, class ApplyA, class Resid, class Finish>
static int fgmres_core(int N, double *V, double *Z, double *w, double *r, ReduceWs &red,
                       ApplyM apply_M, ApplyA apply_A, Resid resid, Finish finish,
                       const double *b, double *x, const ras_krylov_opts &o,
                       ras_krylov_stats *stats, cudaStream_t st) {
    const int m = o.restart;
    if (m < 1 || m > MAX_MDOT - 1 || o.maxit < 1) return RAS_EINVAL;
    const long long ld = N;
    auto push = [&](double v) {
        if (stats && stats->history && stats->history_len < stats->history_cap)
            stats->history[stats->history_len++] = v;
    };
    if (stats) { stats->history_len = 0; stats->iters = 0; stats->converged = 0; }

    double bnorm;
    RAS_TRY(norm2_sync(red, b, N, &bnorm, st));
    if (!std::isfinite(bnorm)) return RAS_ENAN;
    const double tol = std::max(o.rtol * bnorm, o.atol);
    RAS_TRY(vec_set(x, 0.0, N, st));
    RAS_TRY(vec_copy(r, b, N, st));
    double beta = bnorm;
    push(beta);
    int it = 0;
    bool converged = beta <= tol;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1);
    auto Hc = [&](int i, int j) -> double & { return H[(size_t)i * m + j]; };
    while (!converged && it < o.maxit) {
        std::fill(H.begin(), H.end(), 0.0);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        RAS_TRY(vec_axpby(V, 1.0 / beta, r, 0.0, N, st));
        int jend = 0;
        for (int j = 0; j < m; ++j) {
            const int k = j + 1;
            double *Vj = V + (size_t)j * N, *Zj = Z + (size_t)j * N;
            RAS_TRY(apply_M(Vj, Zj));
            RAS_TRY(apply_A(Zj, w));
            // CGS pass 1 (+ ||w||^2 before orthogonalisation)
            RAS_TRY(launch_mdot(V, ld, k, 1, w, N, red.partials, st));
            k_finalize_rows<<<k + 1, RED_THREADS, 0, st>>>(red.partials, k + 1, red.out, 0, 0);
            RAS_LAUNCHED();
            RAS_TRY(launch_update<false>(V, ld, k, red.out, w, N, nullptr, st));
            // CGS pass 2
            RAS_TRY(launch_mdot(V, ld, k, 0, w, N, red.partials, st));
            k_finalize_rows<<<k, RED_THREADS, 0, st>>>(red.partials, k, red.out, k + 1, 0);
            RAS_LAUNCHED();
            RAS_TRY(launch_update<true>(V, ld, k, red.out + k + 1, w, N, red.partials, st));
            k_finalize_rows<<<1, RED_THREADS, 0, st>>>(red.partials, 1, red.out, 2 * k + 1, 1);
            RAS_LAUNCHED();
            // v_{j+1} = w / h_{j+1,j} (unused if this step breaks down)
            RAS_TRY(vec_scale_dev(V + (size_t)(j + 1) * N, w, red.out + 2 * k + 1, N, st));
            RAS_CK(cudaMemcpyAsync(red.host, red.out, (2 * k + 2) * sizeof(double),
                                   cudaMemcpyDeviceToHost, st));
            RAS_CK(cudaStreamSynchronize(st));
            const double *hh = red.host;
            for (int i = 0; i < k; ++i) Hc(i, j) = hh[i] + hh[k + 1 + i];
            const double wnorm0 = std::sqrt(hh[k]);
            const double hn = hh[2 * k + 1];
            Hc(j + 1, j) = hn;
            if (!std::isfinite(hn) || !std::isfinite(wnorm0)) return RAS_ENAN;
            const bool breakdown = hn <= 1e-14 * wnorm0;
            for (int i = 0; i < j; ++i) {
                const double t = cs[i] * Hc(i, j) + sn[i] * Hc(i + 1, j);
                Hc(i + 1, j) = -sn[i] * Hc(i, j) + cs[i] * Hc(i + 1, j);
                Hc(i, j) = t;
            }
            const double den = std::hypot(Hc(j, j), Hc(j + 1, j));
            cs[j] = Hc(j, j) / den;
            sn[j] = Hc(j + 1, j) / den;
            Hc(j, j) = den;
            Hc(j + 1, j) = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++it;
            const double res = std::fabs(g[j + 1]);
            push(res);
            jend = j + 1;
            if (res <= tol || breakdown || it >= o.maxit) break;
        }
        const int k = jend;
        Coefs c;
        for (int i = k - 1; i >= 0; --i) {
            double s = g[i];
            for (int l = i + 1; l < k; ++l) s -= Hc(i, l) * c.y[l];
            c.y[i] = s / Hc(i, i);
        }
        k_combine<<<gridn(N), 256, 0, st>>>(x, Z, ld, k, c, N);
        RAS_LAUNCHED();
        RAS_TRY(resid(b, x, r));
        RAS_TRY(norm2_sync(red, r, N, &beta, st));
        if (!std::isfinite(beta)) return RAS_ENAN;
        converged = beta <= tol || std::fabs(g[k]) <= tol;
        if (!converged && it < o.maxit) push(beta);
    }
    RAS_TRY(finish());
    if (stats) {
        stats->iters = it;
        stats->converged = converged ? 1 : 0;
        stats->r0 = bnorm;
        stats->rfinal = beta;
    }
    return converged ? RAS_OK : RAS_GMRES_MAXIT;
}

int fgmres(ras_problem *P, const Stencil7 &A, ras_precond *pc, const double *b, double *x,
           const ras_krylov_opts &o, ras_krylov_stats *stats, cudaStream_t st) {
    if (o.restart < 1 || o.restart > MAX_MDOT - 1 || o.maxit < 1) return RAS_EINVAL;
    RAS_TRY(ensure_krylov(P, o.restart));
    const int nx = P->nx, ny = P->ny, nz = P->nz;
    return fgmres_core(
        P->N, P->kV, P->kZ, P->kw, P->kr, P->red,
        [&](const double *v, double *z) { return precond_apply(pc, v, z, st); },
        [&](const double *z, double *y) { return stencil_apply(A, nx, ny, nz, z, y, st); },
        [&](const double *bb, const double *xx, double *rr) {
            return stencil_residual(A, nx, ny, nz, bb, xx, rr, st);
        },
        [&]() { return precond_check(pc, st); }, b, x, o, stats, st);
}

// ---------------------------------------------------------------------------
// inexact coarse solve (Remark 2): FGMRES on the Galerkin coarse operator,
// preconditioned by left-RAS with ILU(0) on the coarse grid
// ---------------------------------------------------------------------------

struct IterCoarse {
    Transfer *xfer = nullptr;
    int c[3] = {1, 1, 1}, Nc = 0, Nf = 0;     // coarse grid, fine cells
    double *Ac = nullptr;                     // [125][Nc] FP64
    Ras125 M;
    double *V = nullptr, *Z = nullptr, *w = nullptr, *r = nullptr;
    double *tc = nullptr, *xc = nullptr;
    ReduceWs red;
    ras_krylov_opts ko{};
};

int itcoarse_setup(IterCoarse **out, int nx, int ny, int nz, const ras_opts &o) {
    *out = nullptr;
    IterCoarse *c = new IterCoarse();
    auto fail = [&](int s) { itcoarse_free(c); return s; };
    int rc = transfer_setup(&c->xfer, nx, ny, nz, o.coarsen, o.interp_order);
    if (rc) return fail(rc);
    transfer_dims(c->xfer, c->c);
    c->Nc = c->c[0] * c->c[1] * c->c[2];
    c->Nf = nx * ny * nz;
    const int parts[3] = {std::min(o.px, c->c[0]), std::min(o.py, c->c[1]), std::min(o.pz, c->c[2])};
    if ((rc = ras125_setup(c->M, c->c[0], c->c[1], c->c[2], parts[0], parts[1], parts[2],
                           o.coarse_overlap, o.coarse_prec == 32 ? 32 : 64)))
        return fail(rc);
    c->ko.restart = 30;
    c->ko.maxit = 200;
    c->ko.rtol = o.coarse_rtol;
    c->ko.atol = 0.0;
    const size_t Nc = c->Nc;
    if ((rc = dalloc(&c->Ac, 125 * Nc)) || (rc = dalloc(&c->V, (c->ko.restart + 1) * Nc)) ||
        (rc = dalloc(&c->Z, c->ko.restart * Nc)) || (rc = dalloc(&c->w, Nc)) ||
        (rc = dalloc(&c->r, Nc)) || (rc = dalloc(&c->tc, Nc)) || (rc = dalloc(&c->xc, Nc)) ||
        (rc = reduce_ws_init(c->red)))
        return fail(rc);
    *out = c;
    return RAS_OK;
}

void itcoarse_free(IterCoarse *c) {
    if (!c) return;
    if (c->xfer) transfer_free(c->xfer);
    ras125_free(c->M);
    dfree(c->Ac); dfree(c->V); dfree(c->Z); dfree(c->w); dfree(c->r); dfree(c->tc); dfree(c->xc);
    reduce_ws_free(c->red);
    delete c;
}

int itcoarse_factor(IterCoarse *c, const Stencil7 &A, cudaStream_t st) {
    RAS_TRY(transfer_galerkin7(c->xfer, A, c->Ac, nullptr, st));
    return ras125_factor(c->M, c->Ac, st);
}

int itcoarse_check(IterCoarse *c, cudaStream_t st) { return ras125_check(c->M, st); }

int itcoarse_correct(IterCoarse *c, const double *t, double *z, int accumulate, cudaStream_t st) {
    RAS_TRY(transfer_restrict(c->xfer, t, c->tc, st));
    const int *d = c->c;
    const int s = fgmres_core(
        c->Nc, c->V, c->Z, c->w, c->r, c->red,
        [&](const double *v, double *y) { return ras125_apply(c->M, v, y, 0, st); },
        [&](const double *y, double *q) { return spmv125(c->Ac, d[0], d[1], d[2], y, nullptr, q, st); },
        [&](const double *bb, const double *xx, double *rr) {
            return spmv125(c->Ac, d[0], d[1], d[2], xx, bb, rr, st);
        },
        [&]() { return RAS_OK; }, c->tc, c->xc, c->ko, nullptr, st);
    if (s < 0) return s;   // an inexact coarse solve that ran out of iterations is still used
    if (!accumulate) RAS_TRY(vec_set(z, 0.0, c->Nf, st));
    return transfer_prolong(c->xfer, c->xc, z, st);
}

int residual_eval_impl(ras_problem *P, const double *p, const double *pl, const double *plm1,
                       double dt, int order, double *F, double *const *J, cudaStream_t st);

// ---------------------------------------------------------------------------
// Newton
// ---------------------------------------------------------------------------

int ensure_newton(ras_problem *P) {
    if (P->nw_ready) return RAS_OK;
    for (int b = 0; b < 2; ++b) {
        RAS_TRY(dalloc(&P->nX[b], P->N));
        RAS_TRY(dalloc(&P->nF[b], P->N));
        for (int s = 0; s < 7; ++s) RAS_TRY(dalloc(&P->nJ[b][s], P->N));
    }
    RAS_TRY(dalloc(&P->ns, P->N));
    RAS_TRY(dalloc(&P->nrhs, P->N));
    RAS_TRY(dalloc(&P->ntmp, P->N));
    P->nw_ready = true;
    return RAS_OK;
}

// next trial step length of the cubic backtracking (Dennis-Schnabel)
double backtrack(double lam, double lam_prev, double phi0, double slope, double phi_lam,
                 double phi_prev, bool first) {
    double nl;
    if (first) {
        nl = -slope / (2.0 * (phi_lam - phi0 - slope));
    } else {
        const double t1 = phi_lam - phi0 - lam * slope;
        const double t2 = phi_prev - phi0 - lam_prev * slope;
        const double a = (t1 / (lam * lam) - t2 / (lam_prev * lam_prev)) / (lam - lam_prev);
        const double b = (-lam_prev * t1 / (lam * lam) + lam * t2 / (lam_prev * lam_prev)) / (lam - lam_prev);
        if (a == 0.0) {
            nl = -slope / (2.0 * b);
        } else {
            const double d = b * b - 3.0 * a * slope;
            nl = d < 0.0 ? 0.5 * lam : (-b + std::sqrt(d)) / (3.0 * a);
        }
    }
    if (!std::isfinite(nl)) nl = 0.5 * lam;
    return std::min(std::max(nl, 0.1 * lam), 0.5 * lam);
}

int newton(ras_problem *P, ras_precond *pc, double *p, const double *pl, const double *plm1,
           double dt, int order, const ras_newton_opts &o, ras_newton_stats *stats,
           cudaStream_t st) {
    RAS_TRY(ensure_newton(P));
    const int N = P->N;
    int cur = 0;
    RAS_TRY(vec_copy(P->nX[cur], p, N, st));
    double fnorm;
    int nres = 0;
    RAS_TRY(residual_eval_impl(P, P->nX[cur], pl, plm1, dt, order, P->nF[cur], P->nJ[cur], st));
    ++nres;
    RAS_TRY(norm2_sync(P->red, P->nF[cur], N, &fnorm, st));
    if (noroot_take(P)) return RAS_ENOROOT;   // the starting state has no admissible EOS root
    if (!std::isfinite(fnorm)) return RAS_ENAN;
    const double f0 = fnorm;
    const double tol = std::max(o.rtol * f0, o.atol);
    if (stats) {
        stats->fhistory_len = 0;
        stats->iters = 0;
        stats->lin_iters = 0;
        if (stats->fhistory && stats->fhistory_cap > 0) stats->fhistory[stats->fhistory_len++] = f0;
    }
    int status = RAS_OK, k = 0, lin_total = 0;
    while (fnorm > tol) {
        if (k >= o.maxit) { status = RAS_NEWTON_MAXIT; break; }
        Stencil7 A;
        ras_stencil Js;
        for (int s = 0; s < 7; ++s) { A.c[s] = P->nJ[cur][s]; Js.c[s] = P->nJ[cur][s]; }
        RAS_TRY(precond_factor(pc, &Js, st));
        RAS_TRY(vec_axpby(P->nrhs, -1.0, P->nF[cur], 0.0, N, st));
        ras_krylov_stats ks{};
        int ls = fgmres(P, A, pc, P->nrhs, P->ns, o.lin, &ks, st);
        if (ls < 0) return ls;
        lin_total += ks.iters;
        if (stats && stats->lin_history && k < stats->lin_history_cap) stats->lin_history[k] = ks.iters;
        // slope = F^T J s
        RAS_TRY(stencil_apply(A, P->nx, P->ny, P->nz, P->ns, P->ntmp, st));
        double slope;
        RAS_TRY(dot_sync(P->red, P->nF[cur], P->ntmp, N, &slope, st));
        if (!(slope < 0.0)) slope = -fnorm * fnorm;
        const double phi0 = 0.5 * fnorm * fnorm;
        double lam = 1.0, lam_prev = 0.0, phi_prev = 0.0, ft = 0.0;
        bool first = true;
        const int nxt = 1 - cur;
        for (;;) {
            // trial X + lambda s
            RAS_TRY(vec_copy(P->nX[nxt], P->nX[cur], N, st));
            RAS_TRY(vec_axpby(P->nX[nxt], lam, P->ns, 1.0, N, st));
            RAS_TRY(residual_eval_impl(P, P->nX[nxt], pl, plm1, dt, order, P->nF[nxt], P->nJ[nxt], st));
            ++nres;
            RAS_TRY(norm2_sync(P->red, P->nF[nxt], N, &ft, st));
            if (noroot_take(P)) ft = NAN;   // an inadmissible trial state: shorten the step
            if (std::isfinite(ft) && ft <= (1.0 - o.ls_alpha * lam) * fnorm) break;
            const double phit = std::isfinite(ft) ? 0.5 * ft * ft : 1e300;
            const double nl = backtrack(lam, lam_prev, phi0, slope, phit, phi_prev, first);
            first = false;
            lam_prev = lam;
            phi_prev = phit;
            lam = nl;
            if (lam < o.ls_min_lambda) { status = RAS_LINESEARCH_FAIL; break; }
        }
        if (status == RAS_LINESEARCH_FAIL) break;
        if (stats && stats->lambdas && k < stats->lin_history_cap) stats->lambdas[k] = lam;
        cur = nxt;
        fnorm = ft;
        ++k;
        if (stats && stats->fhistory && stats->fhistory_len < stats->fhistory_cap)
            stats->fhistory[stats->fhistory_len++] = fnorm;
    }
    RAS_TRY(vec_copy(p, P->nX[cur], N, st));
    RAS_CK(cudaStreamSynchronize(st));
    if (stats) {
        stats->iters = k;
        stats->lin_iters = lin_total;
        stats->residual_evals = nres;
        stats->f0 = f0;
        stats->ffinal = fnorm;
    }
    return status;
}

}  // namespace ras

using namespace ras;

extern "C" int gmres_solve(ras_problem *P, const ras_stencil *J, ras_precond *pc, const double *b,
                           double *x, const ras_krylov_opts *opts, ras_krylov_stats *stats,
                           void *stream) {
    if (!P || !J || !pc || !b || !x || !opts || b == x) return RAS_EINVAL;
    Stencil7 A;
    for (int s = 0; s < 7; ++s) {
        if (!J->c[s]) return RAS_EINVAL;
        A.c[s] = J->c[s];
    }
    return fgmres(P, A, pc, b, x, *opts, stats, S(stream));
}

extern "C" int newton_step(ras_problem *P, ras_precond *pc, double *p, const double *p_l,
                           const double *p_lm1, double dt, int bdf_order,
                           const ras_newton_opts *opts, ras_newton_stats *stats, void *stream) {
    if (!P || !pc || !p || !p_l || !opts || !(dt > 0)) return RAS_EINVAL;
    if (bdf_order != 1 && bdf_order != 2) return RAS_EINVAL;
    if (bdf_order == 2 && !p_lm1) return RAS_EINVAL;
    return newton(P, pc, p, p_l, p_lm1, dt, bdf_order, *opts, stats, S(stream));
}
