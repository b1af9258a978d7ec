// ras_setup / ras_factor / ras_apply: the one-level left-RAS preconditioner of
// Eq. equ:as-left, the two-level combinations of Section 3.2.1 and the
// three-level V-cycle of Algorithm 1.
#include "precond.cuh"

namespace ras {

static int fine_apply(ras_precond *pc, const double *r, double *z, int accumulate, cudaStream_t st) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (pc->timing) {
        if (pc->ev_used + 2 > pc->ev.size()) {
            for (int i = 0; i < 64; ++i) {
                cudaEvent_t e;
                RAS_CK(cudaEventCreate(&e));
                pc->ev.push_back(e);
            }
        }
        e0 = pc->ev[pc->ev_used++];
        e1 = pc->ev[pc->ev_used++];
        RAS_CK(cudaEventRecord(e0, st));
    }
    if (pc->use125) RAS_TRY(ras125_apply(pc->fine125, r, z, accumulate, st));
    else RAS_TRY(ras1_apply(pc->fine, r, z, accumulate, st));
    if (pc->timing) RAS_CK(cudaEventRecord(e1, st));
    return RAS_OK;
}

int precond_factor(ras_precond *pc, const ras_stencil *J, cudaStream_t st) {
    Stencil7 A;
    for (int s = 0; s < 7; ++s) A.c[s] = J->c[s];
    if (pc->coarse || pc->icoarse) {
        // the multilevel combinations apply J again inside ras_apply: keep a copy
        const int N = pc->prob->N;
        for (int s = 0; s < 7; ++s) {
            RAS_CK(cudaMemcpyAsync(pc->Acopy[s], J->c[s], (size_t)N * sizeof(double),
                                   cudaMemcpyDeviceToDevice, st));
            pc->A.c[s] = pc->Acopy[s];
        }
    }
    // two levels with the exact coarse solve: the fine factors run on a side stream
    // while the Galerkin product and the block assembly run on st; st waits for
    // them before the cooperative block elimination, which needs every SM
    const bool overlap = pc->coarse && !pc->xfer && !pc->use125;
    if (overlap && !pc->side) {
        if (cudaStreamCreateWithFlags(&pc->side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&pc->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&pc->ev_join, cudaEventDisableTiming) != cudaSuccess)
            return RAS_ECUDA;
    }
    if (pc->use125) {
        const ras_problem *P = pc->prob;
        RAS_TRY(embed7(A, P->nx, P->ny, P->nz, pc->A125, st));
        RAS_TRY(ras125_factor(pc->fine125, pc->A125, st));
    } else if (overlap) {
        RAS_CK(cudaEventRecord(pc->ev_fork, st));
        RAS_CK(cudaStreamWaitEvent(pc->side, pc->ev_fork, 0));
        RAS_TRY(ras1_factor(pc->fine, A, pc->side));
        RAS_CK(cudaEventRecord(pc->ev_join, pc->side));
    } else {
        RAS_TRY(ras1_factor(pc->fine, A, st));
    }
    if (pc->xfer) {
        // level 1: A_1 = P_1^T A P_1, its subdomain ILU(0) factors, and the
        // coarsest operator A_0 = P_0^T A_1 P_0 with its dense block LU
        RAS_TRY(transfer_galerkin7(pc->xfer, A, pc->A1, pc->A1f, st));
        RAS_TRY(ras125_factor(pc->mid, pc->A1, st));
        RAS_TRY(coarse_factor125(pc->coarse, pc->A1, st));
    } else if (overlap) {
        RAS_TRY(coarse_factor_prepare(pc->coarse, A, st));
        RAS_CK(cudaStreamWaitEvent(st, pc->ev_join, 0));
        RAS_TRY(coarse_factor_blocks(pc->coarse, st));
    } else if (pc->coarse) {
        RAS_TRY(coarse_factor(pc->coarse, A, st));
    } else if (pc->icoarse) {
        RAS_TRY(itcoarse_factor(pc->icoarse, A, st));
    }
    if (pc->use125) RAS_TRY(ras125_check(pc->fine125, st));
    else RAS_TRY(ras1_check(pc->fine, st));
    if (pc->xfer) RAS_TRY(ras125_check(pc->mid, st));
    if (pc->coarse) RAS_TRY(coarse_check(pc->coarse, st));
    if (pc->icoarse) RAS_TRY(itcoarse_check(pc->icoarse, st));
    return RAS_OK;
}

// two-level coarse correction z (+)= P A_c^{-1} R t, exact or inexact
static int coarse_corr(ras_precond *pc, const double *t, double *z, int accumulate, cudaStream_t st) {
    if (pc->icoarse) return itcoarse_correct(pc->icoarse, t, z, accumulate, st);
    return coarse_correct(pc->coarse, t, z, accumulate, st);
}

// Algorithm 1 with three levels, one pre- and one post-smoothing step of
// Schwarz-preconditioned Richardson on the fine and middle levels, zero
// initial guesses, exact solve on the coarsest level:
//   z = M_2 r;  b_1 = P_1^T (r - A z);
//   x_1 = M_1 b_1;  x_1 += P_0 A_0^{-1} P_0^T (b_1 - A_1 x_1);  x_1 += M_1 (b_1 - A_1 x_1);
//   z += P_1 x_1;  z += M_2 (r - A z).
static int three_level_apply(ras_precond *pc, const double *r, double *z, cudaStream_t st) {
    const ras_problem *P = pc->prob;
    const int nx = P->nx, ny = P->ny, nz = P->nz;
    const int *m = pc->n1;
    double *t = pc->t1;
    RAS_TRY(fine_apply(pc, r, z, 0, st));
    RAS_TRY(stencil_residual(pc->A, nx, ny, nz, r, z, t, st));
    RAS_TRY(transfer_restrict(pc->xfer, t, pc->b1, st));
    RAS_TRY(ras125_apply(pc->mid, pc->b1, pc->x1, 0, st));
    RAS_TRY(spmv125(pc->A1, m[0], m[1], m[2], pc->x1, pc->b1, pc->r1, st));
    RAS_TRY(coarse_correct(pc->coarse, pc->r1, pc->x1, 1, st));
    RAS_TRY(spmv125(pc->A1, m[0], m[1], m[2], pc->x1, pc->b1, pc->r1, st));
    RAS_TRY(ras125_apply(pc->mid, pc->r1, pc->x1, 1, st));
    RAS_TRY(transfer_prolong(pc->xfer, pc->x1, z, st));
    RAS_TRY(stencil_residual(pc->A, nx, ny, nz, r, z, t, st));
    RAS_TRY(fine_apply(pc, t, z, 1, st));
    return RAS_OK;
}

int precond_check(ras_precond *pc, cudaStream_t st) {
    return pc->coarse ? coarse_check(pc->coarse, st) : RAS_OK;   // the inexact coarse solve has no deferred error
}

// z = M^{-1} r for the configured preconditioner
int precond_apply(ras_precond *pc, const double *r, double *z, cudaStream_t st) {
    const ras_problem *P = pc->prob;
    if (!pc->coarse && !pc->icoarse) return fine_apply(pc, r, z, 0, st);
    if (pc->xfer) return three_level_apply(pc, r, z, st);
    const int nx = P->nx, ny = P->ny, nz = P->nz;
    double *t = pc->t1;
    switch (pc->opts.mlevel_type) {
        case 0:  // V-cycle, Eq. equ:v-cycle
            RAS_TRY(fine_apply(pc, r, z, 0, st));                       // e1 = M r
            RAS_TRY(stencil_residual(pc->A, nx, ny, nz, r, z, t, st));   // t = r - A e1
            RAS_TRY(coarse_corr(pc, t, z, 1, st));                       // e2 = e1 + P Ac^-1 R t
            RAS_TRY(stencil_residual(pc->A, nx, ny, nz, r, z, t, st));   // t = r - A e2
            RAS_TRY(fine_apply(pc, t, z, 1, st));                        // e = e2 + M t
            return RAS_OK;
        case 1:  // left-Kaskade, Eq. equ:left-Kas: c + M (r - A c)
            RAS_TRY(coarse_corr(pc, r, z, 0, st));
            RAS_TRY(stencil_residual(pc->A, nx, ny, nz, r, z, t, st));
            RAS_TRY(fine_apply(pc, t, z, 1, st));
            return RAS_OK;
        case 2:  // right-Kaskade, Eq. equ:right-Kas: e + C (r - A e)
            RAS_TRY(fine_apply(pc, r, z, 0, st));
            RAS_TRY(stencil_residual(pc->A, nx, ny, nz, r, z, t, st));
            RAS_TRY(coarse_corr(pc, t, z, 1, st));
            return RAS_OK;
        case 3:  // additive, Eq. equ:two-additive
            RAS_TRY(fine_apply(pc, r, z, 0, st));
            RAS_TRY(coarse_corr(pc, r, z, 1, st));
            return RAS_OK;
        case 4:  // coarse only, Eq. equ:coarse-level
            return coarse_corr(pc, r, z, 0, st);
        default:
            return RAS_EINVAL;
    }
}

}  // namespace ras

using namespace ras;

extern "C" int ras_setup(const ras_problem *P, const ras_opts *o, ras_precond **out) {
    if (!P || !o || !out) return RAS_EINVAL;
    *out = nullptr;
    if (o->ras_type < 0 || o->ras_type > 2 || o->ilu_k < 0) return RAS_EINVAL;
    if (o->ilu_k > 0 && o->ras_type != 1) return RAS_EINVAL;
    if (o->nlevels < 1 || o->nlevels > 3) return RAS_EINVAL;
    if (o->mlevel_type < 0 || o->mlevel_type > 4) return RAS_EINVAL;
    if (o->nlevels == 3 && (o->mlevel_type != 0 || o->coarse_overlap < 0)) return RAS_EINVAL;
    if (o->coarse_solver < 0 || o->coarse_solver > 1) return RAS_EINVAL;
    if (o->nlevels > 1 && o->interp_order != 1 && o->interp_order != 2) return RAS_EINVAL;
    if (o->coarse_solver == 1 && (o->nlevels != 2 || !(o->coarse_rtol > 0.0) || o->coarse_overlap < 0))
        return RAS_EINVAL;
    ras_precond *pc = new ras_precond();
    pc->prob = P;
    pc->opts = *o;
    int rc;
    if (o->ilu_k > 0) {
        pc->use125 = true;
        rc = ras125_setup(pc->fine125, P->nx, P->ny, P->nz, o->px, o->py, o->pz, o->overlap,
                          o->factor_prec, o->ilu_k);
        if (!rc) rc = dalloc(&pc->A125, (size_t)125 * P->N);
        if (!rc && cudaMemset(pc->A125, 0, (size_t)125 * P->N * sizeof(double)) != cudaSuccess)
            rc = RAS_ECUDA;
    } else {
        rc = ras1_setup(pc->fine, P->nx, P->ny, P->nz, o->px, o->py, o->pz, o->overlap,
                        o->factor_prec, o->ras_type);
    }
    if (rc) { ras_precond_destroy(pc); return rc; }
    if (o->nlevels == 3) {
        rc = transfer_setup(&pc->xfer, P->nx, P->ny, P->nz, o->coarsen, o->interp_order);
        if (!rc) {
            transfer_dims(pc->xfer, pc->n1);
            pc->N1 = pc->n1[0] * pc->n1[1] * pc->n1[2];
            rc = ras125_setup(pc->mid, pc->n1[0], pc->n1[1], pc->n1[2], o->px, o->py, o->pz,
                              o->coarse_overlap, o->factor_prec);
        }
        if (!rc) rc = coarse_setup_grid(&pc->coarse, pc->n1[0], pc->n1[1], pc->n1[2], *o);
        if (!rc) rc = dalloc(&pc->A1, (size_t)125 * pc->N1);
        // reduced-precision factors: the middle operator is formed in FP32, as
        // the coarse operator of the two-level method is for coarse_prec 32
        if (!rc && o->factor_prec != 64) rc = dalloc(&pc->A1f, (size_t)125 * pc->N1);
        if (!rc) rc = dalloc(&pc->b1, pc->N1);
        if (!rc) rc = dalloc(&pc->x1, pc->N1);
        if (!rc) rc = dalloc(&pc->r1, pc->N1);
        if (rc) { ras_precond_destroy(pc); return rc; }
    }
    if (o->nlevels >= 2) {
        if (o->coarse_solver == 1) rc = itcoarse_setup(&pc->icoarse, P->nx, P->ny, P->nz, *o);
        else if (!pc->coarse) rc = coarse_setup(&pc->coarse, P, *o);
        if (!rc) rc = dalloc(&pc->t1, P->N);
        if (!rc) rc = dalloc(&pc->t2, P->N);
        if (!rc) rc = dalloc(&pc->t3, P->N);
        for (int s = 0; s < 7 && !rc; ++s) rc = dalloc(&pc->Acopy[s], P->N);
        if (rc) { ras_precond_destroy(pc); return rc; }
    }
    *out = pc;
    return RAS_OK;
}

extern "C" void ras_precond_destroy(ras_precond *pc) {
    if (!pc) return;
    ras1_free(pc->fine);
    ras125_free(pc->fine125);
    dfree(pc->A125);
    if (pc->coarse) coarse_free(pc->coarse);
    if (pc->icoarse) itcoarse_free(pc->icoarse);
    if (pc->xfer) transfer_free(pc->xfer);
    ras125_free(pc->mid);
    dfree(pc->A1); dfree(pc->A1f); dfree(pc->b1); dfree(pc->x1); dfree(pc->r1);
    dfree(pc->t1); dfree(pc->t2); dfree(pc->t3);
    for (int s = 0; s < 7; ++s) dfree(pc->Acopy[s]);
    for (auto e : pc->ev) cudaEventDestroy(e);
    if (pc->ev_fork) cudaEventDestroy(pc->ev_fork);
    if (pc->ev_join) cudaEventDestroy(pc->ev_join);
    if (pc->side) cudaStreamDestroy(pc->side);
    delete pc;
}

extern "C" int ras_factor(ras_precond *pc, const ras_stencil *J, void *stream) {
    if (!pc || !J) return RAS_EINVAL;
    for (int s = 0; s < 7; ++s) if (!J->c[s]) return RAS_EINVAL;
    return precond_factor(pc, J, S(stream));
}

extern "C" int ras_apply(ras_precond *pc, const double *r, double *z, void *stream) {
    if (!pc || !r || !z || r == z) return RAS_EINVAL;
    return precond_apply(pc, r, z, S(stream));
}

extern "C" int ras_timing_enable(ras_precond *pc, int enable) {
    if (!pc) return RAS_EINVAL;
    pc->timing = enable != 0;
    return RAS_OK;
}

extern "C" int ras_timing_read(ras_precond *pc, double *total_ms, long long *launches, int reset) {
    if (!pc) return RAS_EINVAL;
    for (size_t i = 0; i + 1 < pc->ev_used; i += 2) {
        RAS_CK(cudaEventSynchronize(pc->ev[i + 1]));
        float ms = 0.f;
        RAS_CK(cudaEventElapsedTime(&ms, pc->ev[i], pc->ev[i + 1]));
        pc->acc_ms += ms;
        pc->acc_n += 1;
    }
    pc->ev_used = 0;
    if (total_ms) *total_ms = pc->acc_ms;
    if (launches) *launches = pc->acc_n;
    if (reset) { pc->acc_ms = 0.0; pc->acc_n = 0; }
    return RAS_OK;
}

extern "C" double ras_apply_bytes(const ras_precond *pc) {
    if (!pc) return 0.0;
    return pc->use125 ? ras125_bytes(pc->fine125) : ras1_bytes(pc->fine);
}

extern "C" int ras_set_apply_schedule(ras_precond *pc, int chunk_cells, int threads) {
    if (!pc || pc->use125) return RAS_EINVAL;
    return ras1_set_schedule(pc->fine, chunk_cells, threads);
}

extern "C" int ras_set_apply_kernel(ras_precond *pc, int kernel) {
    if (!pc || pc->use125) return RAS_EINVAL;
    return ras1_set_kernel(pc->fine, kernel);
}

extern "C" int ras_get_apply_kernel(const ras_precond *pc, int *kernel) {
    if (!pc || !kernel) return RAS_EINVAL;
    *kernel = pc->use125 ? 0 : pc->fine.pipe;
    return RAS_OK;
}

extern "C" int ras_get_apply_schedule(const ras_precond *pc, int *chunk_cells, int *threads) {
    if (!pc || pc->use125 || !chunk_cells || !threads) return RAS_EINVAL;
    *chunk_cells = pc->fine.chunk_cells;
    *threads = pc->fine.block;
    return RAS_OK;
}
