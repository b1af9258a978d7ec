// The preconditioner handle: one-level left-RAS, optionally combined with a
// coarse-grid correction (Section 3.2).
#pragma once

#include "ras125.cuh"
#include "schwarz.cuh"

namespace ras {
struct Coarse;
int coarse_setup(Coarse **out, const ras_problem *P, const ras_opts &o);
// the same on the grid of a coarser level (fine grid nx x ny x nz)
int coarse_setup_grid(Coarse **out, int nx, int ny, int nz, const ras_opts &o);
void coarse_free(Coarse *c);
int coarse_factor(Coarse *c, const Stencil7 &A, cudaStream_t st);
// the same from a 125-point level operator Af [125][nx*ny*nz] (FP64)
int coarse_factor125(Coarse *c, const double *Af, cudaStream_t st);
// reads and clears the coarse pivot / layout flag (synchronises)
int coarse_check(Coarse *c, cudaStream_t st);
// The poll limit the coarse kernels' grid barriers take at their next launch
// (RAS_BARRIER_POLLS; 0: the default). A captured launch keeps the value it was
// captured with, so a graph holding one is captured again when this changes.
long long coarse_barrier_polls();
// bytes of the dense block factors read by one coarse solve
double coarse_bytes(const Coarse *c);
// ec = A_c^{-1} R t, then z (+)= P ec  (accumulate selects += )
int coarse_correct(Coarse *c, const double *t, double *z, int accumulate, cudaStream_t st);
// z += P A_c^{-1} P^T t for several handles in one cooperative launch (a group of
// CTAs and a barrier word per handle); t, z: the handles' fine vectors
// concatenated at off[h] (device); handles off in `active` (device) do nothing.
// The coarse factors must be current (coarse_factor); errors go to each handle's
// flag (coarse_check). RAS_EINVAL when the handles' precisions differ or there are
// more handles than co-resident CTAs.
struct CoarseBatch;
int coarse_batch_setup(Coarse *const *cs, int n, CoarseBatch **out);
void coarse_batch_free(CoarseBatch *cb);
int coarse_correct_batch(CoarseBatch *cb, const long long *d_off, const unsigned char *d_active, const double *t,
                         double *z, cudaStream_t st);
// The first part of coarse_factor (Galerkin product, block assembly, couplings),
// then the block eliminations of several handles in one cooperative launch
// (handles off in `active` skip it); coarse_check per handle afterwards.
int coarse_factor_prepare(Coarse *c, const Stencil7 &A, cudaStream_t st);
// the block elimination of blocks assembled by coarse_factor_prepare
int coarse_factor_blocks(Coarse *c, cudaStream_t st);
int coarse_factor_batch(CoarseBatch *cb, const unsigned char *d_active, cudaStream_t st);

// grid transfer to the next coarser level (linear interpolation P, R = P^T)
struct Transfer;
int transfer_setup(Transfer **out, int nx, int ny, int nz, const int ratio[3], int order = 2);
void transfer_free(Transfer *t);
void transfer_dims(const Transfer *t, int c[3]);
// Ac [125][Nc] = P^T A P for a 7-point operator A, stored in FP64; formed in
// FP64, or in FP32 (then widened) when an FP32 scratch [125][Nc] is given
int transfer_galerkin7(Transfer *t, const Stencil7 &A, double *Ac, float *scratch, cudaStream_t st);
int transfer_restrict(Transfer *t, const double *x, double *xc, cudaStream_t st);   // xc = P^T x
int transfer_prolong(Transfer *t, const double *xc, double *x, cudaStream_t st);    // x += P xc

// inexact coarse solve: FGMRES on A_c = P^T A P preconditioned by left-RAS(ILU(0))
// on the coarse grid, to a relative tolerance
struct IterCoarse;
int itcoarse_setup(IterCoarse **out, int nx, int ny, int nz, const ras_opts &o);
void itcoarse_free(IterCoarse *c);
int itcoarse_factor(IterCoarse *c, const Stencil7 &A, cudaStream_t st);
int itcoarse_check(IterCoarse *c, cudaStream_t st);
// xc ~= A_c^{-1} R t, then z (+)= P xc
int itcoarse_correct(IterCoarse *c, const double *t, double *z, int accumulate, cudaStream_t st);
}  // namespace ras

struct ras_precond {
    const ras_problem *prob = nullptr;
    ras_opts opts{};
    ras::Ras1 fine;
    // ILU(k > 0): the fine level runs on the 125-offset machinery (7-point
    // operator embedded, level-of-fill pattern per box shape)
    bool use125 = false;
    ras::Ras125 fine125;
    double *A125 = nullptr;             // [125][N] embedded fine operator
    ras::Coarse *coarse = nullptr;
    ras::IterCoarse *icoarse = nullptr;   // coarse_solver = 1 (two levels)
    ras::Stencil7 A{};          // copy of the operator of the last ras_factor (fine residuals)
    double *Acopy[7] = {};      // owned storage of that copy (two-level only)
    double *t1 = nullptr, *t2 = nullptr, *t3 = nullptr;  // multilevel scratch [N]
    // three levels (Algorithm 1): fine -> middle level 1 -> coarsest level 0
    ras::Transfer *xfer = nullptr;       // fine grid -> level 1
    int n1[3] = {0, 0, 0}, N1 = 0;       // level-1 grid
    double *A1 = nullptr;                // [125][N1] Galerkin operator of level 1
    float *A1f = nullptr;                // FP32 scratch of A1 (reduced-precision factors)
    ras::Ras125 mid;                     // RAS(ILU(0)) smoother of level 1
    double *b1 = nullptr, *x1 = nullptr, *r1 = nullptr;  // level-1 vectors [N1]
    // factorisation: the fine factors on a side stream next to the Galerkin product
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    double acc_ms = 0.0;
    long long acc_n = 0;
};

namespace ras {
int precond_factor(ras_precond *pc, const ras_stencil *J, cudaStream_t st);
int precond_apply(ras_precond *pc, const double *r, double *z, cudaStream_t st);
// reports (and clears) an error recorded by the asynchronous coarse solves
int precond_check(ras_precond *pc, cudaStream_t st);
// Newton helpers shared by the single and the batched drivers
int ensure_newton(ras_problem *P);
double backtrack(double lam, double lam_prev, double phi0, double slope, double phi_lam,
                 double phi_prev, bool first);
int residual_eval_impl(ras_problem *P, const double *p, const double *pl, const double *plm1,
                       double dt, int order, double *F, double *const *J, cudaStream_t st);
// reads and clears the problem's no-admissible-EOS-root flag (after a synchronisation)
bool noroot_take(ras_problem *P);
}  // namespace ras
