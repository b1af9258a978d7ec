// The preconditioner handle: one-level left-RAS, optionally combined with a
// coarse-grid correction (Section 3.2).
#pragma once

#include "schwarz.cuh"

namespace ras {
struct Coarse;
int coarse_setup(Coarse **out, const ras_problem *P, const ras_opts &o);
void coarse_free(Coarse *c);
int coarse_factor(Coarse *c, const Stencil7 &A, cudaStream_t st);
// reads and clears the coarse pivot / layout flag (synchronises)
int coarse_check(Coarse *c, cudaStream_t st);
// bytes of the dense block factors read by one coarse solve
double coarse_bytes(const Coarse *c);
// ec = A_c^{-1} R t, then z (+)= P ec  (accumulate selects += )
int coarse_correct(Coarse *c, const double *t, double *z, int accumulate, cudaStream_t st);
}  // namespace ras

struct ras_precond {
    const ras_problem *prob = nullptr;
    ras_opts opts{};
    ras::Ras1 fine;
    ras::Coarse *coarse = nullptr;
    ras::Stencil7 A{};          // copy of the operator of the last ras_factor (fine residuals)
    double *Acopy[7] = {};      // owned storage of that copy (two-level only)
    double *t1 = nullptr, *t2 = nullptr, *t3 = nullptr;  // multilevel scratch [N]
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
}  // namespace ras
