// Coarse-grid correction of the two-level preconditioners (Section 3.2).
#include "precond.cuh"

namespace ras {

struct Coarse {
    int dummy;
};

int coarse_setup(Coarse **out, const ras_problem *, const ras_opts &) {
    *out = nullptr;
    return RAS_EINVAL;
}
void coarse_free(Coarse *c) { delete c; }
int coarse_factor(Coarse *, const Stencil7 &, cudaStream_t) { return RAS_EINVAL; }
int coarse_correct(Coarse *, const double *, double *, int, cudaStream_t) { return RAS_EINVAL; }

}  // namespace ras
