// Dense FP32 matrix products on the fifth-generation tensor cores (tcgen05) with
// the three-term TF32 split, for the dense blocks of the coarse-level block
// elimination (Section 3.2, the exact coarse solve of the two-level methods).
#pragma once

#include "common.cuh"

namespace ras {

// One product of a batch: C = alpha A B + beta C, row-major FP32, A m x k, B k x n.
struct GemmTask {
    const float *A, *B;
    float *C;
    int lda, ldb, ldc;
};

// Every task of the batch has the same m, n, k: m, n multiples of 128, k a
// multiple of 32, leading dimensions multiples of 4 and 16-byte aligned bases.
// tasks: device array of ntask entries. err: device word set to 2 when a bounded
// wait for the tensor core gave up. No synchronisation.
int tc_gemm_batch(const GemmTask *tasks, int ntask, int m, int n, int k, float alpha, float beta,
                  int *err, cudaStream_t st);

}  // namespace ras
