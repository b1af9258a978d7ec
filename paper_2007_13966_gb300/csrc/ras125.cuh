// Schwarz smoothing on a coarse level of the multilevel method (Section 3.2,
// Algorithm 1): the level operator is a Galerkin product whose couplings reach
// at most two cells along each axis, stored as 125 offset arrays.
#pragma once

#include "common.cuh"

namespace ras {

// slot o = (dx + 2) + 5 (dy + 2) + 25 (dz + 2) of a 125-point operator
constexpr int OP125 = 125;
constexpr int CENTRE125 = 62;
constexpr int RREC = 64;        // values per factor record row (62 couplings + pad + pivot)

// y = A x (b == nullptr) or y = b - A x, A: [125][nx*ny*nz] FP64 on the level grid
int spmv125(const double *A, int nx, int ny, int nz, const double *x, const double *b, double *y,
            cudaStream_t st);

// per overlapped-box shape: level schedule and the offsets split by natural order
struct Shape125 {
    int bx, by, bz, ncell, nlev, maxw;
    int lvl_off, cell_off;
    int nL;                     // offsets whose neighbour precedes a cell (= those after it)
    unsigned char lowo[64];     // lower offsets, ascending natural distance
    unsigned char upo[64];      // upper offsets, ascending natural distance
    signed char uslot[128];     // offset -> position in upo, or -1
    int mask_off;               // ILU(k) pattern: 4 words of offset bits per cell (natural order)
};

struct Sub125 {
    int e0x, e0y, e0z, shape;
    int ox0, oy0, oz0, ox1, oy1, oz1;
    long long foff;             // first factor row (rows in level order)
};

// left-RAS with ILU(0) subdomain solves on a 125-point operator: natural order
// inside each overlapped box, the operator's nonzero pattern, no pivoting
struct Ras125 {
    int nx = 0, ny = 0, nz = 0, N = 0;
    int prec = 64;
    int nsub = 0, nwarps = 8, ycap = 0, lcap = 0;
    long long nrow = 0;                  // factor rows (sum of box cells)
    size_t smem_apply = 0, smem_factor = 0;
    std::vector<Sub125> subs;
    std::vector<Shape125> shapes;
    Sub125 *d_subs = nullptr;
    Shape125 *d_shapes = nullptr;
    int *d_lvl = nullptr;
    unsigned *d_cells = nullptr;
    double *d_work = nullptr;            // [nrow][64] FP64 upper rows + 1/pivot (factor only)
    void *d_fwd = nullptr, *d_bwd = nullptr;   // [nrow][64] records at prec
    int *d_err = nullptr;
    int ilu_k = 0;                       // 0: pattern = nonzeros of A; k > 0: level-of-fill k
    unsigned *d_mask = nullptr;          // ILU(k) patterns per box shape
};

// ilu_k > 0: ILU(k) on the 7-point structure of each box (fill must stay within
// two cells along each axis: k <= 2 for natural order; RAS_EINVAL otherwise)
int ras125_setup(Ras125 &R, int nx, int ny, int nz, int px, int py, int pz, int overlap, int prec,
                 int ilu_k = 0);
// A125 [125][N] <- the 7-point operator A (the other slots must already be zero)
int embed7(const Stencil7 &A, int nx, int ny, int nz, double *A125, cudaStream_t st);
double ras125_bytes(const Ras125 &R);
void ras125_free(Ras125 &R);
// ILU(0) of every A_i = R_i^delta A (R_i^delta)^T; A: [125][N] FP64; no synchronisation
int ras125_factor(Ras125 &R, const double *A, cudaStream_t st);
// reads and clears the pivot flag (synchronises)
int ras125_check(Ras125 &R, cudaStream_t st);
// z = M^{-1} r (accumulate = 0) or z += M^{-1} r; r, z FP64 level vectors
int ras125_apply(Ras125 &R, const double *r, double *z, int accumulate, cudaStream_t st);

}  // namespace ras
