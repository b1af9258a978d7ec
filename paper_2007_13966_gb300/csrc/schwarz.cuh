// One-level restricted additive Schwarz on the GPU: set-up tables, ILU(0)
// factorisation and the level-scheduled subdomain solves (Section 3.1).
#pragma once

#include "common.cuh"

namespace ras {

// One distinct overlapped-box shape: its wavefront (level) schedule is shared
// by every subdomain of that shape.
struct ShapeInfo {
    int bx, by, bz, ncell;
    int nlev, nchunk;
    int lvl_off;     // into lvl_tab: nlev + 1 level starts (cell positions)
    int cell_off;    // into cell_tab: ncell packed entries (multiple of 4 aligned)
    int chunk_off;   // into chunk_tab: nchunk + 1 level indices
    int maxw;        // widest level
    int diag_off;    // into diag_tab: by + bz - 1 anti-diagonals d = j + k of the x-pencils (j, k)
    int pxy;         // plane stride of the pipelined apply's vector (bx*by or bx*by + 1)
};

// One anti-diagonal d = j + k of a box's x-pencils (j, k): its first j, its
// pencil count, and the number of pencils on the diagonals before it (inside a
// wavefront level the cells are grouped by diagonal, then ordered by j).
struct DiagInfo {
    int jmin_cnt;    // jmin | cnt << 16
    int base;        // sum of cnt over the diagonals d' < d
};

// One subdomain: overlapped box origin, its shape, owned box (relative to the
// overlapped origin) and the offset of its factor records.
struct SubInfo {
    int e0x, e0y, e0z, shape;
    int ox0, oy0, oz0, ox1, oy1, oz1;
    long long foff;
};

// cell entry: i | j << 8 | k << 16 | flags << 24 (local coordinates)
enum : unsigned {
    F_MX = 1u, F_MY = 2u, F_MZ = 4u, F_PX = 8u, F_PY = 16u, F_PZ = 32u
};

struct Ras1 {
    int nx, ny, nz, N;
    int nsub = 0, nshape = 0;
    int prec = 64;          // 64, 32, 16
    int rec_bytes = 32;     // bytes of one factor record (4 values)
    int block = 128;        // threads per subdomain CTA
    int chunk_cells = 1024; // max cells per staged chunk
    int nbuf = 3;           // staged chunks in flight
    int ycap = 0, lcap = 0; // smem capacities (cells, levels + 1)
    int gcap = 0;           // zero guard band on each side of the apply's vector (cells)
    int maxw = 0;           // widest level over the box shapes
    std::vector<int> h_lvl; // host copy of the level starts (rescheduling)
    size_t smem_apply = 0, smem_factor = 0;
    long long nrec = 0;     // factor records (incl. padding)
    long long ncell_total = 0;  // sum of overlapped cells
    long long nown = 0;
    SubInfo *d_subs = nullptr;
    ShapeInfo *d_shapes = nullptr;
    int *d_lvl = nullptr, *d_chunk = nullptr;
    unsigned *d_cells = nullptr;
    int *d_cidx = nullptr;  // level-ordered local natural index of each cell (apply)
    void *d_fwd = nullptr, *d_bwd = nullptr;
    int *d_err = nullptr;
    // AS (kind 0) and right-RAS (kind 2): each box's whole solution goes to zbuf
    // (at the box's record offset), then every cell sums the boxes covering it
    int kind = 1;
    double *zbuf = nullptr;
    int *d_clo[3] = {}, *d_chi[3] = {}; // per axis and coordinate: first / last part covering it
    int parts[3] = {1, 1, 1};
    std::vector<SubInfo> subs;
    std::vector<ShapeInfo> shapes;
    // pencil-wavefront subdomain solves (left-RAS, FP32 / BF16 factors): one warp
    // per group of x-pencil anti-diagonals
    int pipe = 0;
    int pipe_ok = 0;          // the handle's shapes and options allow the pipelined solves
    int pipe_warps = 0;       // warps per box
    int dcap_pipe = 0;        // anti-diagonal table capacity
    size_t smem_pipe = 0;
    int ycap_pipe = 0;        // floats of the padded box vector
    DiagInfo *d_diag = nullptr;
};

int ras1_setup(Ras1 &R, int nx, int ny, int nz, int px, int py, int pz, int overlap, int prec,
               int kind = 1);
void ras1_free(Ras1 &R);
// numeric ILU(0) of every A_i = R_i^delta A (R_i^delta)^T; no synchronisation
int ras1_factor(Ras1 &R, const Stencil7 &A, cudaStream_t st);
// reads and clears the pivot flag (synchronises)
int ras1_check(Ras1 &R, cudaStream_t st);
// z = M^{-1} r (accumulate = 0) or z += M^{-1} r (accumulate = 1), with
// M^{-1} = sum_i (R_i^0)^T A_i^{-1} R_i^delta (left-RAS, kind 1),
// sum_i (R_i^delta)^T A_i^{-1} R_i^delta (AS, kind 0) or
// sum_i (R_i^delta)^T A_i^{-1} R_i^0 (right-RAS, kind 2)
int ras1_apply(Ras1 &R, const double *r, double *z, int accumulate, cudaStream_t st);
// new chunk size / threads per box for the subdomain solves (0: default); synchronous
int ras1_set_schedule(Ras1 &R, int chunk_cells, int threads);
// subdomain-solve kernel: 0 level-scheduled, 1 pencil-wavefront (both read the
// same records and give the same bits); RAS_EINVAL if not eligible
int ras1_set_kernel(Ras1 &R, int kernel);

// parameters of one handle's apply kernel
struct ApplyParams {
    const SubInfo *subs;
    const ShapeInfo *shapes;
    const int *lvl, *chunk;
    const int *cidx;          // per shape, level order: local natural index of each cell
    const unsigned char *fwd, *bwd;
    const double *r;
    double *z;
    int nx, ny, nz;
    int accumulate;
    int ycap, gcap, lcap, nbuf, chunk_cells;
    int kind;        // 1 left-RAS; 0 AS, 2 right-RAS (box solutions to zbuf)
    double *zbuf;
};
// Left-RAS (kind 1) of several handles in one launch: a persistent kernel whose CTAs
// take boxes (handle, box) from a work queue, largest first (see k_ras_apply_batch)
struct BatchApply {
    const ApplyParams *inst;          // [handles] device copies of the handles' parameters
    const int *box_inst, *box_local;  // [CTAs] handle and box of every CTA
    const long long *off;             // [handles] offset of the handle's cells in r and z
    const unsigned char *active;      // [handles] 0: skip
    const double *r;
    double *z;
    int accumulate;                   // z += (instead of =) the correction
    int nitems;                       // boxes in the work queue (box_inst / box_local order)
    int *qcount;                      // device work counter, cleared before each launch
};
void ras1_apply_params(const Ras1 &R, ApplyParams &P);
// parameters of one handle's ILU(0) factorisation kernel on operator A
struct FactorParams {
    const SubInfo *subs;
    const ShapeInfo *shapes;
    const int *lvl;
    const unsigned *cells;
    Stencil7 A;
    void *fwd, *bwd;
    int nx, ny, nz;
    int *err;
};
void ras1_factor_params(const Ras1 &R, const Stencil7 &A, FactorParams &P);
// the ILU(0) factorisations of several handles in one launch: CTA b factors box
// d_box_local[b] of handle d_box_inst[b] (d_inst: device copies of the handles'
// parameters); no synchronisation (each handle's ras1_check reads its pivot flag)
int ras1_factor_batch(const FactorParams *d_inst, const int *d_box_inst, const int *d_box_local,
                      const unsigned char *d_active, int nbox, int prec, int block, size_t smem, cudaStream_t st);
// persistent launch of `grid` CTAs over the B.nitems boxes of the work queue
int ras1_apply_batch(const BatchApply &B, int grid, int prec, int block, size_t smem, cudaStream_t st);
// CTAs of the batched solve that are co-resident on the device (its persistent grid)
int ras1_batch_grid(int prec, int block, size_t smem, int nitems, int *grid);
double ras1_bytes(const Ras1 &R);

}  // namespace ras
