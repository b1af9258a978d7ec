// One-level restricted additive Schwarz (Section 3.1) on sm_103a.
//
// The paper's subdomains (one per MPI rank on Tianhe-2) become one CTA each.
// Inside a subdomain the natural-order ILU(0) triangular solves are run as a
// wavefront: cells with equal i + j + k form a level, levels are separated by
// CTA barriers, and the working vector lives in shared memory. Factor records
// are stored in level order so that each staged chunk of consecutive levels is
// one contiguous range, streamed into a shared-memory ring with cp.async ahead
// of the sweep that consumes it.
#include "schwarz.cuh"

#include <algorithm>
#include <cstdlib>
#include <map>
#include <tuple>

namespace ras {

// ---------------------------------------------------------------------------
// factor record types
// ---------------------------------------------------------------------------

struct RecF64 { double a, b, c, d; };
struct __align__(16) RecF32 { float a, b, c, d; };
struct __align__(8) RecB16 { __nv_bfloat16 a, b, c, d; };

template <int PREC> struct RecT;
template <> struct RecT<64> { using T = RecF64; using Acc = double; };
template <> struct RecT<32> { using T = RecF32; using Acc = float; };
template <> struct RecT<16> { using T = RecB16; using Acc = float; };

__device__ __forceinline__ RecF64 make_rec64(double a, double b, double c, double d) {
    return RecF64{a, b, c, d};
}

template <int PREC>
__device__ __forceinline__ void store_rec(void *base, long long idx, double a, double b, double c,
                                          double d) {
    if constexpr (PREC == 64) {
        reinterpret_cast<RecF64 *>(base)[idx] = RecF64{a, b, c, d};
    } else if constexpr (PREC == 32) {
        reinterpret_cast<RecF32 *>(base)[idx] = RecF32{(float)a, (float)b, (float)c, (float)d};
    } else {
        // FP64 -> FP32 -> BF16, each round to nearest even
        RecB16 r;
        r.a = __float2bfloat16_rn((float)a);
        r.b = __float2bfloat16_rn((float)b);
        r.c = __float2bfloat16_rn((float)c);
        r.d = __float2bfloat16_rn((float)d);
        reinterpret_cast<RecB16 *>(base)[idx] = r;
    }
}

template <typename Acc, typename R>
__device__ __forceinline__ void load_rec(const unsigned char *p, Acc &a, Acc &b, Acc &c, Acc &d) {
    if constexpr (sizeof(R) == 32) {
        const double2 *q = reinterpret_cast<const double2 *>(p);
        const double2 u = q[0], v = q[1];
        a = u.x; b = u.y; c = v.x; d = v.y;
    } else if constexpr (sizeof(R) == 16) {
        const float4 u = *reinterpret_cast<const float4 *>(p);
        a = u.x; b = u.y; c = u.z; d = u.w;
    } else {
        const RecB16 u = *reinterpret_cast<const RecB16 *>(p);
        a = __bfloat162float(u.a); b = __bfloat162float(u.b);
        c = __bfloat162float(u.c); d = __bfloat162float(u.d);
    }
}

// Multiply-adds of the triangular sweeps, fused explicitly so that every kernel
// that runs them rounds identically: fmsub(a, b, s) = s - a b, fmadd(a, b, s) = s + a b.
__device__ __forceinline__ float fmsub(float a, float b, float s) { return __fmaf_rn(-a, b, s); }
__device__ __forceinline__ double fmsub(double a, double b, double s) { return __fma_rn(-a, b, s); }
__device__ __forceinline__ float fmadd(float a, float b, float s) { return __fmaf_rn(a, b, s); }
__device__ __forceinline__ double fmadd(double a, double b, double s) { return __fma_rn(a, b, s); }

// ---------------------------------------------------------------------------
// cp.async staging
// ---------------------------------------------------------------------------

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// copy the 16-byte-aligned window around global bytes [b0, b1) of `base`
// into `dst`; the data of byte b0 lands at dst + (b0 & 15)
__device__ __forceinline__ void stage_bytes(unsigned char *dst, const unsigned char *base,
                                            long long b0, long long b1) {
    const long long a0 = b0 & ~15LL;
    const long long a1 = (b1 + 15) & ~15LL;
    for (long long o = a0 + 16LL * threadIdx.x; o < a1; o += 16LL * blockDim.x)
        cp_async16(dst + (o - a0), base + o);
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// q / d for 0 <= q < 2^16 and 1 <= d <= 256 as a multiply-high by ceil(2^32 / d)
// (exact in that range: q (ceil(2^32/d) d - 2^32) < 2^32 since the excess is < d)
__host__ __device__ __forceinline__ unsigned magic_div(int d) {
    return d == 1 ? 0u : (unsigned)((0x100000000ull + (unsigned)d - 1) / (unsigned)d);
}
__device__ __forceinline__ int fast_div(int q, int d, unsigned m) {
    return d == 1 ? q : (int)__umulhi((unsigned)q, m);
}



// One subdomain solve (one CTA): box `box` of the handle described by P, input r,
// output z (whole-grid vectors of that handle).
template <int PREC, int NBUF>
__device__ __forceinline__ void ras_apply_box(const ApplyParams &P, int box, const double *r, double *z,
                                              int accumulate) {
    using R = typename RecT<PREC>::T;
    using Acc = typename RecT<PREC>::Acc;
    constexpr int RB = (int)sizeof(R);
    extern __shared__ __align__(16) unsigned char smem[];
    // [zero guard: gcap][Y: ycap][zero guard: gcap][level starts][ring]
    Acc *Y = reinterpret_cast<Acc *>(smem) + P.gcap;
    const size_t ybytes = ((size_t)P.ycap + 2 * (size_t)P.gcap) * sizeof(Acc);
    int *lvl_s = reinterpret_cast<int *>(smem + ybytes);
    unsigned char *ring = smem + ybytes + (size_t)P.lcap * sizeof(int);
    const int rcap = ((P.chunk_cells * RB + 32) + 15) & ~15;
    const int ccap = ((P.chunk_cells * 4 + 32) + 15) & ~15;
    unsigned char *ring_rec = ring;
    unsigned char *ring_cell = ring + (size_t)NBUF * rcap;

    const SubInfo si = P.subs[box];
    const ShapeInfo sh = P.shapes[si.shape];
    const int *chunk_lev = P.chunk + sh.chunk_off;
    for (int t = threadIdx.x; t <= sh.nlev; t += blockDim.x) lvl_s[t] = P.lvl[sh.lvl_off + t];
    for (int t = threadIdx.x; t < sh.bx * sh.by; t += blockDim.x) {
        Y[-1 - t] = (Acc)0;
        Y[sh.ncell + t] = (Acc)0;
    }
    __syncthreads();

    const int nstage = 2 * sh.nchunk;
    const bool one = (int)blockDim.x >= sh.maxw;   // one cell per thread per level
    auto issue = [&](int t) {
        if (t < nstage) {
            const bool fw = t < sh.nchunk;
            const int c = fw ? t : nstage - 1 - t;
            const int qa = lvl_s[chunk_lev[c]], qb = lvl_s[chunk_lev[c + 1]];
            const int slot = t % NBUF;
            stage_bytes(ring_rec + (size_t)slot * rcap, fw ? P.fwd : P.bwd,
                        (si.foff + qa) * (long long)RB, (si.foff + qb) * (long long)RB);
            stage_bytes(ring_cell + (size_t)slot * ccap,
                        reinterpret_cast<const unsigned char *>(P.cidx),
                        (sh.cell_off + (long long)qa) * 4, (sh.cell_off + (long long)qb) * 4);
        }
        cp_async_commit();
    };
#pragma unroll
    for (int t = 0; t < NBUF - 1; ++t) issue(t);

    // gather R_i^delta r into shared memory, flat over the box's cells with GB
    // loads in flight per thread before any is consumed (the gather is bound by
    // the bytes in flight per SM, not by bandwidth)
    constexpr int GB = 10;   // a batch that stays in 64 registers with the direct z stores
    const int bx = sh.bx, by = sh.by, bxy = sh.bx * sh.by;
    const int nx = P.nx, nxy = P.nx * P.ny;
    const long long g0 = si.e0x + (long long)nx * (si.e0y + (long long)P.ny * si.e0z);
    const double *rg = r + g0;
    const unsigned mbx = magic_div(bx), mby = magic_div(by);
    for (int q0 = threadIdx.x; q0 < sh.ncell; q0 += GB * blockDim.x) {
        double v[GB];
#pragma unroll
        for (int m = 0; m < GB; ++m) {
            const int q = q0 + m * (int)blockDim.x;
            if (q < sh.ncell) {
                const int row = fast_div(q, bx, mbx), k = fast_div(row, by, mby);
                v[m] = __ldg(rg + (q - row * bx) + nx * (row - k * by) + nxy * k);
            }
        }
#pragma unroll
        for (int m = 0; m < GB; ++m) {
            const int q = q0 + m * (int)blockDim.x;
            if (q < sh.ncell) {
                bool own = true;
                if (P.kind == 2) {   // right-RAS: R_i^0 on the input (cells of other boxes read as 0)
                    const int row = fast_div(q, bx, mbx), k = fast_div(row, by, mby);
                    const int i = q - row * bx, j = row - k * by;
                    own = i >= si.ox0 && i < si.ox1 && j >= si.oy0 && j < si.oy1 && k >= si.oz0 &&
                          k < si.oz1;
                }
                Y[q] = own ? (Acc)v[m] : (Acc)0;
            }
        }
    }

    // Left-RAS writes each owned cell's z as soon as the backward sweep has it
    // ((R_i^0)^T: one owner per cell, so an add when accumulating is a plain update)
    const bool direct = P.kind == 1;
    double *zg = z + g0;
    auto put = [&](int n, Acc y) {
        const int row = fast_div(n, bx, mbx), k = fast_div(row, by, mby);
        const int i = n - row * bx, j = row - k * by;
        if (i >= si.ox0 && i < si.ox1 && j >= si.oy0 && j < si.oy1 && k >= si.oz0 && k < si.oz1) {
            double *zp = zg + (i + nx * j + nxy * k);
            if (accumulate) atomicAdd(zp, (double)y);
            else *zp = (double)y;
        }
    };

    // Sweeps, level by level. A neighbour outside the box has a zero factor value and
    // reads a finite value (a cell of the box or the zero guard band on either side
    // of Y), so no cell needs a flag test.
    for (int t = 0; t < nstage; ++t) {
        cp_async_wait<NBUF - 2>();
        __syncthreads();
        issue(t + NBUF - 1);
        const bool fw = t < sh.nchunk;
        const int c = fw ? t : nstage - 1 - t;
        const int l0 = chunk_lev[c], l1 = chunk_lev[c + 1];
        const int qa = lvl_s[l0];
        const int slot = t % NBUF;
        const unsigned char *rec = ring_rec + (size_t)slot * rcap +
                                   (int)(((si.foff + qa) * (long long)RB) & 15);
        const int *cel = reinterpret_cast<const int *>(
            ring_cell + (size_t)slot * ccap + (int)(((sh.cell_off + (long long)qa) * 4) & 15));
        // When the block covers the widest level, a level is one guarded pass (no loop
        // back-edge before the barrier) with addresses from per-chunk bases.
        const int tid = threadIdx.x;
        const int *cel_t = cel - qa + tid;                       // cel_t[lo]: cell lo + tid
        const unsigned char *rec_t = rec + (long long)RB * (tid - qa);
        if (one) {
            if (fw) {
#pragma unroll 2
                for (int l = l0; l < l1; ++l) {
                    const int lo = lvl_s[l];
                    if (lo + tid < lvl_s[l + 1]) {
                        const int n = cel_t[lo];
                        Acc ax, ay, az, dinv;
                        load_rec<Acc, R>(rec_t + (size_t)RB * lo, ax, ay, az, dinv);
                        Acc *yn = Y + n;
                        Acc s = yn[0];
                        s = fmsub(az, yn[-bxy], s);
                        s = fmsub(ay, yn[-bx], s);
                        s = fmsub(ax, yn[-1], s);
                        yn[0] = s * dinv;
                    }
                    __syncthreads();
                }
            } else {
#pragma unroll 2
                for (int l = l1 - 1; l >= l0; --l) {
                    const int lo = lvl_s[l];
                    if (lo + tid < lvl_s[l + 1]) {
                        const int n = cel_t[lo];
                        Acc ax, ay, az, dinv;
                        load_rec<Acc, R>(rec_t + (size_t)RB * lo, ax, ay, az, dinv);
                        Acc *yn = Y + n;
                        Acc s = ax * yn[1];
                        s = fmadd(ay, yn[bx], s);
                        s = fmadd(az, yn[bxy], s);
                        const Acc y = fmsub(dinv, s, yn[0]);
                        yn[0] = y;
                        if (direct) put(n, y);
                    }
                    __syncthreads();
                }
            }
            continue;
        }
        if (fw) {
            // forward: w_n = (r_n - sum_{m<n} a_nm w_m) / d_n, w = D^{-1} L^{-1} r
            for (int l = l0; l < l1; ++l) {
                const int q1 = lvl_s[l + 1];
                for (int q = lvl_s[l] + threadIdx.x; q < q1; q += blockDim.x) {
                    const int n = cel[q - qa];
                    Acc ax, ay, az, dinv;
                    load_rec<Acc, R>(rec + (size_t)RB * (q - qa), ax, ay, az, dinv);
                    Acc s = Y[n];
                    s = fmsub(az, Y[n - bxy], s);
                    s = fmsub(ay, Y[n - bx], s);
                    s = fmsub(ax, Y[n - 1], s);
                    Y[n] = s * dinv;
                }
                __syncthreads();
            }
        } else {
            // backward: z_n = w_n - d_n^{-1} sum_{m>n} a_nm z_m
            for (int l = l1 - 1; l >= l0; --l) {
                const int q1 = lvl_s[l + 1];
                for (int q = lvl_s[l] + threadIdx.x; q < q1; q += blockDim.x) {
                    const int n = cel[q - qa];
                    Acc ax, ay, az, dinv;
                    load_rec<Acc, R>(rec + (size_t)RB * (q - qa), ax, ay, az, dinv);
                    Acc s = ax * Y[n + 1];
                    s = fmadd(ay, Y[n + bx], s);
                    s = fmadd(az, Y[n + bxy], s);
                    const Acc y = fmsub(dinv, s, Y[n]);
                    Y[n] = y;
                    if (direct) put(n, y);
                }
                __syncthreads();
            }
        }
    }
    cp_async_wait<0>();

    if (P.kind != 1) {   // AS / right-RAS: the whole box solution, summed per cell later
        double *dst = P.zbuf + si.foff;
        for (int q = threadIdx.x; q < sh.ncell; q += blockDim.x) dst[q] = (double)Y[q];
        return;
    }
}

template <int PREC, int NBUF>
__global__ void __launch_bounds__(512, 2) k_ras_apply(ApplyParams P) {
    ras_apply_box<PREC, NBUF>(P, blockIdx.x, P.r, P.z, P.accumulate);
}

// Left-RAS of many handles in one persistent launch: every CTA takes the next
// item of a work queue (an atomic counter over the table of (handle, box), sorted
// largest box first) until the queue is empty, and solves box box_local[item] of
// handle box_inst[item] (items of inactive handles are skipped); r and z are the
// handles' vectors concatenated at off[handle]. No CTA waits on another.
template <int PREC, int NBUF>
__global__ void __launch_bounds__(512, 2) k_ras_apply_batch(BatchApply B) {
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(B.qcount, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();   // every thread holds the item, and the last box's shared memory is free
        if (it >= B.nitems) return;
        const int h = B.box_inst[it];
        if (!B.active[h]) continue;
        ras_apply_box<PREC, NBUF>(B.inst[h], B.box_local[it], B.r + B.off[h], B.z + B.off[h], B.accumulate);
    }
}

// ---------------------------------------------------------------------------
// Pencil-wavefront subdomain solves (left-RAS, FP32 / BF16 factors)
//
// The natural-order ILU(0) sweeps of a box run over its x-pencils (j, k), one
// thread per pencil: pencil (j, k) handles its cells i = 0 .. bx-1 one per
// wavefront level, cell i at level i + j + k, so that its -y and -z neighbours,
// cells of the pencils (j-1, k) and (j, k-1), were finished at the previous level
// and its -x neighbour is the pencil's previous value, kept in a register (the
// backward sweep mirrors this). Consecutive levels are separated by one CTA
// barrier. Pencils are numbered by anti-diagonal d = j + k, then j, so that a warp
// holds pencils of one or two neighbouring diagonals: it is busy for about bx + 2
// levels of a sweep with most lanes active and idles (only the barrier) otherwise.
// A thread's cell, neighbour and record positions follow from its pencil and the
// level with no table look-up on the dependent chain (level start -> cell index ->
// values in the level-scheduled kernel). The factor records are in level order with
// the cells of a level grouped by anti-diagonal, then j (the layout both solve
// kernels read): the record of pencil number p at level l is record lb[l] + p with
// lb[l] = (start of level l) - (pencils on the diagonals below the level's first).
// Chunks of consecutive levels are staged into a shared-memory ring with cp.async
// two chunks ahead. The backward sweep writes each owned cell's z as soon as it is
// final (an add when accumulating: one owner per cell). The arithmetic of every
// cell is the same as in the level-scheduled kernel, in the same order.
// ---------------------------------------------------------------------------

struct PipeParams {
    const SubInfo *subs;
    const ShapeInfo *shapes;
    const DiagInfo *diag;
    const int *lvl, *chunk;
    const unsigned char *fwd, *bwd;
    const double *r;
    double *z;
    int nx, ny, nz;
    int accumulate;
    int ycap;          // elements of the padded box vector
    int lcap;          // level starts (incl. the end) capacity
    int chunk_cells;   // ring slot capacity (cells)
};

template <int PREC>
__global__ void __launch_bounds__(1024, 1) k_ras_pipe(PipeParams P) {
    using R = typename RecT<PREC>::T;
    using Acc = typename RecT<PREC>::Acc;
    constexpr int RB = (int)sizeof(R);
    constexpr int NBUF = 3;
    extern __shared__ __align__(16) unsigned char smem[];

    const SubInfo si = P.subs[blockIdx.x];
    const ShapeInfo sh = P.shapes[si.shape];
    const int bx = sh.bx, by = sh.by, bz = sh.bz;
    const int D = by + bz - 1, S = bx + D - 1;
    const int PX = bx, PXY = sh.pxy;
    const int nx = P.nx, nxy = P.nx * P.ny;
    const long long g0 = si.e0x + (long long)nx * (si.e0y + (long long)P.ny * si.e0z);

    // shared memory: [Y: ycap, zero cell, pad][level starts: lcap][lb: lcap][diagonals: dcap][ring]
    Acc *Y = reinterpret_cast<Acc *>(smem);
    int *lvl_s = reinterpret_cast<int *>(smem + (((size_t)(P.ycap + 4) * sizeof(Acc) + 15) & ~(size_t)15));
    int *lb = lvl_s + P.lcap;
    DiagInfo *dg = reinterpret_cast<DiagInfo *>(lb + P.lcap);
    unsigned char *ring = reinterpret_cast<unsigned char *>(dg + ((D + 1) & ~1));
    const int rcap = ((P.chunk_cells * RB + 32) + 15) & ~15;

    const int *chunk_lev = P.chunk + sh.chunk_off;
    const int nchunk = sh.nchunk, nstage = 2 * nchunk;
    for (int t = threadIdx.x; t <= S; t += blockDim.x) lvl_s[t] = P.lvl[sh.lvl_off + t];
    for (int t = threadIdx.x; t < D; t += blockDim.x) dg[t] = P.diag[sh.diag_off + t];

    // stage t < nchunk: forward chunk t; t >= nchunk: backward chunk 2 nchunk - 1 - t
    auto issue = [&](int t) {
        if (t < nstage) {
            const bool fw = t < nchunk;
            const int c = fw ? t : nstage - 1 - t;
            const int qa = P.lvl[sh.lvl_off + chunk_lev[c]], qb = P.lvl[sh.lvl_off + chunk_lev[c + 1]];
            stage_bytes(ring + (size_t)(t % NBUF) * rcap, fw ? P.fwd : P.bwd,
                        (si.foff + qa) * (long long)RB, (si.foff + qb) * (long long)RB);
        }
        cp_async_commit();
    };
#pragma unroll
    for (int t = 0; t < NBUF - 1; ++t) issue(t);

    // gather R_i^delta r into the padded box vector (GB loads in flight per thread)
    {
        constexpr int GB = 8;
        const double *rg = P.r + g0;
        const unsigned mbx = magic_div(bx), mby = magic_div(by);
        const int ncell = sh.ncell;
        for (int q0 = threadIdx.x; q0 < ncell; q0 += GB * blockDim.x) {
            double v[GB];
            int yo[GB];
#pragma unroll
            for (int m = 0; m < GB; ++m) {
                const int q = q0 + m * (int)blockDim.x;
                if (q < ncell) {
                    const int row = fast_div(q, bx, mbx), k = fast_div(row, by, mby);
                    const int i = q - row * bx, j = row - k * by;
                    v[m] = __ldg(rg + i + (long long)nx * j + (long long)nxy * k);
                    yo[m] = i + PX * j + PXY * k;
                }
            }
#pragma unroll
            for (int m = 0; m < GB; ++m) {
                const int q = q0 + m * (int)blockDim.x;
                if (q < ncell) Y[yo[m]] = (Acc)v[m];
            }
        }
    }
    __syncthreads();
    for (int l = threadIdx.x; l < S; l += blockDim.x) lb[l] = lvl_s[l] - dg[max(0, l - bx + 1)].base;

    // this thread's pencil: number p = threadIdx.x in (d, j) order
    const int p = threadIdx.x;
    const bool live = p < by * bz;
    int d = 0, j = 0, k = 0;
    if (live) {
        while (d + 1 < D && dg[d + 1].base <= p) ++d;
        j = (dg[d].jmin_cnt & 0xffff) + (p - dg[d].base);
        k = d - j;
    }
    // -y / -z (forward) and +y / +z (backward) neighbour rows of the pencil; a
    // neighbour outside the box reads the zero cell Y[ycap] (stride 0 along i)
    Acc *Yz = Y + P.ycap;
    const int n0 = PX * j + PXY * k;                       // Y index of cell i = 0
    Acc *const my = j > 0 ? Y + n0 - PX : Yz, *const mz = k > 0 ? Y + n0 - PXY : Yz;
    Acc *const py = j < by - 1 ? Y + n0 + PX : Yz, *const pz = k < bz - 1 ? Y + n0 + PXY : Yz;
    const int smy = j > 0, smz = k > 0, spy = j < by - 1, spz = k < bz - 1;
    Acc *const yp = Y + n0;
    double *zp0 = P.z + g0 + ((long long)nx * j + (long long)nxy * k);
    const bool own_jk = live && j >= si.oy0 && j < si.oy1 && k >= si.oz0 && k < si.oz1;
    const unsigned owx = (unsigned)(si.ox1 - si.ox0);
    const bool acc = P.accumulate != 0;
    if (threadIdx.x == 0) *Yz = (Acc)0;

    int t = -1, lev_lo = 0, lev_hi = -1;   // current ring stage and its level range
    const unsigned char *rp = ring;         // this pencil's record base in the current stage
    // a new ring stage: wait for its chunk, refill the slot two stages back
    auto next_stage = [&]() {
        ++t;
        cp_async_wait<NBUF - 2>();
        __syncthreads();
        issue(t + NBUF - 1);
        const int c = t < nchunk ? t : nstage - 1 - t;
        lev_lo = chunk_lev[c];
        lev_hi = chunk_lev[c + 1] - 1;
        const int qa = lvl_s[lev_lo];
        rp = ring + ((long long)(t % NBUF) * rcap + (((si.foff + qa) * (long long)RB) & 15) +
                     (long long)RB * (p - qa));
    };
    // forward sweep: w_n = (r_n - a_z w_{n-bxy} - a_y w_{n-bx} - a_x w_{n-1}) / d_n
    {
        Acc xprev = (Acc)0;
        Acc ax = 0, ay = 0, az = 0, dinv = 0;
        bool have = false;                   // the record of the coming level is in registers
        for (int lev = 0; lev < S; ++lev) {
            if (lev > lev_hi) { next_stage(); have = false; }
            const int i = lev - d;
            const bool on = live && (unsigned)i < (unsigned)bx;
            if (on) {
                if (!have) load_rec<Acc, R>(rp + (long long)RB * lb[lev], ax, ay, az, dinv);
                const Acc yz = mz[i * smz], yy = my[i * smy];
                Acc s = yp[i];
                s = fmsub(az, yz, s);
                s = fmsub(ay, yy, s);
                s = fmsub(ax, xprev, s);
                const Acc y = s * dinv;
                yp[i] = y;
                xprev = y;
            }
            // the next level's record (independent of this level's values), if staged
            have = false;
            if (lev + 1 <= lev_hi && live && (unsigned)(i + 1) < (unsigned)bx) {
                load_rec<Acc, R>(rp + (long long)RB * lb[lev + 1], ax, ay, az, dinv);
                have = true;
            }
            __syncthreads();   // level done: its values are the next level's neighbours
        }
    }
    // backward sweep: z_n = w_n - d_n^{-1} (a_x z_{n+1} + a_y z_{n+bx} + a_z z_{n+bxy})
    {
        Acc xprev = (Acc)0;
        Acc ax = 0, ay = 0, az = 0, dinv = 0;
        bool have = false;
        next_stage();
        for (int lev = S - 1; lev >= 0; --lev) {
            if (lev < lev_lo) { next_stage(); have = false; }
            const int i = lev - d;
            const bool on = live && (unsigned)i < (unsigned)bx;
            if (on) {
                if (!have) load_rec<Acc, R>(rp + (long long)RB * lb[lev], ax, ay, az, dinv);
                const Acc zy = py[i * spy], zz = pz[i * spz];
                Acc s = ax * xprev;
                s = fmadd(ay, zy, s);
                s = fmadd(az, zz, s);
                const Acc y = fmsub(dinv, s, yp[i]);
                yp[i] = y;
                xprev = y;
                if (own_jk && (unsigned)(i - si.ox0) < owx) {
                    if (acc) atomicAdd(zp0 + i, (double)y);   // one owner per cell
                    else zp0[i] = (double)y;
                }
            }
            have = false;
            if (lev - 1 >= lev_lo && live && (unsigned)(i - 1) < (unsigned)bx) {
                load_rec<Acc, R>(rp + (long long)RB * lb[lev - 1], ax, ay, az, dinv);
                have = true;
            }
            __syncthreads();
        }
    }
    cp_async_wait<0>();
}

// z (+)= sum over the overlapped boxes covering each cell of their solution
// ((R_i^delta)^T), boxes in ascending index order (deterministic)
struct SumParams {
    const SubInfo *subs;
    const ShapeInfo *shapes;
    const int *clo[3], *chi[3];   // per axis and coordinate: parts whose boxes cover it
    int parts[3];
    int nx, ny, nz;
    const double *zbuf;
    double *z;
    int accumulate;
};

__global__ void __launch_bounds__(256) k_ras_sum(SumParams P) {
    const long long N = (long long)P.nx * P.ny * P.nz;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const int c[3] = {(int)(n % P.nx), (int)((n / P.nx) % P.ny), (int)(n / ((long long)P.nx * P.ny))};
        double acc = 0.0;
        for (int pz = P.clo[2][c[2]]; pz <= P.chi[2][c[2]]; ++pz) {
            for (int py = P.clo[1][c[1]]; py <= P.chi[1][c[1]]; ++py) {
                for (int px = P.clo[0][c[0]]; px <= P.chi[0][c[0]]; ++px) {
                    const SubInfo si = P.subs[px + P.parts[0] * (py + P.parts[1] * pz)];
                    const ShapeInfo &sh = P.shapes[si.shape];
                    const int q = (c[0] - si.e0x) + sh.bx * ((c[1] - si.e0y) + sh.by * (c[2] - si.e0z));
                    acc += P.zbuf[si.foff + q];
                }
            }
        }
        P.z[n] = P.accumulate ? P.z[n] + acc : acc;
    }
}


// ILU(0) of A_i in natural order: only the diagonal changes,
// d_n = a_nn - sum_{m<n neighbour} (a_nm / d_m) a_mn   (m: -z, -y, -x).
// One CTA per box (box `box` of the handle described by P).
template <int PREC>
__device__ __forceinline__ void ras_factor_box(const FactorParams &P, int box) {
    extern __shared__ __align__(16) unsigned char smem[];
    double *D = reinterpret_cast<double *>(smem);
    const SubInfo si = P.subs[box];
    const ShapeInfo sh = P.shapes[si.shape];
    const int *lvl = P.lvl + sh.lvl_off;
    const unsigned *cells = P.cells + sh.cell_off;
    const int bx = sh.bx, by = sh.by, bxy = bx * by;
    const int nx = P.nx, nxy = P.nx * P.ny;
    const long long g0 = si.e0x + (long long)nx * (si.e0y + (long long)P.ny * si.e0z);
    const double *Ac = P.A.c[0], *Amx = P.A.c[1], *Apx = P.A.c[2], *Amy = P.A.c[3],
                 *Apy = P.A.c[4], *Amz = P.A.c[5], *Apz = P.A.c[6];
    for (int l = 0; l < sh.nlev; ++l) {
        const int q1 = lvl[l + 1];
        for (int q = lvl[l] + threadIdx.x; q < q1; q += blockDim.x) {
            const unsigned e = cells[q];
            const int i = e & 255u, j = (e >> 8) & 255u, k = (e >> 16) & 255u;
            const unsigned fl = e >> 24;
            const int n = i + bx * j + bxy * k;
            const long long g = g0 + i + (long long)nx * j + (long long)nxy * k;
            double d = Ac[g];
            if (fl & F_MZ) { const double lm = Amz[g] / D[n - bxy]; d -= lm * Apz[g - nxy]; }
            if (fl & F_MY) { const double lm = Amy[g] / D[n - bx]; d -= lm * Apy[g - nx]; }
            if (fl & F_MX) { const double lm = Amx[g] / D[n - 1]; d -= lm * Apx[g - 1]; }
            if (!(d != 0.0) || !isfinite(d)) atomicExch(P.err, 1);
            D[n] = d;
        }
        __syncthreads();
    }
    for (int q = threadIdx.x; q < sh.ncell; q += blockDim.x) {
        const unsigned e = cells[q];
        const int i = e & 255u, j = (e >> 8) & 255u, k = (e >> 16) & 255u;
        const unsigned fl = e >> 24;
        const int n = i + bx * j + bxy * k;
        const long long g = g0 + i + (long long)nx * j + (long long)nxy * k;
        const double dinv = 1.0 / D[n];
        store_rec<PREC>(P.fwd, si.foff + q, (fl & F_MX) ? Amx[g] : 0.0, (fl & F_MY) ? Amy[g] : 0.0,
                        (fl & F_MZ) ? Amz[g] : 0.0, dinv);
        store_rec<PREC>(P.bwd, si.foff + q, (fl & F_PX) ? Apx[g] : 0.0, (fl & F_PY) ? Apy[g] : 0.0,
                        (fl & F_PZ) ? Apz[g] : 0.0, dinv);
    }
}

template <int PREC>
__global__ void __launch_bounds__(512) k_ras_factor(FactorParams P) {
    ras_factor_box<PREC>(P, blockIdx.x);
}

// The subdomain ILU(0) factorisations of several handles in one launch: CTA b
// factors box box_local[b] of handle box_inst[b] (CTAs of inactive handles return).
template <int PREC>
__global__ void __launch_bounds__(512) k_ras_factor_batch(const FactorParams *__restrict__ inst,
                                                          const int *__restrict__ box_inst,
                                                          const int *__restrict__ box_local,
                                                          const unsigned char *__restrict__ active) {
    const int h = box_inst[blockIdx.x];
    if (!active[h]) return;
    ras_factor_box<PREC>(inst[h], box_local[blockIdx.x]);
}

// ---------------------------------------------------------------------------
// host set-up
// ---------------------------------------------------------------------------

static std::vector<int> split_axis(int n, int parts) {
    std::vector<int> s(parts + 1);
    const int q = n / parts, r = n % parts;
    for (int p = 0; p <= parts; ++p) s[p] = p * q + std::min(p, r);
    return s;
}

// The opt-in limit is raised to the per-CTA maximum once: a later set-up with
// a smaller need must not lower it under a handle that needs more.
constexpr int SMEM_OPTIN = 227 * 1024;
template <int PREC, int NBUF>
static int set_apply_attr(size_t) {
    RAS_CK(cudaFuncSetAttribute(k_ras_apply<PREC, NBUF>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_OPTIN));
    cudaFuncAttributes fa{};   // the persistent batch kernel has a little static shared memory
    RAS_CK(cudaFuncGetAttributes(&fa, k_ras_apply_batch<PREC, NBUF>));
    RAS_CK(cudaFuncSetAttribute(k_ras_apply_batch<PREC, NBUF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                SMEM_OPTIN - (int)fa.sharedSizeBytes));
    return RAS_OK;
}
template <int PREC>
static int set_pipe_attr() {
    RAS_CK(cudaFuncSetAttribute(k_ras_pipe<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_OPTIN));
    return RAS_OK;
}
template <int PREC>
static int set_factor_attr(size_t) {
    RAS_CK(cudaFuncSetAttribute(k_ras_factor<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                SMEM_OPTIN));
    RAS_CK(cudaFuncSetAttribute(k_ras_factor_batch<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                SMEM_OPTIN));
    return RAS_OK;
}

// shared memory of the pipelined solves for the handle's current chunk size
static size_t pipe_smem(Ras1 &R) {
    const size_t acc = R.prec == 64 ? 8 : 4;
    const size_t ybytes = (((size_t)(R.ycap_pipe + 4) * acc) + 15) & ~(size_t)15;
    const size_t rcap = ((R.chunk_cells * R.rec_bytes + 32) + 15) & ~15;
    R.smem_pipe = ybytes + 2 * (size_t)R.lcap * sizeof(int) + (size_t)R.dcap_pipe * sizeof(DiagInfo) +
                  3 * rcap;
    return R.smem_pipe;
}

// Level schedule of the subdomain solves: chunks of consecutive levels with at most
// chunk_cells cells (staged into the shared-memory ring together) and threads per
// box. 0 takes the default (chunk 1024 cells, 384 in FP64; threads: the widest
// level rounded up to a warp), or the RAS_APPLY_CHUNK / RAS_APPLY_THREADS tuning
// knobs. Fills the shapes' chunk offsets, chunk_tab, block and smem_apply.
static int schedule_tables(Ras1 &R, int chunk_cells, int threads, std::vector<int> &chunk_tab) {
    int base_chunk = R.prec == 64 ? 384 : 1024;
    if (const char *e = getenv("RAS_APPLY_CHUNK")) {     // tuning knob
        const int v = atoi(e);
        if (v >= 64 && v <= 8192) base_chunk = v;
    }
    if (chunk_cells > 0) base_chunk = chunk_cells;
    const int cc = std::max(base_chunk, R.maxw);
    int block = std::min(512, std::max(64, ((R.maxw + 31) / 32) * 32));
    if (const char *e = getenv("RAS_APPLY_THREADS")) {   // tuning knob
        const int v = atoi(e);
        if (v >= 32 && v <= 512 && v % 32 == 0) block = v;
    }
    if (threads > 0) {
        if (threads > 512 || threads % 32) return RAS_EINVAL;
        block = threads;
    }
    const size_t acc = R.prec == 64 ? 8 : 4;
    const size_t rcap = ((cc * R.rec_bytes + 32) + 15) & ~15;
    const size_t ccap = ((cc * 4 + 32) + 15) & ~15;
    const size_t smem = (R.ycap + 2 * (size_t)R.gcap) * acc + R.lcap * sizeof(int) + R.nbuf * (rcap + ccap);
    if (smem > 227 * 1024) return RAS_EINVAL;
    chunk_tab.clear();
    for (auto &sh : R.shapes) {
        sh.chunk_off = (int)chunk_tab.size();
        const int *lv = &R.h_lvl[sh.lvl_off];
        int l = 0;
        chunk_tab.push_back(0);
        int nch = 0;
        while (l < sh.nlev) {
            int l1 = l + 1;
            while (l1 < sh.nlev && lv[l1 + 1] - lv[l] <= cc) ++l1;
            chunk_tab.push_back(l1);
            ++nch;
            l = l1;
        }
        sh.nchunk = nch;
    }
    R.chunk_cells = cc;
    R.block = block;
    R.smem_apply = smem;
    return RAS_OK;
}

int ras1_set_schedule(Ras1 &R, int chunk_cells, int threads) {
    if (chunk_cells < 0 || threads < 0) return RAS_EINVAL;
    Ras1 T = R;                 // the tables only change if the new schedule is valid
    std::vector<int> chunk_tab;
    RAS_TRY(schedule_tables(T, chunk_cells, threads, chunk_tab));
    int *d = nullptr;
    RAS_TRY(dalloc(&d, chunk_tab.size()));
    if (cudaMemcpy(d, chunk_tab.data(), chunk_tab.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(R.d_shapes, T.shapes.data(), T.shapes.size() * sizeof(ShapeInfo), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        dfree(d);
        return RAS_ECUDA;
    }
    dfree(R.d_chunk);
    R.d_chunk = d;
    R.shapes = T.shapes;
    R.chunk_cells = T.chunk_cells;
    R.block = T.block;
    R.smem_apply = T.smem_apply;
    if (R.pipe_ok && pipe_smem(R) > 227 * 1024) R.pipe = R.pipe_ok = 0;
    return RAS_OK;
}

int ras1_setup(Ras1 &R, int nx, int ny, int nz, int px, int py, int pz, int overlap, int prec,
               int kind) {
    if (px < 1 || py < 1 || pz < 1 || overlap < 0) return RAS_EINVAL;
    if (kind < 0 || kind > 2) return RAS_EINVAL;
    R.kind = kind;
    if (px > nx || py > ny || pz > nz) return RAS_EINVAL;
    if (prec != 64 && prec != 32 && prec != 16) return RAS_EINVAL;
    R.nx = nx; R.ny = ny; R.nz = nz; R.N = nx * ny * nz;
    R.prec = prec;
    R.rec_bytes = prec == 64 ? 32 : (prec == 32 ? 16 : 8);
    const int dims[3] = {nx, ny, nz};
    const int parts[3] = {px, py, pz};
    std::vector<int> cuts[3];
    for (int a = 0; a < 3; ++a) cuts[a] = split_axis(dims[a], parts[a]);

    std::map<std::tuple<int, int, int>, int> shape_id;
    std::vector<int> lvl_tab;
    std::vector<unsigned> cell_tab;
    std::vector<int> cidx_tab;        // same positions as cell_tab: i + bx (j + by k)
    std::vector<DiagInfo> diag_tab;
    R.subs.clear();
    R.shapes.clear();
    long long foff = 0;
    int maxw_all = 0, ycap = 0, lcap = 0, gcap = 0;
    for (int kz = 0; kz < pz; ++kz)
        for (int jy = 0; jy < py; ++jy)
            for (int ix = 0; ix < px; ++ix) {
                const int p[3] = {ix, jy, kz};
                int o0[3], o1[3], e0[3], e1[3];
                for (int a = 0; a < 3; ++a) {
                    o0[a] = cuts[a][p[a]];
                    o1[a] = cuts[a][p[a] + 1];
                    e0[a] = dims[a] > 1 ? std::max(o0[a] - overlap, 0) : 0;
                    e1[a] = dims[a] > 1 ? std::min(o1[a] + overlap, dims[a]) : 1;
                }
                const int bx = e1[0] - e0[0], by = e1[1] - e0[1], bz = e1[2] - e0[2];
                if (bx > 256 || by > 256 || bz > 256) return RAS_EINVAL;
                const int ncell = bx * by * bz;
                if (ncell > 16384) return RAS_EINVAL;  // shared-memory pivots in the factor
                auto key = std::make_tuple(bx, by, bz);
                auto it = shape_id.find(key);
                int sid = it == shape_id.end() ? -1 : it->second;
                if (sid < 0) {
                    sid = (int)R.shapes.size();
                    shape_id[key] = sid;
                    ShapeInfo sh{};
                    sh.bx = bx; sh.by = by; sh.bz = bz; sh.ncell = ncell;
                    sh.nlev = bx + by + bz - 2;
                    // level schedule: cells ordered by (i + j + k, natural index)
                    std::vector<std::vector<unsigned>> levels(sh.nlev);
                    for (int k = 0; k < bz; ++k)
                        for (int j = 0; j < by; ++j)
                            for (int i = 0; i < bx; ++i) {
                                unsigned fl = 0;
                                if (i > 0) fl |= F_MX;
                                if (j > 0) fl |= F_MY;
                                if (k > 0) fl |= F_MZ;
                                if (i < bx - 1) fl |= F_PX;
                                if (j < by - 1) fl |= F_PY;
                                if (k < bz - 1) fl |= F_PZ;
                                levels[i + j + k].push_back((unsigned)i | ((unsigned)j << 8) |
                                                            ((unsigned)k << 16) | (fl << 24));
                            }
                    // inside a level, cells grouped by x-pencil anti-diagonal d = j + k,
                    // then by j (the pipelined solves read a diagonal's cells contiguously;
                    // the cells of a level are independent, so the order is free)
                    for (auto &L : levels)
                        std::sort(L.begin(), L.end(), [&](unsigned a, unsigned b) {
                            auto key = [&](unsigned e) {
                                const int j = (int)((e >> 8) & 255u), k = (int)((e >> 16) & 255u);
                                return (j + k) * 256 + j;
                            };
                            return key(a) < key(b);
                        });
                    while (cell_tab.size() % 4) { cell_tab.push_back(0); cidx_tab.push_back(0); }
                    sh.cell_off = (int)cell_tab.size();
                    sh.lvl_off = (int)lvl_tab.size();
                    int pos = 0, maxw = 0;
                    for (auto &L : levels) {
                        lvl_tab.push_back(pos);
                        for (unsigned e : L) {
                            cell_tab.push_back(e);
                            cidx_tab.push_back((int)(e & 255u) + bx * ((int)((e >> 8) & 255u) +
                                                                       by * (int)((e >> 16) & 255u)));
                        }
                        pos += (int)L.size();
                        maxw = std::max(maxw, (int)L.size());
                    }
                    lvl_tab.push_back(pos);
                    sh.maxw = maxw;
                    // x-pencil anti-diagonals d = j + k for the pipelined layout
                    sh.diag_off = (int)diag_tab.size();
                    int dbase = 0;
                    for (int d = 0; d < by + bz - 1; ++d) {
                        const int jmin = std::max(0, d - (bz - 1)), jmax = std::min(d, by - 1);
                        const int cnt = jmax - jmin + 1;
                        diag_tab.push_back(DiagInfo{jmin | (cnt << 16), dbase});
                        dbase += cnt;
                    }
                    sh.pxy = bx * by + (((bx * (by - 1)) % 2 == 0) ? 1 : 0);
                    maxw_all = std::max(maxw_all, maxw);
                    ycap = std::max(ycap, ncell);
                    gcap = std::max(gcap, bx * by);
                    lcap = std::max(lcap, sh.nlev + 1);
                    R.shapes.push_back(sh);
                    sid = (int)R.shapes.size() - 1;
                }
                SubInfo si{};
                si.e0x = e0[0]; si.e0y = e0[1]; si.e0z = e0[2];
                si.shape = sid;
                si.ox0 = o0[0] - e0[0]; si.oy0 = o0[1] - e0[1]; si.oz0 = o0[2] - e0[2];
                si.ox1 = o1[0] - e0[0]; si.oy1 = o1[1] - e0[1]; si.oz1 = o1[2] - e0[2];
                si.foff = foff;
                foff += (ncell + 3) & ~3;
                R.ncell_total += ncell;
                R.nown += (long long)(o1[0] - o0[0]) * (o1[1] - o0[1]) * (o1[2] - o0[2]);
                R.subs.push_back(si);
            }
    R.nsub = (int)R.subs.size();
    R.nshape = (int)R.shapes.size();
    // every overlapped box must lie inside the grid and match its shape
    for (const SubInfo &si : R.subs) {
        if (si.shape < 0 || si.shape >= R.nshape) return RAS_EINVAL;
        const ShapeInfo &sh = R.shapes[si.shape];
        if (si.e0x < 0 || si.e0y < 0 || si.e0z < 0 || si.e0x + sh.bx > nx ||
            si.e0y + sh.by > ny || si.e0z + sh.bz > nz)
            return RAS_EINVAL;
        if (si.ox0 < 0 || si.oy0 < 0 || si.oz0 < 0 || si.ox1 > sh.bx || si.oy1 > sh.by ||
            si.oz1 > sh.bz)
            return RAS_EINVAL;
    }
    R.nrec = foff;
    R.ycap = (ycap + 3) & ~3;
    R.gcap = (gcap + 3) & ~3;
    R.lcap = (lcap + 3) & ~3;
    R.maxw = maxw_all;
    R.h_lvl = lvl_tab;
    std::vector<int> chunk_tab;
    RAS_TRY(schedule_tables(R, 0, 0, chunk_tab));
    R.smem_factor = (size_t)R.ycap * sizeof(double);
    if (R.smem_apply > 227 * 1024 || R.smem_factor > 227 * 1024) return RAS_EINVAL;
    // pencil-wavefront subdomain solves: left-RAS with FP32 / BF16 factors, at most
    // 1024 x-pencils per box (one thread each)
    {
        bool ok = kind == 1 && prec != 64;
        int pens = 1, ycp = 0, dmax = 1;
        for (const ShapeInfo &sh : R.shapes) {
            pens = std::max(pens, sh.by * sh.bz);
            ycp = std::max(ycp, sh.pxy * sh.bz);
            dmax = std::max(dmax, sh.by + sh.bz - 1);
        }
        if (pens > 1024) ok = false;
        R.pipe_warps = (pens + 31) / 32;
        R.ycap_pipe = (ycp + 3) & ~3;
        R.dcap_pipe = (dmax + 1) & ~1;
        if (pipe_smem(R) > 227 * 1024) ok = false;
        R.pipe_ok = ok ? 1 : 0;
        R.pipe = 0;   // the level-scheduled solves are faster on the measured workloads
    }
    RAS_TRY(dalloc(&R.d_subs, R.subs.size()));
    RAS_TRY(dalloc(&R.d_shapes, R.shapes.size()));
    RAS_TRY(dalloc(&R.d_lvl, lvl_tab.size()));
    RAS_TRY(dalloc(&R.d_chunk, chunk_tab.size()));
    RAS_TRY(dalloc(&R.d_cells, cell_tab.size() + 16));
    RAS_TRY(dalloc(&R.d_cidx, cidx_tab.size() + 16));
    RAS_TRY(dalloc(&R.d_err, 1));
    RAS_TRY(dalloc(&R.d_diag, diag_tab.size()));
    RAS_CK(cudaMemcpy(R.d_diag, diag_tab.data(), diag_tab.size() * sizeof(DiagInfo), cudaMemcpyHostToDevice));
    unsigned char *fw = nullptr, *bw = nullptr;
    RAS_TRY(dalloc(&fw, (size_t)R.nrec * R.rec_bytes + 64));
    RAS_TRY(dalloc(&bw, (size_t)R.nrec * R.rec_bytes + 64));
    R.d_fwd = fw; R.d_bwd = bw;
    RAS_CK(cudaMemcpy(R.d_subs, R.subs.data(), R.subs.size() * sizeof(SubInfo), cudaMemcpyHostToDevice));
    RAS_CK(cudaMemcpy(R.d_shapes, R.shapes.data(), R.shapes.size() * sizeof(ShapeInfo),
                      cudaMemcpyHostToDevice));
    RAS_CK(cudaMemcpy(R.d_lvl, lvl_tab.data(), lvl_tab.size() * sizeof(int), cudaMemcpyHostToDevice));
    RAS_CK(cudaMemcpy(R.d_chunk, chunk_tab.data(), chunk_tab.size() * sizeof(int),
                      cudaMemcpyHostToDevice));
    RAS_CK(cudaMemset(R.d_cells, 0, (cell_tab.size() + 16) * sizeof(unsigned)));
    RAS_CK(cudaMemset(R.d_cidx, 0, (cidx_tab.size() + 16) * sizeof(int)));
    RAS_CK(cudaMemcpy(R.d_cidx, cidx_tab.data(), cidx_tab.size() * sizeof(int), cudaMemcpyHostToDevice));
    RAS_CK(cudaMemcpy(R.d_cells, cell_tab.data(), cell_tab.size() * sizeof(unsigned),
                      cudaMemcpyHostToDevice));
    RAS_CK(cudaMemset(R.d_err, 0, sizeof(int)));
    RAS_CK(cudaMemset(R.d_fwd, 0, (size_t)R.nrec * R.rec_bytes + 64));
    RAS_CK(cudaMemset(R.d_bwd, 0, (size_t)R.nrec * R.rec_bytes + 64));
    if (prec == 64) { RAS_TRY(set_apply_attr<64, 3>(R.smem_apply)); RAS_TRY(set_factor_attr<64>(R.smem_factor)); }
    if (prec == 32) { RAS_TRY(set_apply_attr<32, 3>(R.smem_apply)); RAS_TRY(set_factor_attr<32>(R.smem_factor)); RAS_TRY(set_pipe_attr<32>()); }
    if (prec == 16) { RAS_TRY(set_apply_attr<16, 3>(R.smem_apply)); RAS_TRY(set_factor_attr<16>(R.smem_factor)); RAS_TRY(set_pipe_attr<16>()); }
    if (kind != 1) {
        // per axis and coordinate, the (contiguous) range of parts whose overlapped
        // boxes cover it; box solutions are kept per record offset
        R.parts[0] = px; R.parts[1] = py; R.parts[2] = pz;
        for (int a = 0; a < 3; ++a) {
            std::vector<int> lo(dims[a], parts[a]), hi(dims[a], -1);
            for (int q = 0; q < parts[a]; ++q) {
                const int e0 = std::max(cuts[a][q] - overlap, 0);
                const int e1 = std::min(cuts[a][q + 1] + overlap, dims[a]);
                for (int i = e0; i < e1; ++i) { lo[i] = std::min(lo[i], q); hi[i] = std::max(hi[i], q); }
            }
            RAS_TRY(dalloc(&R.d_clo[a], lo.size()));
            RAS_TRY(dalloc(&R.d_chi[a], hi.size()));
            RAS_CK(cudaMemcpy(R.d_clo[a], lo.data(), lo.size() * sizeof(int), cudaMemcpyHostToDevice));
            RAS_CK(cudaMemcpy(R.d_chi[a], hi.data(), hi.size() * sizeof(int), cudaMemcpyHostToDevice));
        }
        RAS_TRY(dalloc(&R.zbuf, (size_t)R.nrec));
        RAS_CK(cudaMemset(R.zbuf, 0, (size_t)R.nrec * sizeof(double)));
    }
    return RAS_OK;
}

void ras1_free(Ras1 &R) {
    dfree(R.d_subs); dfree(R.d_shapes); dfree(R.d_lvl); dfree(R.d_chunk); dfree(R.d_cells);
    dfree(R.d_cidx); dfree(R.d_err); dfree(R.d_diag);
    if (R.d_fwd) cudaFree(R.d_fwd);
    if (R.d_bwd) cudaFree(R.d_bwd);
    R.d_fwd = R.d_bwd = nullptr;
    dfree(R.zbuf);
    for (int a = 0; a < 3; ++a) { dfree(R.d_clo[a]); dfree(R.d_chi[a]); }
}

int ras1_factor(Ras1 &R, const Stencil7 &A, cudaStream_t st) {
    FactorParams P;
    P.subs = R.d_subs; P.shapes = R.d_shapes; P.lvl = R.d_lvl; P.cells = R.d_cells;
    P.A = A; P.fwd = R.d_fwd; P.bwd = R.d_bwd;
    P.nx = R.nx; P.ny = R.ny; P.nz = R.nz; P.err = R.d_err;
    const int block = std::min(R.block, 256);
    if (R.prec == 64) k_ras_factor<64><<<R.nsub, block, R.smem_factor, st>>>(P);
    else if (R.prec == 32) k_ras_factor<32><<<R.nsub, block, R.smem_factor, st>>>(P);
    else k_ras_factor<16><<<R.nsub, block, R.smem_factor, st>>>(P);
    RAS_LAUNCHED();
    return RAS_OK;
}

void ras1_factor_params(const Ras1 &R, const Stencil7 &A, FactorParams &P) {
    P.subs = R.d_subs; P.shapes = R.d_shapes; P.lvl = R.d_lvl; P.cells = R.d_cells;
    P.A = A; P.fwd = R.d_fwd; P.bwd = R.d_bwd;
    P.nx = R.nx; P.ny = R.ny; P.nz = R.nz; P.err = R.d_err;
}

int ras1_factor_batch(const FactorParams *d_inst, const int *d_box_inst, const int *d_box_local,
                      const unsigned char *d_active, int nbox, int prec, int block, size_t smem, cudaStream_t st) {
    if (nbox <= 0) return RAS_OK;
    if (prec == 64) k_ras_factor_batch<64><<<nbox, block, smem, st>>>(d_inst, d_box_inst, d_box_local, d_active);
    else if (prec == 32) k_ras_factor_batch<32><<<nbox, block, smem, st>>>(d_inst, d_box_inst, d_box_local, d_active);
    else k_ras_factor_batch<16><<<nbox, block, smem, st>>>(d_inst, d_box_inst, d_box_local, d_active);
    RAS_LAUNCHED();
    return RAS_OK;
}

int ras1_check(Ras1 &R, cudaStream_t st) {
    int h = 0;
    RAS_CK(cudaMemcpyAsync(&h, R.d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    RAS_CK(cudaStreamSynchronize(st));
    if (h) {
        RAS_CK(cudaMemsetAsync(R.d_err, 0, sizeof(int), st));
        return RAS_EZEROPIVOT;
    }
    return RAS_OK;
}

int ras1_set_kernel(Ras1 &R, int kernel) {
    if (kernel != 0 && kernel != 1) return RAS_EINVAL;
    if (kernel == 1 && !R.pipe_ok) return RAS_EINVAL;
    R.pipe = kernel;
    return RAS_OK;
}


void ras1_apply_params(const Ras1 &R, ApplyParams &P) {
    P = ApplyParams{};
    P.subs = R.d_subs; P.shapes = R.d_shapes; P.lvl = R.d_lvl; P.chunk = R.d_chunk;
    P.cidx = R.d_cidx;
    P.fwd = (const unsigned char *)R.d_fwd; P.bwd = (const unsigned char *)R.d_bwd;
    P.nx = R.nx; P.ny = R.ny; P.nz = R.nz; P.accumulate = 0;
    P.ycap = R.ycap; P.gcap = R.gcap; P.lcap = R.lcap; P.nbuf = R.nbuf; P.chunk_cells = R.chunk_cells;
    P.kind = R.kind; P.zbuf = R.zbuf;
}

int ras1_apply_batch(const BatchApply &B, int grid, int prec, int block, size_t smem, cudaStream_t st) {
    if (grid <= 0 || B.nitems <= 0) return RAS_OK;
    RAS_CK(cudaMemsetAsync(B.qcount, 0, sizeof(int), st));
    if (prec == 64) k_ras_apply_batch<64, 3><<<grid, block, smem, st>>>(B);
    else if (prec == 32) k_ras_apply_batch<32, 3><<<grid, block, smem, st>>>(B);
    else k_ras_apply_batch<16, 3><<<grid, block, smem, st>>>(B);
    RAS_LAUNCHED();
    return RAS_OK;
}

int ras1_batch_grid(int prec, int block, size_t smem, int nitems, int *grid) {
    int dev = 0, sms = 0, per = 0;
    RAS_CK(cudaGetDevice(&dev));
    RAS_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (prec == 64) RAS_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ras_apply_batch<64, 3>, block, smem));
    else if (prec == 32) RAS_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ras_apply_batch<32, 3>, block, smem));
    else RAS_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ras_apply_batch<16, 3>, block, smem));
    if (per < 1) return RAS_EINVAL;
    *grid = std::min(nitems, sms * per);
    return RAS_OK;
}

int ras1_apply(Ras1 &R, const double *r, double *z, int accumulate, cudaStream_t st) {
    if (R.pipe) {
        PipeParams Q;
        Q.subs = R.d_subs; Q.shapes = R.d_shapes; Q.diag = R.d_diag;
        Q.lvl = R.d_lvl; Q.chunk = R.d_chunk;
        Q.fwd = (const unsigned char *)R.d_fwd; Q.bwd = (const unsigned char *)R.d_bwd;
        Q.r = r; Q.z = z; Q.nx = R.nx; Q.ny = R.ny; Q.nz = R.nz; Q.accumulate = accumulate;
        Q.ycap = R.ycap_pipe; Q.lcap = R.lcap; Q.chunk_cells = R.chunk_cells;
        const int threads = 32 * R.pipe_warps;
        if (R.prec == 32) k_ras_pipe<32><<<R.nsub, threads, R.smem_pipe, st>>>(Q);
        else k_ras_pipe<16><<<R.nsub, threads, R.smem_pipe, st>>>(Q);
        RAS_LAUNCHED();
        return RAS_OK;
    }
    ApplyParams P;
    P.subs = R.d_subs; P.shapes = R.d_shapes; P.lvl = R.d_lvl; P.chunk = R.d_chunk;
    P.cidx = R.d_cidx;
    P.fwd = (const unsigned char *)R.d_fwd; P.bwd = (const unsigned char *)R.d_bwd;
    P.r = r; P.z = z; P.nx = R.nx; P.ny = R.ny; P.nz = R.nz; P.accumulate = accumulate;
    P.ycap = R.ycap; P.gcap = R.gcap; P.lcap = R.lcap; P.nbuf = R.nbuf; P.chunk_cells = R.chunk_cells;
    P.kind = R.kind; P.zbuf = R.zbuf;
    if (R.prec == 64) k_ras_apply<64, 3><<<R.nsub, R.block, R.smem_apply, st>>>(P);
    else if (R.prec == 32) k_ras_apply<32, 3><<<R.nsub, R.block, R.smem_apply, st>>>(P);
    else k_ras_apply<16, 3><<<R.nsub, R.block, R.smem_apply, st>>>(P);
    RAS_LAUNCHED();
    if (R.kind != 1) {
        SumParams Q;
        Q.subs = R.d_subs; Q.shapes = R.d_shapes;
        for (int a = 0; a < 3; ++a) { Q.clo[a] = R.d_clo[a]; Q.chi[a] = R.d_chi[a]; Q.parts[a] = R.parts[a]; }
        Q.nx = R.nx; Q.ny = R.ny; Q.nz = R.nz;
        Q.zbuf = R.zbuf; Q.z = z; Q.accumulate = accumulate;
        const int grid = (int)std::min<long long>(((long long)R.N + 255) / 256, 152LL * 16);
        k_ras_sum<<<grid, 256, 0, st>>>(Q);
        RAS_LAUNCHED();
    }
    return RAS_OK;
}

// Algorithmic bytes of one apply: the ILU(0) factors once (7 values per
// overlapped cell: 3 lower, 3 upper off-diagonals and the inverse pivot, at the
// storage precision), r read once and z written once in FP64. (The kernel's
// records carry the inverse pivot twice and r is re-read over the overlap;
// those bytes are not counted.)
double ras1_bytes(const Ras1 &R) {
    const double val = R.prec == 64 ? 8.0 : (R.prec == 32 ? 4.0 : 2.0);
    return 7.0 * val * (double)R.ncell_total + 16.0 * (double)R.N;
}

}  // namespace ras
