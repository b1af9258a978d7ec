// Dense FP32 matrix products on the tcgen05 tensor cores of sm_103a.
//
// FP32 accuracy from the TF32 tensor path by splitting every operand into a TF32
// head and an FP32 tail (x = h + l, h = x rounded to TF32): A B ~ Ah Bh + Ah Bl + Al Bh,
// three MMAs per k-step accumulated in FP32 in tensor memory (the dropped Al Bl term
// and the tails' own rounding to TF32 leave errors near FP32 rounding).
//
// One CTA of 128 threads computes a 128 x 128 tile of C: the k dimension is walked
// in chunks of 32; each chunk of A (128 x 32) and of B^T (128 x 32) is split and
// written by the threads into shared memory in the canonical K-major layout without
// swizzle (8-row x 16-byte core matrices, LBO = 128 B between core matrices along k,
// SBO = 1024 B between 8-row groups), two chunks double-buffered; one thread issues
// the MMAs (M = 128, N = 128, K = 8 per instruction: 4 k-steps x 3 terms per chunk)
// and commits them to an mbarrier of the buffer, which the threads wait on (bounded)
// before refilling it. The accumulator (128 lanes x 128 FP32 columns of tensor
// memory) is read back with tcgen05.ld, each warp its 32 lanes (rows).
#include "tc_gemm.cuh"

namespace ras {

namespace {

constexpr int TM = 128, TN = 128, KC = 32;
constexpr int CORE_B = 128;                    // bytes of one 8 x 16-byte core matrix
constexpr int SBO = (KC / 4) * CORE_B;         // 1024: next 8-row group
constexpr int LBO = CORE_B;                    // 128: next 4 k-elements
constexpr int OPB = TM * KC * 4;               // 16 KB: one operand part (A or B^T, head or tail)
constexpr long long POLL_LIMIT = 1LL << 26;    // bounded mbarrier waits

// byte offset of element (row, k) of a 128 x 32 operand part
__device__ __forceinline__ int kmaj_off(int row, int k) {
    return (row >> 3) * SBO + (k >> 2) * LBO + (row & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start, LBO, SBO (>> 4), descriptor version 1,
// base offset 0, relative LBO, no swizzle
__device__ __forceinline__ unsigned long long mat_desc(unsigned addr) {
    unsigned long long d = 0;
    d |= (unsigned long long)((addr & 0x3FFFFu) >> 4);
    d |= (unsigned long long)((LBO >> 4) & 0x3FFF) << 16;
    d |= (unsigned long long)((SBO >> 4) & 0x3FFF) << 32;
    d |= 1ull << 46;
    return d;
}

// instruction descriptor, kind::tf32: D FP32, A and B TF32, both K-major, N, M
constexpr unsigned IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(TN >> 3) << 17) |
                           ((unsigned)(TM >> 4) << 24);

__device__ __forceinline__ float tf32_head(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

// bounded wait for the completion of phase `parity` of an mbarrier; false if it gave up
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, unsigned parity) {
    const unsigned a = smem_u32(b);
    for (long long it = 0; it < POLL_LIMIT; ++it) {
        unsigned ok;
        asm volatile(
            "{\n.reg .pred p;\n"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok) : "r"(a), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void mma_tf32(unsigned dtmem, unsigned long long ad, unsigned long long bd,
                                         unsigned acc) {
    asm volatile(
        "{\n.reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(dtmem), "l"(ad), "l"(bd), "r"(IDESC), "r"(acc) : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned long long *b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(b)) : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 tensor-memory lanes
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float (&v)[32]) {
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
          "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
          "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

struct GemmSmem {
    // [buffer][part]: part 0 A head, 1 A tail, 2 B^T head, 3 B^T tail
    alignas(1024) unsigned char op[2][4][OPB];
    unsigned long long mbar[2];
    unsigned tmem_base;
};

}  // namespace

__global__ void __launch_bounds__(128, 1) k_tc_gemm(const GemmTask *tasks, int m, int n, int k, float alpha,
                                                    float beta, int *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // the dynamic window is aligned up to 1024 bytes inside the allocation
    GemmSmem &sm = *reinterpret_cast<GemmSmem *>(
        smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023));
    const GemmTask tk = tasks[blockIdx.z];
    const int row0 = blockIdx.y * TM, col0 = blockIdx.x * TN;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&sm.tmem_base)), "r"(TN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&sm.mbar[0], 1);
        mbar_init(&sm.mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = sm.tmem_base;

    // this thread's share of a chunk: A rows (tid) x 32 k, B^T rows (tid: a column of B) x 32 k
    const float *Arow = tk.A + (long long)(row0 + tid) * tk.lda;
    const float *Bcol = tk.B + col0 + tid;
    float ra[KC], rb[KC];
    auto load_chunk = [&](int c) {
        const float4 *a4 = reinterpret_cast<const float4 *>(Arow + c * KC);
#pragma unroll
        for (int q = 0; q < KC / 4; ++q) {
            const float4 v = __ldg(a4 + q);
            ra[4 * q] = v.x; ra[4 * q + 1] = v.y; ra[4 * q + 2] = v.z; ra[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int q = 0; q < KC; ++q) rb[q] = __ldg(Bcol + (long long)(c * KC + q) * tk.ldb);
    };
    auto store_chunk = [&](int buf) {
#pragma unroll
        for (int q = 0; q < KC; ++q) {
            const int off = kmaj_off(tid, q);
            const float ah = tf32_head(ra[q]), bh = tf32_head(rb[q]);
            *reinterpret_cast<float *>(sm.op[buf][0] + off) = ah;
            *reinterpret_cast<float *>(sm.op[buf][1] + off) = ra[q] - ah;
            *reinterpret_cast<float *>(sm.op[buf][2] + off) = bh;
            *reinterpret_cast<float *>(sm.op[buf][3] + off) = rb[q] - bh;
        }
    };

    const int nk = k / KC;
    bool ok = true;
    load_chunk(0);
    for (int c = 0; c < nk; ++c) {
        const int buf = c & 1;
        if (c >= 2 && !mbar_wait(&sm.mbar[buf], ((c - 2) >> 1) & 1)) ok = false;   // buffer free
        store_chunk(buf);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned a_h = smem_u32(sm.op[buf][0]), a_l = smem_u32(sm.op[buf][1]);
            const unsigned b_h = smem_u32(sm.op[buf][2]), b_l = smem_u32(sm.op[buf][3]);
#pragma unroll
            for (int s = 0; s < KC / 8; ++s) {
                const unsigned o = s * 2 * LBO;   // k-step of 8: two core matrices along k
                mma_tf32(tmem, mat_desc(a_l + o), mat_desc(b_h + o), (c > 0 || s > 0) ? 1u : 0u);
                mma_tf32(tmem, mat_desc(a_h + o), mat_desc(b_l + o), 1u);
                mma_tf32(tmem, mat_desc(a_h + o), mat_desc(b_h + o), 1u);
            }
            mma_commit(&sm.mbar[buf]);
        }
        if (c + 1 < nk) load_chunk(c + 1);
    }
    // the last commit covers every MMA issued before it
    if (!mbar_wait(&sm.mbar[(nk - 1) & 1], ((nk - 1) >> 1) & 1)) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // epilogue: warp w holds rows 32 w .. 32 w + 31 (one per lane), 128 columns
    const int row = row0 + 32 * warp + lane;
    float *Crow = tk.C + (long long)row * tk.ldc + col0;
#pragma unroll 1
    for (int cb = 0; cb < TN; cb += 32) {
        float v[32];
        tmem_ld32(tmem + ((unsigned)(32 * warp) << 16) + cb, v);
#pragma unroll
        for (int q = 0; q < 32; q += 4) {
            float4 o;
            o.x = alpha * v[q]; o.y = alpha * v[q + 1]; o.z = alpha * v[q + 2]; o.w = alpha * v[q + 3];
            if (beta != 0.0f) {
                const float4 p = *reinterpret_cast<const float4 *>(Crow + cb + q);
                o.x += beta * p.x; o.y += beta * p.y; o.z += beta * p.z; o.w += beta * p.w;
            }
            *reinterpret_cast<float4 *>(Crow + cb + q) = o;
        }
    }
    if (!ok && lane == 0) atomicExch(err, 2);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN) : "memory");
}

static bool aligned16(const void *p) { return ((unsigned long long)p & 15) == 0; }

int tc_gemm_batch(const GemmTask *tasks, int ntask, int m, int n, int k, float alpha, float beta,
                  int *err, cudaStream_t st) {
    if (ntask <= 0 || m <= 0 || n <= 0 || k <= 0) return ntask == 0 ? RAS_OK : RAS_EINVAL;
    if (m % TM || n % TN || k % KC || !tasks || !err) return RAS_EINVAL;
    static bool attr = false;
    const size_t smem = sizeof(GemmSmem) + 1024;
    if (!attr) {
        RAS_CK(cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    const dim3 grid(n / TN, m / TM, ntask);
    k_tc_gemm<<<grid, 128, smem, st>>>(tasks, m, n, k, alpha, beta, err);
    RAS_LAUNCHED();
    return RAS_OK;
}

}  // namespace ras

using namespace ras;

extern "C" int ras_gemm_f32(int m, int n, int k, float alpha, const float *A, int lda, const float *B, int ldb,
                            float beta, float *C, int ldc, void *stream) {
    if (m < 0 || n < 0 || k < 0) return RAS_EINVAL;
    if (m == 0 || n == 0) return RAS_OK;
    if (!A || !B || !C || m % TM || n % TN || k % KC || k == 0) return RAS_EINVAL;
    if (lda < k || ldb < n || ldc < n || lda % 4 || ldb % 4 || ldc % 4) return RAS_EINVAL;
    if (!aligned16(A) || !aligned16(B) || !aligned16(C)) return RAS_EINVAL;
    cudaStream_t st = S(stream);
    GemmTask *d = nullptr;
    int *err = nullptr;
    RAS_TRY(dalloc(&d, 1));
    RAS_TRY(dalloc(&err, 1));
    const GemmTask t{A, B, C, lda, ldb, ldc};
    int rc = RAS_OK;
    if (cudaMemcpyAsync(d, &t, sizeof t, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess)
        rc = RAS_ECUDA;
    if (rc == RAS_OK) rc = tc_gemm_batch(d, 1, m, n, k, alpha, beta, err, st);
    int h = 0;
    if (rc == RAS_OK) {
        if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = RAS_ECUDA;
        else if (h)
            rc = RAS_ETIMEOUT;
    }
    cudaStreamSynchronize(st);
    dfree(d);
    dfree(err);
    return rc;
}
