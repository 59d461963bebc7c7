// m2l_tc.cu -- M2L + L2L (Eq. 2.21) for many right-hand sides on the GB300 tensor cores
// (tcgen05.mma, kind::tf32, accumulators in tensor memory).
//
// For one target box, one domain and a tile of 64 columns (3 Cartesian components x right-hand
// sides), D[:, tile] = T_ll(oct) D[parent][:, tile] + sum_FF T_o C[src][:, tile] is a chain of
// complex (p^2 x p^2) x (p^2 x 64) products.  Written in interleaved real form -- row 2r + a is
// the real (a = 0) or imaginary (a = 1) part of coefficient r, and likewise for K -- each product
// is a real 128 x 128 x 64 GEMM (p <= 8, zero padded):
//   A[2r+a][2k+b] = [[Re T, -Im T], [Im T, Re T]][a][b],  B[2k+b][n] = (Re, Im)[b] C[src][n][k],
// and B column n is exactly the coefficient vector of column n as stored (re, im interleaved), so
// it is K-major without any rearrangement.  The A matrices are precomputed once per (domain,
// level, offset), rounded to TF32 and stored in the canonical no-swizzle K-major core-matrix
// layout (8 rows x 16 bytes per core matrix, K-adjacent core matrices 128 bytes apart, 8-row
// groups 4096 bytes apart), so staging A is a straight 64 KiB copy.
//
// One CTA of 128 threads: all threads stage A and B into one of two shared-memory stages; thread
// 0 issues the 16 MMAs of the product (K = 8 each) and commits them to the stage's mbarrier;
// while the tensor cores work, the threads stage the next product into the other stage.  Waits
// on mbarriers are bounded: on time-out the kernel records an error flag and stops issuing work.
// Finally each warp reads its 32 accumulator lanes with tcgen05.ld and writes the complex result.
#include <algorithm>

#include "fmbem_internal.cuh"

namespace {

constexpr int TC_M = 128;          // real-form rows (p^2 <= 64 complex)
constexpr int TC_K = 128;          // real-form reduction length
constexpr int TC_N = 64;           // columns per tile
constexpr int A_BYTES = TC_M * TC_K * 4;   // 64 KiB
constexpr int B_BYTES = TC_N * TC_K * 4;   // 32 KiB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr unsigned SPIN_LIMIT = 1u << 22;  // one product takes about a microsecond

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// float index of element (row, k) in the core-matrix layout of a rows x 128 K-major operand
__host__ __device__ __forceinline__ int core_index(int row, int k) {
    return (row >> 3) * 1024 + (k >> 2) * 32 + (row & 7) * 4 + (k & 3);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    const uint64_t lbo = 128, sbo = 4096;  // K-adjacent core matrices, 8-row groups
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= ((lbo >> 4) & 0x3FFFu) << 16;
    d |= ((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of the sm_100 family; base offset 0, no swizzle
    return d;
}

// instruction descriptor: D f32, A and B tf32, both K-major, N and M
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                           ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void mbar_init(uint64_t *m, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *m, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(m)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait; returns false on time-out
__device__ __forceinline__ bool mbar_wait(uint64_t *m, uint32_t parity) {
    for (unsigned it = 0; it < SPIN_LIMIT; ++it)
        if (mbar_try_wait(m, parity)) return true;
    return false;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *m) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(m))
                 : "memory");
}

// stage one product: A (precomputed layout, straight copy) and B (64 columns of interleaved
// complex coefficients, p2 complex each, rounded to tf32, zero beyond p2 and beyond ncol)
__device__ __forceinline__ void stage_product(float *sA, float *sB, const float4 *__restrict__ Ag, const float *Bcols,
                                              int p2, int ncol) {
    float4 *sA4 = reinterpret_cast<float4 *>(sA);
    for (int i = threadIdx.x; i < A_BYTES / 16; i += blockDim.x) sA4[i] = Ag[i];
    // B: column n, K chunk kc (4 floats): core_index(n, 4kc) .. +3
    for (int i = threadIdx.x; i < TC_N * (TC_K / 4); i += blockDim.x) {
        const int n = i / (TC_K / 4), kc = i % (TC_K / 4);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n < ncol && 4 * kc < 2 * p2) {
            const float4 g = *reinterpret_cast<const float4 *>(Bcols + (int64_t)n * 2 * p2 + 4 * kc);
            v = make_float4(to_tf32(g.x), to_tf32(g.y), to_tf32(g.z), to_tf32(g.w));
        }
        *reinterpret_cast<float4 *>(sB + core_index(n, 4 * kc)) = v;
    }
}

__global__ void __launch_bounds__(128) k_m2l_tc(int64_t off, int l, int lmax, int64_t nr, int p2, int64_t nbox,
                                                const int32_t *parent, const uint64_t *key, const int32_t *ff_start,
                                                const int32_t *ff_src, const int16_t *ff_off, const float4 *Atc,
                                                const float4 *Lltc, const float *C, float *D, int *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    const int64_t g = off + blockIdx.x;
    const int d = blockIdx.y;
    const int ncols = (int)(3 * nr);
    const int col0 = blockIdx.z * TC_N;
    const int nh = min(TC_N, ncols - col0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TC_N)
                     : "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    const int e0 = ff_start[g], e1 = ff_start[g + 1];
    const bool has_l2l = l >= 3;
    const int nprod = (has_l2l ? 1 : 0) + (e1 - e0);
    const int64_t tbl_level = ((int64_t)d * (lmax + 1) + l);
    // waits are taken by thread 0 alone and their outcome is shared, so every thread leaves the
    // loop at the same product even when a bounded wait times out
    __shared__ int s_ok;
    bool ok = true;
    for (int i = 0; i < nprod && ok; ++i) {
        const int s = i & 1;
        float *sA = reinterpret_cast<float *>(smem_raw + s * STAGE_BYTES);
        float *sB = reinterpret_cast<float *>(smem_raw + s * STAGE_BYTES + A_BYTES);
        if (i >= 2) {  // the MMAs that read this stage two products ago must be done
            if (threadIdx.x == 0) s_ok = mbar_wait(&mbar[s], ((i - 2) >> 1) & 1) ? 1 : 0;
            __syncthreads();
            ok = s_ok != 0;
            if (!ok) break;
        }
        const float4 *Ag;
        const float *Bc;
        if (has_l2l && i == 0) {
            Ag = Lltc + (tbl_level * 8 + (int)(key[g] & 7)) * (A_BYTES / 16);
            Bc = D + (((int64_t)d * nbox + parent[g]) * ncols + col0) * 2 * p2;
        } else {
            const int e = e0 + i - (has_l2l ? 1 : 0);
            Ag = Atc + (tbl_level * 316 + ff_off[e]) * (A_BYTES / 16);
            Bc = C + (((int64_t)d * nbox + ff_src[e]) * ncols + col0) * 2 * p2;
        }
        stage_product(sA, sB, Ag, Bc, p2, nh);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // make generic stores visible to the tensor cores
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
            for (int kk = 0; kk < TC_K / 8; ++kk)  // each MMA consumes two K-adjacent core matrices
                mma_tf32(tmem, smem_desc(a0 + kk * 256), smem_desc(b0 + kk * 256), (i > 0 || kk > 0) ? 1u : 0u);
            mma_commit(&mbar[s]);
        }
    }
    if (threadIdx.x == 0) {
        bool fin = ok;
        if (fin && nprod > 0) fin = mbar_wait(&mbar[(nprod - 1) & 1], ((nprod - 1) >> 1) & 1);
        if (!fin) atomicExch(err, 1);
        s_ok = fin ? 1 : 0;
    }
    __syncthreads();
    ok = s_ok != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (nprod == 0) {  // no translation reaches this box: its local expansion is zero
        float *Dout = D + (((int64_t)d * nbox + g) * ncols + col0) * 2 * p2;
        for (int i = threadIdx.x; i < nh * 2 * p2; i += blockDim.x) Dout[i] = 0.f;
    } else if (ok) {
        // warp w owns accumulator lanes 32w..32w+31 = real-form rows; row R = 2r + a
        const int R = warp * 32 + lane, r = R >> 1, a = R & 1;
        float *Dout = D + (((int64_t)d * nbox + g) * ncols + col0) * 2 * p2;
#pragma unroll
        for (int c0 = 0; c0 < TC_N; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (r < p2)
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (c0 + j < nh) Dout[(int64_t)(c0 + j) * 2 * p2 + 2 * r + a] = __uint_as_float(v[j]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
}

// real-form TF32 image of one complex p2 x p2 matrix stored input-major (T[c][r]) in double
// precision, written in the core-matrix layout: A[2r+a][2k+b]
__global__ void k_build_tc_tables(const c64 *T, int64_t nmat, int p2, float *out) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nmat * TC_M * TC_K) return;
    const int64_t m = idx / (TC_M * TC_K);
    const int R = (int)(idx % (TC_M * TC_K)) / TC_K, K = (int)(idx % TC_K);
    const int r = R >> 1, a = R & 1, k = K >> 1, b = K & 1;
    float v = 0.f;
    if (r < p2 && k < p2) {
        const c64 t = T[(m * p2 + k) * p2 + r];
        // [[Re, -Im], [Im, Re]]
        double x = (a == 0) ? (b == 0 ? t.re : -t.im) : (b == 0 ? t.im : t.re);
        v = to_tf32((float)x);
    }
    out[m * (TC_M * TC_K) + core_index(R, K)] = v;
}

}  // namespace

// p^2 <= 64 fills the 128-row real form; an even p keeps every column 16-byte aligned
bool m2l_tc_supported(const fmbem *h) { return h->p <= 8 && h->p % 2 == 0; }

void build_tc_tables(fmbem *h, cudaStream_t s) {
    const int p2 = h->p2;
    const int64_t n_m2l = (int64_t)(h->J + 1) * (h->lmax + 1) * 316, n_oct = (int64_t)(h->J + 1) * (h->lmax + 1) * 8;
    h->Atc = (float *)dev_alloc(h, (size_t)A_BYTES * n_m2l);
    h->Lltc = (float *)dev_alloc(h, (size_t)A_BYTES * n_oct);
    const int tb = 256;
    k_build_tc_tables<<<(unsigned)((n_m2l * TC_M * TC_K + tb - 1) / tb), tb, 0, s>>>(h->T_m2l64, n_m2l, p2, h->Atc);
    CKL("k_build_tc_tables");
    k_build_tc_tables<<<(unsigned)((n_oct * TC_M * TC_K + tb - 1) / tb), tb, 0, s>>>(h->T_ll64, n_oct, p2, h->Lltc);
    CKL("k_build_tc_tables");
    h->tc_err = (int *)dev_alloc(h, sizeof(int));
    CK(cudaMemsetAsync(h->tc_err, 0, sizeof(int), s));
}

// downward pass for all levels, single precision coefficients (C, D as interleaved floats)
void run_m2l_tc(fmbem *h, const float *C, float *D, int64_t nr, cudaStream_t s) {
    const size_t smem = 2 * (size_t)STAGE_BYTES;
    CK(cudaFuncSetAttribute(k_m2l_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const unsigned ntile = (unsigned)((3 * nr + TC_N - 1) / TC_N);
    for (int l = 2; l <= h->lmax; ++l) {
        const LevelInfo &Lv = h->lev[l];
        k_m2l_tc<<<dim3((unsigned)Lv.n, h->J + 1, ntile), 128, smem, s>>>(
            Lv.off, l, h->lmax, nr, h->p2, h->nbox, h->box_parent, h->box_key, h->ff_start, h->ff_src, h->ff_off,
            (const float4 *)h->Atc, (const float4 *)h->Lltc, C, D, h->tc_err);
        CKL("k_m2l_tc");
    }
}
