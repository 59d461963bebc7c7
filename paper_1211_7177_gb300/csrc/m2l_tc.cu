// m2l_tc.cu -- M2L + L2L (Eq. 2.21) for many right-hand sides on the GB300 tensor cores
// (tcgen05.mma kind::tf32 with the accumulator in tensor memory, operands brought in by TMA).
//
// For one target box, one domain and a tile of N columns (3 Cartesian components x right-hand
// sides), D[:, tile] = T_ll(oct) D[parent][:, tile] + sum_FF T_o C[src][:, tile] is a chain of
// complex (p^2 x p^2) x (p^2 x N) products.  In interleaved real form -- row 2r + a is the real
// (a = 0) or imaginary (a = 1) part of coefficient r, and likewise along K -- each product is a
// real 128 x (2 p^2) x N GEMM:
//   A[2r+a][2k+b] = [[Re T, -Im T], [Im T, Re T]][a][b],   B[2k+b][n] = (Re, Im)[b] C[src][n][k].
// Column n of B is the coefficient vector of column n exactly as the expansions are stored
// (re, im interleaved, 2 p^2 floats), so B is K-major in global memory as it stands: TMA reads a
// 32-float (128-byte) K block of N consecutive columns into shared memory with the 128-byte
// swizzle.  The A images are precomputed per (domain, level, offset), rounded to TF32 and stored
// in global memory already in the same swizzled K-major layout, one 16 KiB block per K block, so
// a plain bulk copy stages them.
//
// Roles (128 threads, one CTA per (target box, domain, tile of up to 512 columns held as one or
// two accumulators of up to 256 TMEM columns)): thread 0 is the producer (waits for a free stage,
// arms the stage's mbarrier with the byte count, issues the A bulk copy and one B tensor copy per
// sub-tile), thread 32 issues the MMAs (waits for a full stage, four K = 8 MMAs per K block and
// sub-tile, commits to the stage's "empty" mbarrier, finally to the "done" mbarrier), and all
// four warps read the accumulators with tcgen05.ld and write D.  Every mbarrier wait is bounded (2 s by
// %globaltimer); on time-out the kernel raises an error flag, stops issuing work, waits (bounded)
// for its own copies and MMAs in flight, frees its tensor memory and returns.
//
// The BF16x3 form (precision FMBEM_BF16X3) runs the same chain with kind::f16 MMAs on bf16
// operands: every real-form value x is split into x_hi = bf16(x) and x_lo = bf16(x - x_hi), and
// each product is accumulated as A_hi B_hi + A_hi B_lo + A_lo B_hi (the dropped A_lo B_lo is
// ~2^-16 of the product), which brings the rounding error from TF32's ~2^-11 to ~2^-16 per
// product while moving the same bytes: a 32-element K block of hi and lo bf16 rows is 64 + 64
// bytes, staged with the 64-byte swizzle.  The expansions C are split once before the pass and
// the local expansions of non-leaf levels are split in the epilogue for the next level's L2L.
#include <cuda.h>  // CUtensorMap and its enums; the encoder itself is looked up at run time
#include <cuda_bf16.h>

#include <algorithm>
#include <string>

#include "fmbem_internal.cuh"

namespace {

constexpr int TC_M = 128;                    // real-form rows (2 p^2 <= 128)
constexpr int KBLK = 32;                     // TF32 elements per 128-byte swizzle row
constexpr int A_KB_BYTES = TC_M * KBLK * 4;  // 16 KiB of A per K block
constexpr int MAX_STAGES = 8;
constexpr int SMEM_BUDGET = 200 * 1024;      // dynamic shared memory for the stages
constexpr uint64_t WAIT_NS = 2000000000ull;  // a stage turns over in about a microsecond

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// float index of element (row, k) of one 128-row K block in the 128-byte-swizzled K-major layout:
// rows 128 bytes apart, the 16-byte chunk c of row m stored at chunk c ^ (m mod 8)
__host__ __device__ __forceinline__ int sw128_index(int row, int k) {
    return row * KBLK + (((k >> 2) ^ (row & 7)) << 2) + (k & 3);
}

// shared-memory matrix descriptor, K-major, 128-byte swizzle: 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
    d |= (uint64_t)1 << 46;            // descriptor version of the sm_100 family
    d |= (uint64_t)2 << 61;            // 128-byte swizzle
    return d;
}

// instruction descriptor: D f32, A and B tf32, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}
// instruction descriptor of kind::f16: D f32, A and B bf16, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

// bf16 index of element (row, k) of one K block (32 bf16 = 64 bytes per row) in the 64-byte-swizzled
// K-major layout: the 16-byte chunk c of row m stored at chunk c ^ ((m / 2) mod 4)
__host__ __device__ __forceinline__ int sw64_index(int row, int k) {
    return row * KBLK + ((((k >> 3) ^ (row >> 1)) & 3) << 3) + (k & 7);
}

// shared-memory matrix descriptor, K-major, 64-byte swizzle: 8-row groups 512 bytes apart
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;           // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(512 >> 4) << 32;  // stride byte offset
    d |= (uint64_t)1 << 46;           // descriptor version of the sm_100 family
    d |= (uint64_t)4 << 61;           // 64-byte swizzle
    return d;
}

__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
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
// bounded wait for the phase of the given parity; false on time-out
__device__ __noinline__ bool mbar_wait(uint64_t *m, uint32_t parity) {
    if (mbar_try_wait(m, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (;;) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try_wait(m, parity)) return true;
        if (globaltimer() - t0 > WAIT_NS) return false;
    }
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *m, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}
// 1-D bulk copy global -> shared, completion counted on the mbarrier
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint64_t *m) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(smem_u32(m))
                 : "memory");
}
// 2-D tiled tensor copy global -> shared (box and swizzle from the tensor map)
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *tm, int x, int y, uint64_t *m) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(smem_u32(m))
        : "memory");
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *m) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(m))
                 : "memory");
}

struct TcLevel {
    int64_t off;          // first box of the level
    int l, lmax;
    int64_t nbox;
    int ncols;            // 3 * n_rhs
    int p2, kblocks;      // K blocks of 32 real-form elements: ceil(2 p^2 / 32)
    int n, nsub, stages;  // columns per sub-tile (multiple of 16, <= 256), sub-tiles per CTA, depth
    uint32_t tmem_cols;   // power of two >= nsub * n
    int round_out;        // round D to TF32 (it feeds the next level's L2L product)
    int m2m;              // 1: M2M (Eq. 2.20): box g of level l - 1 sums S|S C(child) over its children
};

// BF3 = false: TF32 operands (tmC, tmD over the TF32-rounded FP32 expansions, A images of TF32
// values).  BF3 = true: bf16 hi/lo operands (tmC/tmD over the hi parts, tmC2/tmD2 over the lo
// parts, A images of [hi | lo] 8 KiB halves per K block), three products per K step, and on
// non-leaf levels the epilogue also writes the hi/lo split of D (Dh, Dl) for the next level.
template <bool BF3>
__global__ void __launch_bounds__(128, 1)
    k_m2l_tc(const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmD,
             const __grid_constant__ CUtensorMap tmC2, const __grid_constant__ CUtensorMap tmD2, const TcLevel P,
             const int32_t *__restrict__ parent, const uint64_t *__restrict__ key, const int32_t *__restrict__ ff_start,
             const int32_t *__restrict__ ff_src, const int16_t *__restrict__ ff_off, const float *__restrict__ Atc,
             const float *__restrict__ Lltc, float *D, __nv_bfloat16 *Dh, __nv_bfloat16 *Dl, int *err,
             const int32_t *__restrict__ cbeg, const int32_t *__restrict__ cend) {
    // M2M: a box without children (a leaf of an adaptive tree) keeps its P2M expansion
    if (P.m2m && cbeg[P.off + blockIdx.x] == cend[P.off + blockIdx.x]) return;
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t full[MAX_STAGES], empty[MAX_STAGES], done;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_abort;
    __shared__ int s_fin;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t g = P.off + blockIdx.x;
    const int d = blockIdx.y;
    const int col0 = blockIdx.z * P.n * P.nsub;  // first column of this CTA's tile
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;  // swizzle atoms need 1024-byte alignment
    const uint32_t b_bytes = (uint32_t)P.n * 128u;                 // one sub-tile's K block of B
    const uint32_t stage_bytes = A_KB_BYTES + (uint32_t)P.nsub * b_bytes;

    if (threadIdx.x == 0) {
        for (int s = 0; s < P.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        s_abort = *(volatile int *)err;  // an earlier CTA timed out: issue nothing
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmC)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmD)) : "memory");
        if (BF3) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmC2)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmD2)) : "memory");
        }
    }
    if (warp == 0)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(P.tmem_cols)
                     : "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    // products: M2L + L2L (the parent's R|R, then the FF list), or M2M (the children's S|S; Atc
    // then holds the S|S images, Lltc is unused)
    const int e0 = P.m2m ? cbeg[g] : ff_start[g], e1 = P.m2m ? cend[g] : ff_start[g + 1];
    const int has_l2l = P.l >= 3 && !P.m2m ? 1 : 0;
    const int nprod = has_l2l + (e1 - e0);
    const int nunits = nprod * P.kblocks;
    const int64_t tbl = (int64_t)d * (P.lmax + 1) + P.l;
    const int64_t a_mat = (int64_t)P.kblocks * (A_KB_BYTES / 4);  // floats per A image
    int issued = 0;

    if (threadIdx.x == 0 && nunits > 0) {
        // ------------------------------------------------------------------ producer
        bool ok = true;
        int s = 0, q = 0;
        for (int u = 0; u < nunits; ++u) {
            if (q > 0 && !mbar_wait(&empty[s], (uint32_t)(q - 1) & 1u)) { ok = false; break; }
            if (s_abort || *(volatile int *)err) break;
            const int i = u / P.kblocks, kb = u - i * P.kblocks;
            const float *Asrc;
            const CUtensorMap *tm, *tm2;
            int y;
            if (has_l2l && i == 0) {
                Asrc = Lltc + (tbl * 8 + (int)(key[g] & 7)) * a_mat;
                tm = &tmD;
                tm2 = &tmD2;
                y = (int)(((int64_t)d * P.nbox + parent[g]) * P.ncols + col0);
            } else if (P.m2m) {
                const int ch = e0 + i;
                Asrc = Atc + (tbl * 8 + (int)(key[ch] & 7)) * a_mat;
                tm = &tmC;
                tm2 = &tmC2;
                y = (int)(((int64_t)d * P.nbox + ch) * P.ncols + col0);
            } else {
                const int e = e0 + i - has_l2l;
                Asrc = Atc + (tbl * 316 + ff_off[e]) * a_mat;
                tm = &tmC;
                tm2 = &tmC2;
                y = (int)(((int64_t)d * P.nbox + ff_src[e]) * P.ncols + col0);
            }
            const uint32_t sA = sbase + (uint32_t)s * stage_bytes, sB = sA + A_KB_BYTES;
            mbar_arrive_expect_tx(&full[s], stage_bytes);
            bulk_load(sA, Asrc + (int64_t)kb * (A_KB_BYTES / 4), A_KB_BYTES, &full[s]);
            for (int j = 0; j < P.nsub; ++j) {
                tma_load_2d(sB + j * b_bytes, tm, kb * KBLK, y + j * P.n, &full[s]);
                // bf16: the lo rows follow the n hi rows of 64 bytes
                if (BF3) tma_load_2d(sB + j * b_bytes + (uint32_t)P.n * 64u, tm2, kb * KBLK, y + j * P.n, &full[s]);
            }
            ++issued;
            if (++s == P.stages) { s = 0; ++q; }
        }
        if (!ok) { atomicExch(err, 1); s_abort = 1; }
    } else if (threadIdx.x == 32 && nunits > 0) {
        // ------------------------------------------------------------------ MMA issuer
        const uint32_t idesc = BF3 ? idesc_bf16(P.n) : idesc_tf32(P.n);
        bool ok = true;
        int s = 0, q = 0;
        for (int u = 0; u < nunits && !s_abort; ++u) {
            if (!mbar_wait(&full[s], (uint32_t)q & 1u)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sA = sbase + (uint32_t)s * stage_bytes, sB = sA + A_KB_BYTES;
            for (int t = 0; t < P.nsub; ++t) {  // one accumulator of n TMEM columns per sub-tile
                const uint32_t acc = tmem + (uint32_t)(t * P.n);
                if (BF3) {
#pragma unroll
                    for (int j = 0; j < 2; ++j) {  // K = 16 bf16 per MMA = 32 bytes along the 64-byte row
                        const uint64_t ah = smem_desc_sw64(sA + 32u * j), al = smem_desc_sw64(sA + 8192u + 32u * j);
                        const uint64_t bh = smem_desc_sw64(sB + t * b_bytes + 32u * j);
                        const uint64_t bl = smem_desc_sw64(sB + t * b_bytes + (uint32_t)P.n * 64u + 32u * j);
                        mma_bf16(acc, ah, bh, idesc, (u > 0 || j > 0) ? 1u : 0u);
                        mma_bf16(acc, ah, bl, idesc, 1u);
                        mma_bf16(acc, al, bh, idesc, 1u);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < KBLK / 8; ++j)  // K = 8 TF32 per MMA = 32 bytes along the swizzled row
                        mma_tf32(acc, smem_desc_sw128(sA + 32u * j), smem_desc_sw128(sB + t * b_bytes + 32u * j), idesc,
                                 (u > 0 || j > 0) ? 1u : 0u);
                }
            }
            mma_commit(&empty[s]);
            if (++s == P.stages) { s = 0; ++q; }
        }
        mma_commit(&done);  // arrives once every MMA issued above has completed
        if (!ok) { atomicExch(err, 1); s_abort = 1; }
    }
    __syncwarp();
    __syncthreads();
    if (threadIdx.x == 0) {
        bool fin = !s_abort;
        if (nunits > 0 && !mbar_wait(&done, 0)) { fin = false; atomicExch(err, 1); }
        s_fin = fin ? 1 : 0;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    const int nh = min(P.n * P.nsub, P.ncols - col0);  // valid columns of this CTA's tile
    float *Dout = D + (((int64_t)d * P.nbox + g) * P.ncols + col0) * 2 * P.p2;
    if (nprod == 0) {  // no translation reaches this box: its local expansion is zero
        for (int i = threadIdx.x; i < nh * 2 * P.p2; i += blockDim.x) Dout[i] = 0.f;
        if (BF3 && P.round_out) {
            const int64_t ob = (((int64_t)d * P.nbox + g) * P.ncols + col0) * 2 * P.p2;
            for (int i = threadIdx.x; i < nh * 2 * P.p2; i += blockDim.x) {
                Dh[ob + i] = __float2bfloat16_rn(0.f);
                Dl[ob + i] = __float2bfloat16_rn(0.f);
            }
        }
    } else if (s_fin) {
        // warp w owns accumulator lanes 32w..32w+31 = real-form rows R = 2r + a; sub-tile t sits
        // in TMEM columns t n .. t n + n - 1, so tile column c is TMEM column c
        const int R = warp * 32 + lane;
        const bool row_ok = R < 2 * P.p2;
        for (int c0 = 0; c0 < P.n * P.nsub; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row_ok)
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (c0 + j < nh) {
                        const float x = __uint_as_float(v[j]);
                        const int64_t o = (int64_t)(c0 + j) * 2 * P.p2 + R;
                        if (BF3) {
                            Dout[o] = x;
                            if (P.round_out) {  // the hi/lo split the next level's L2L reads
                                const int64_t ob = (((int64_t)d * P.nbox + g) * P.ncols + col0) * 2 * P.p2 + o;
                                const __nv_bfloat16 hi = __float2bfloat16_rn(x);
                                Dh[ob] = hi;
                                Dl[ob] = __float2bfloat16_rn(x - __bfloat162float(hi));
                            }
                        } else {
                            Dout[o] = P.round_out ? to_tf32(x) : x;
                        }
                    }
        }
    }
    if (threadIdx.x == 0 && issued > 0) {
        // copies still in flight after an abort: wait (bounded) for the last copy of each stage
        for (int u = max(0, issued - P.stages); u < issued; ++u)
            if (!mbar_wait(&full[u % P.stages], (uint32_t)(u / P.stages) & 1u)) atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P.tmem_cols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
}

// real-form TF32 image of one complex p2 x p2 matrix stored input-major (T[c][r]) in double
// precision, written as kblocks swizzled K blocks: A[2r+a][2k+b]
__global__ void k_build_tc_tables(const c64 *T, int64_t nmat, int p2, int kblocks, float *out) {
    const int64_t per = (int64_t)kblocks * TC_M * KBLK;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nmat * per) return;
    const int64_t m = idx / per;
    const int rem = (int)(idx % per);
    const int kb = rem / (TC_M * KBLK), R = (rem % (TC_M * KBLK)) / KBLK, kk = rem % KBLK;
    const int K = kb * KBLK + kk;
    const int r = R >> 1, a = R & 1, k = K >> 1, b = K & 1;
    float v = 0.f;
    if (r < p2 && k < p2) {
        const c64 t = T[(m * p2 + k) * p2 + r];
        const double x = (a == 0) ? (b == 0 ? t.re : -t.im) : (b == 0 ? t.im : t.re);  // [[Re, -Im], [Im, Re]]
        v = to_tf32((float)x);
    }
    out[m * per + (int64_t)kb * TC_M * KBLK + sw128_index(R, kk)] = v;
}

// bf16 hi/lo image of the same matrices: per K block, 128 rows x 32 of hi then of lo, each in the
// 64-byte-swizzled K-major layout (8 KiB + 8 KiB, the byte size of one TF32 K block)
__global__ void k_build_bf3_tables(const c64 *T, int64_t nmat, int p2, int kblocks, __nv_bfloat16 *out) {
    const int64_t per = (int64_t)kblocks * TC_M * KBLK;  // elements of one matrix, per half
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nmat * per) return;
    const int64_t m = idx / per;
    const int rem = (int)(idx % per);
    const int kb = rem / (TC_M * KBLK), R = (rem % (TC_M * KBLK)) / KBLK, kk = rem % KBLK;
    const int K = kb * KBLK + kk;
    const int r = R >> 1, a = R & 1, k = K >> 1, b = K & 1;
    double x = 0.0;
    if (r < p2 && k < p2) {
        const c64 t = T[(m * p2 + k) * p2 + r];
        x = (a == 0) ? (b == 0 ? t.re : -t.im) : (b == 0 ? t.im : t.re);  // [[Re, -Im], [Im, Re]]
    }
    const __nv_bfloat16 hi = __double2bfloat16(x);
    const __nv_bfloat16 lo = __double2bfloat16(x - (double)__bfloat162float(hi));
    __nv_bfloat16 *blk = out + m * 2 * per + (int64_t)kb * 2 * TC_M * KBLK;
    blk[sw64_index(R, kk)] = hi;
    blk[TC_M * KBLK + sw64_index(R, kk)] = lo;
}

// hi/lo bf16 split of a float array (the expansions the BF16x3 products read as B)
__global__ void k_split_bf16(const float *x, __nv_bfloat16 *hi, __nv_bfloat16 *lo, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = x[i];
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[i] = h;
        lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

// round a float array to TF32 in place (the expansions the tensor-core products read as B)
__global__ void k_round_tf32(float *x, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = to_tf32(x[i]);
}

// ------------------------------------------------------------------------------------------
// P2M (Eqs. 2.18-2.19) for many right-hand sides on the tensor cores, BF16x3.  For one leaf and
// domain, C[col][q] = sum over (node i, k = 0..3) of B_k(i, q) W_k(i, col): the P2M basis rows
// (B_0 = R_n^{-m}, B_{1..3} = grad R) times the density weights (W_0 = q_c and
// W_k = v_c n_k + (n.v) delta_ck - n_c v_k for column col = 3 r + c, so that sum_k W_k B_k =
// m_c . grad R + q_c R).  In real form -- row 2q + a the real (a = 0) or imaginary (a = 1) part of
// coefficient q; K index 8 il + 2 k + b for node il of a group of four, b selecting Re / Im W --
//   A[2q][.] = (Re B_k, -Im B_k),  A[2q+1][.] = (Im B_k, Re B_k),  B[col][.] = (Re W_k, Im W_k),
// a 128 x NT x (8 per node) product per (leaf, domain, column tile).  Both operands are formed in
// registers from the basis table and the densities, split into bf16 hi / lo parts and stored into
// shared memory in the 64-byte-swizzled K-major layout (one K block of 32 = four nodes per stage,
// two stages), then thread 0 issues A_hi B_hi + A_hi B_lo + A_lo B_hi (tcgen05.mma kind::f16, FP32
// in tensor memory) after a proxy fence and a block barrier; the stage is rebuilt once the MMAs'
// commit has arrived on its mbarrier (a bounded wait).  The epilogue writes the bf16 hi / lo split
// of C (the operands of the tensor-core M2M and M2L, the only readers of the leaves' expansions on
// this path), and the FP32 values too when C is given.
constexpr int P2M_TC_THREADS = 256, P2M_TC_STAGES = 2;
constexpr uint32_t P2M_TC_A_BYTES = TC_M * KBLK * 2 * 2;  // hi + lo, 16 KiB

struct P2mTc {
    int64_t N, nr, nbox;
    int p2, ncols, nt, ntile;  // columns per tile: a multiple of 48 (whole right-hand sides, N % 16 == 0)
    uint32_t tmem_cols;
};

// eight floats -> eight bf16 hi parts and eight bf16 lo parts (x - hi), as 16-byte words
__device__ __forceinline__ void split8_bf16(const float *v, uint4 &hi, uint4 &lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
        const float2 hf = __bfloat1622float2(hh);
        const __nv_bfloat162 ll = __floats2bfloat162_rn(v[2 * j] - hf.x, v[2 * j + 1] - hf.y);
        h[j] = *reinterpret_cast<const uint32_t *>(&hh);
        l[j] = *reinterpret_cast<const uint32_t *>(&ll);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

__global__ void __launch_bounds__(P2M_TC_THREADS, 2)
    k_p2m_tc(const P2mTc P, const int32_t *__restrict__ leaf_box, const int32_t *__restrict__ nbeg,
             const int32_t *__restrict__ nend, const int32_t *__restrict__ dom, const float *__restrict__ nrm,
             const float2 *__restrict__ dens, const float4 *__restrict__ densS, const c64 *__restrict__ dcons,
             const float2 *__restrict__ Bp2m, float *C, __nv_bfloat16 *Ch, __nv_bfloat16 *Cl, int *err) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t empty[P2M_TC_STAGES], done;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_abort;
    __shared__ int s_fin;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t lf = blockIdx.x / P.ntile;
    const int tile = (int)(blockIdx.x - lf * P.ntile), d = blockIdx.y;
    const int64_t g = leaf_box[lf];
    const int col0 = tile * P.nt;
    const int nh = min(P.nt, P.ncols - col0);  // valid columns of the tile
    const int side = d == 0 ? 0 : 1;
    const float sg = d == 0 ? -1.f : 1.f;
    const int i0 = nbeg[g], i1 = nend[g];
    const int nkb = (i1 - i0 + 3) / 4;
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;  // swizzle atoms: 512-byte alignment
    unsigned char *gbase = smem_raw + (sbase - smem_u32(smem_raw));
    const uint32_t b_half = (uint32_t)P.nt * 64u;  // one K block of B, hi or lo
    const uint32_t stage_bytes = P2M_TC_A_BYTES + 2u * b_half;

    if (threadIdx.x == 0) {
        for (int s = 0; s < P2M_TC_STAGES; ++s) mbar_init(&empty[s], 1);
        mbar_init(&done, 1);
        s_abort = *(volatile int *)err;  // an earlier CTA timed out: issue nothing
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(P.tmem_cols)
                     : "memory");
        // give up the allocation permit at once: the next CTA on this SM may allocate (and be
        // resident) while this one runs
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = idesc_bf16(P.nt);
    int issued = 0;  // K blocks whose MMAs thread 0 issued

    // Each thread stages the same two A items (q0 = tid / 8 and q0 + 32, node il_a, part a) and at
    // most one B item (node il_b, right-hand side rl) of every K block.  Their global inputs are
    // loaded one K block ahead into registers (nxt) while the current block (cur) is converted
    // and stored, so the loads overlap the stores, the barriers and the MMAs.
    const int a_part = threadIdx.x & 1, il_a = (threadIdx.x >> 1) & 3, q0 = threadIdx.x >> 3;
    const int il_b = threadIdx.x & 3, rl = threadIdx.x >> 2;
    const bool b_item = rl < P.nt / 3 && 3 * rl < nh;
    const int64_t r_b = col0 / 3 + rl;
    // densS (node-major densities [block of 32 RHS][node][RHS][(v_0, q_0, s) as 4 float4]) when
    // given, else dens [side][RHS][node][(v, q)]: the scatterer side from v_1 = v_0 + s n and
    // q_1 = -gamma_d q_0
    const cx<float> gam = d > 0 && densS ? to<float>(dcons[3 * d + 2]) : cx<float>{0.f, 0.f};
    struct In {
        float2 a[2][4];  // B_k(i, q0), B_k(i, q0 + 32)
        int dom_a, dom_b;
        float2 b[6];     // the densities (v, q) of node il_b, right-hand side r_b
        float2 sj;       // with densS: s = n . (v_1 - v_0)
        float n[3];
    };
    auto load = [&](In &x, int kb) {
        const int ia = i0 + 4 * kb + il_a, ibn = i0 + 4 * kb + il_b;
        x.dom_a = -1;
        x.dom_b = -1;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int k = 0; k < 4; ++k) x.a[h][k] = make_float2(0.f, 0.f);
        if (ia < i1) {
            x.dom_a = dom[ia];
            const float2 *Bq = Bp2m + ((int64_t)side * P.N + ia) * 4 * P.p2;
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (q0 + 32 * h < P.p2)
#pragma unroll
                    for (int k = 0; k < 4; ++k) x.a[h][k] = Bq[(int64_t)k * P.p2 + q0 + 32 * h];
        }
        if (b_item && ibn < i1) {
            x.dom_b = dom[ibn];
            if (densS) {
                const float4 *o = densS + (((r_b >> 5) * P.N + ibn) * 32 + (r_b & 31)) * 4;
                const float4 o0 = o[0], o1 = o[1], o2 = o[2], o3 = o[3];
                x.b[0] = make_float2(o0.x, o0.y);
                x.b[1] = make_float2(o0.z, o0.w);
                x.b[2] = make_float2(o1.x, o1.y);
                x.b[3] = make_float2(o1.z, o1.w);
                x.b[4] = make_float2(o2.x, o2.y);
                x.b[5] = make_float2(o2.z, o2.w);
                x.sj = make_float2(o3.x, o3.y);
            } else {
                const float2 *dn = dens + (((int64_t)side * P.nr + r_b) * P.N + ibn) * 6;
#pragma unroll
                for (int c = 0; c < 6; ++c) x.b[c] = dn[c];
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) x.n[c] = nrm[3 * ibn + c];
        }
    };
    In cur, nxt;
    if (nkb > 0) load(cur, 0);

    for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % P2M_TC_STAGES;
        if (threadIdx.x == 0 && kb >= P2M_TC_STAGES && !s_abort &&
            !mbar_wait(&empty[s], (uint32_t)(kb / P2M_TC_STAGES - 1) & 1u)) {
            atomicExch(err, 1);
            s_abort = 1;
        }
        __syncthreads();  // stage s is free again (or the CTA gives up)
        if (s_abort) break;
        if (kb + 1 < nkb) load(nxt, kb + 1);
        __nv_bfloat16 *sA = reinterpret_cast<__nv_bfloat16 *>(gbase + (size_t)s * stage_bytes);
        __nv_bfloat16 *sB = sA + P2M_TC_A_BYTES / 2;
        // A: item (q, node il, part a) -> the 16-byte chunk il of row 2q + a (hi and lo); the
        // eight threads of a shared-memory phase fill two whole rows
        {
            const bool ok = cur.dom_a >= 0 && (d == 0 || cur.dom_a == d);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float v[8];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 b = ok ? cur.a[h][k] : make_float2(0.f, 0.f);
                    v[2 * k] = a_part == 0 ? b.x : b.y;
                    v[2 * k + 1] = a_part == 0 ? -b.y : b.x;
                }
                uint4 hi, lo;
                split8_bf16(v, hi, lo);
                const int o = sw64_index(2 * (q0 + 32 * h) + a_part, 8 * il_a);
                *reinterpret_cast<uint4 *>(sA + o) = hi;
                *reinterpret_cast<uint4 *>(sA + TC_M * KBLK + o) = lo;
            }
        }
        // B: item (right-hand side rl of the tile, node il) -> chunk il of rows 3 rl + c
        if (rl < P.nt / 3) {
            float w[3][8];
            if (cur.dom_b >= 0 && (d == 0 || cur.dom_b == d)) {
                float2 v[6];
#pragma unroll
                for (int c = 0; c < 6; ++c) v[c] = cur.b[c];
                if (densS && d > 0) {  // scatterer side from the background's
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        v[c].x += cur.sj.x * cur.n[c];
                        v[c].y += cur.sj.y * cur.n[c];
                        const float2 q0 = cur.b[3 + c];
                        v[3 + c] = make_float2(-(gam.re * q0.x - gam.im * q0.y), -(gam.re * q0.y + gam.im * q0.x));
                    }
                }
                const float n[3] = {sg * cur.n[0], sg * cur.n[1], sg * cur.n[2]};
                const float nvr = n[0] * v[0].x + n[1] * v[1].x + n[2] * v[2].x;
                const float nvi = n[0] * v[0].y + n[1] * v[1].y + n[2] * v[2].y;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    w[c][0] = v[3 + c].x;
                    w[c][1] = v[3 + c].y;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        float tr = n[k] * v[c].x - n[c] * v[k].x, ti = n[k] * v[c].y - n[c] * v[k].y;
                        if (k == c) {
                            tr += nvr;
                            ti += nvi;
                        }
                        w[c][2 + 2 * k] = tr;
                        w[c][3 + 2 * k] = ti;
                    }
                }
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int k = 0; k < 8; ++k) w[c][k] = 0.f;
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                uint4 hi, lo;
                split8_bf16(w[c], hi, lo);
                const int o = sw64_index(3 * rl + c, 8 * il_b);
                *reinterpret_cast<uint4 *>(sB + o) = hi;
                *reinterpret_cast<uint4 *>(sB + P.nt * KBLK + o) = lo;
            }
        }
        if (kb + 1 < nkb) cur = nxt;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the MMAs read what was stored
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t aA = sbase + (uint32_t)s * stage_bytes, aB = aA + P2M_TC_A_BYTES;
#pragma unroll
            for (int j = 0; j < 2; ++j) {  // K = 16 bf16 per MMA = 32 bytes along the 64-byte row
                const uint64_t ah = smem_desc_sw64(aA + 32u * j), al = smem_desc_sw64(aA + 8192u + 32u * j);
                const uint64_t bh = smem_desc_sw64(aB + 32u * j), bl = smem_desc_sw64(aB + b_half + 32u * j);
                mma_bf16(tmem, ah, bh, idesc, (kb > 0 || j > 0) ? 1u : 0u);
                mma_bf16(tmem, ah, bl, idesc, 1u);
                mma_bf16(tmem, al, bh, idesc, 1u);
            }
            mma_commit(&empty[s]);
            ++issued;
        }
    }
    if (threadIdx.x == 0) {
        bool fin = !s_abort && issued == nkb;
        if (issued > 0) {
            mma_commit(&done);  // arrives once every MMA issued above has completed
            if (!mbar_wait(&done, 0)) {
                fin = false;
                atomicExch(err, 1);
            }
        }
        s_fin = fin ? 1 : 0;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    const int64_t ob = (((int64_t)d * P.nbox + g) * P.ncols + col0) * 2 * P.p2;
    if (nkb == 0) {  // no sources: a zero expansion
        for (int i = threadIdx.x; i < nh * 2 * P.p2; i += blockDim.x) {
            if (C) C[ob + i] = 0.f;
            Ch[ob + i] = __float2bfloat16_rn(0.f);
            Cl[ob + i] = __float2bfloat16_rn(0.f);
        }
    } else if (s_fin) {
        // warp w reads accumulator lanes 32 (w mod 4) .. + 31 (real-form rows R); warps 0-3 take the
        // even 16-column groups, warps 4-7 the odd ones
        const int R = (warp & 3) * 32 + lane;
        const bool row_ok = R < 2 * P.p2;
        for (int c0 = 16 * (warp >> 2); c0 < P.nt; c0 += 32) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row_ok)
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (c0 + j < nh) {
                        const float x = __uint_as_float(v[j]);
                        const int64_t o = ob + (int64_t)(c0 + j) * 2 * P.p2 + R;
                        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
                        if (C) C[o] = x;
                        Ch[o] = hi;
                        Cl[o] = __float2bfloat16_rn(x - __bfloat162float(hi));
                    }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P.tmem_cols) : "memory");
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || p == nullptr)
            throw fmbem_error{FMBEM_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver"};
        fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// rows of 2 p^2 floats (one column's coefficients), boxes of 32 floats x n rows, 128-byte swizzle
CUtensorMap make_column_map(const float *base, int64_t rows, int p2, int n) {
    CUtensorMap tm;
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * p2), (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(2 * p2) * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)KBLK, (cuuint32_t)n};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode_tiled()(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides,
                                      box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        throw fmbem_error{FMBEM_ERR_CUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r)};
    return tm;
}

// bf16 rows of 2 p^2 values (one column's coefficients, hi or lo part), boxes of 32 x n rows,
// 64-byte swizzle
CUtensorMap make_column_map_bf16(const __nv_bfloat16 *base, int64_t rows, int p2, int n) {
    CUtensorMap tm;
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * p2), (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(2 * p2) * sizeof(__nv_bfloat16)};
    const cuuint32_t box[2] = {(cuuint32_t)KBLK, (cuuint32_t)n};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode_tiled()(&tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(base), dims,
                                      strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        throw fmbem_error{FMBEM_ERR_CUDA, "cuTensorMapEncodeTiled (bf16) failed with code " + std::to_string((int)r)};
    return tm;
}

int tc_kblocks(int p2) { return (2 * p2 + KBLK - 1) / KBLK; }

// ------------------------------------------------------------------------------------------
// Offset-stationary M2L for few columns (BF16x3 precision, up to 8 right-hand sides): the FF pairs
// of one level and domain, sorted by translation offset and cut into chunks of up to 32 pairs that
// share one S|R matrix, are a GEMM per chunk:
//   Y[pair column m][real-form row n] = sum_k C[source column m][k] S|R[n][k],
// with M = the chunk's pair columns (3 n_rhs per pair, up to 128 per pass), N = 2 p^2 rounded up
// to 16 (the S|R image rows), K = 2 p^2 (32-element blocks).  Both operands are split into bf16 hi
// and lo parts and each K step accumulates M_hi S_hi + M_hi S_lo + M_lo S_hi (tcgen05.mma kind::f16,
// FP32 in tensor memory).  The S|R image arrives by bulk copy; the source columns are gathered by
// the four producer warps (16-byte loads into the 64-byte-swizzled layout, then a proxy fence), warp
// w filling ring slot w; warp 4's first lane issues the MMAs; the producer warps then drain tensor
// memory and store each pair column's 2 p^2 results at the pair's CSR position, the layout
// k_l2l_reduce sums per target.  Every wait is bounded as in k_m2l_tc.
constexpr int OFS_STAGES = 4;
constexpr int OFS_M = 128;

// the work of one launch: every chunk of levels 2..l_max (chunk indices chunk0 + [0, nch)) for
// every domain 0..ndom-1, unit v = d * nch + chunk; Y[d][CSR position][column][2 p^2] floats
constexpr int OFS_MAX_LEVELS = 12;
struct OfsLevel {
    int64_t nbox;
    int ncols;      // columns per pair (3 n_rhs) = rows of C per box
    int p2, kblocks, np;
    int lmax, ndom;
    int ppp;        // pairs per pass: floor(128 / ncols)
    uint32_t tmem_cols;
    int64_t y_dom;  // floats of Y per domain
    int64_t level_first[OFS_MAX_LEVELS + 1];  // first chunk (relative to chunk0) of each level
};

// level of relative chunk index ckl (the levels' chunk ranges are contiguous and ascending)
__device__ __forceinline__ int ofs_level(const OfsLevel &P, int64_t ckl) {
    int l = 2;
    while (l < P.lmax && P.level_first[l + 1] <= ckl) ++l;
    return l;
}

// Persistent form: each CTA walks the chunks blockIdx.x, blockIdx.x + gridDim.x, ... as a sequence
// of (chunk, pass) tiles; warps 0-3 gather (warp w fills ring slot w of every fourth K block of the
// sequence), warp 4 issues the MMAs into one of two tensor-memory accumulators (tile t uses buffer
// t mod 2), and warps 5-8 drain the other accumulator meanwhile (warp 5 + i reads lanes 32 ((i + 1)
// mod 4) ...), so that gathering, MMAs and stores of consecutive tiles overlap.
constexpr int OFS_THREADS = 288;

__global__ void __launch_bounds__(OFS_THREADS, 1)
    k_m2l_ofs(const OfsLevel P, int64_t chunk0, int64_t nch, const int32_t *__restrict__ chunk_cnt,
              const int16_t *__restrict__ chunk_off, const int2 *__restrict__ chunk_pairs, const __nv_bfloat16 *Chi,
              const __nv_bfloat16 *Clo, const __nv_bfloat16 *__restrict__ Aofs, float *Y, int *err) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t full[OFS_STAGES], empty[OFS_STAGES], done[2], tfree[2], fin;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_abort;
    __shared__ int64_t rowoff[4][OFS_M];  // per producer warp: element offset of each pair column's
                                          // coefficients in its current tile, -1 past the tile's pairs
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const uint32_t b_half = (uint32_t)P.np * 64u;  // one bf16 part of an S|R K block
    const uint32_t stage_bytes = 2u * OFS_M * 64u + 2u * b_half;
    const int twop2 = 2 * P.p2;
    const int64_t nunit = nch * P.ndom;
    const bool any = (int64_t)blockIdx.x < nunit;

    if (threadIdx.x == 0) {
        for (int s = 0; s < OFS_STAGES; ++s) {
            mbar_init(&full[s], 33);  // the filling warp's 32 lanes + the bulk copy's expect_tx
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&done[b], 1);
            mbar_init(&tfree[b], 128);
        }
        mbar_init(&fin, 1);
        s_abort = *(volatile int *)err;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(2 * P.tmem_cols)
                     : "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (warp < 4) {
        // ------------------------------------------------------------------ producers
        int64_t last_issued = -1;  // this warp's last unit whose bulk copy was issued
        int64_t u = 0;             // unit (K block of a tile) counter of the CTA's sequence
        bool stop = false;
        for (int64_t v = blockIdx.x; v < nunit && !stop; v += gridDim.x) {
            const int d = (int)(v / nch);
            const int64_t ckl = v - (int64_t)d * nch, ck = chunk0 + ckl;
            const int64_t amat = ((int64_t)d * (P.lmax + 1) + ofs_level(P, ckl)) * 316 + chunk_off[ck];
            // the chunk's (source box, CSR position) pairs, one per lane, and its size
            const int2 pr = chunk_pairs[ck * 32 + lane];
            const int cnt = P.ppp >= 32 ? 32 : chunk_cnt[ck];  // one pass holds every chunk when ppp >= 32
            const int passes = (cnt + P.ppp - 1) / P.ppp;
            for (int pass = 0; pass < passes && !stop; ++pass) {
                bool table = false;  // this tile's source rows are in this warp's table
                for (int kb = 0; kb < P.kblocks; ++kb, ++u) {
                    if ((u & 3) != warp) continue;
                    if (!table) {
                        __syncwarp();
                        for (int m = lane; m < OFS_M; m += 32) {
                            const int jj = pass * P.ppp + m / P.ncols, c = m % P.ncols;
                            const int src = __shfl_sync(0xffffffffu, pr.x, jj & 31);
                            rowoff[warp][m] = (m < P.ppp * P.ncols && jj < 32 && src >= 0)
                                                  ? (((int64_t)d * P.nbox + src) * P.ncols + c) * twop2
                                                  : (int64_t)-1;
                        }
                        __syncwarp();
                        table = true;
                    }
                    const int64_t q = u >> 2;
                    bool ok = q == 0 || mbar_wait(&empty[warp], (uint32_t)(q - 1) & 1u);
                    ok = __all_sync(0xffffffffu, ok);
                    if (!ok || s_abort) {
                        if (lane == 0) { atomicExch(err, 1); s_abort = 1; }
                        stop = true;
                        break;
                    }
                    const uint32_t sM = sbase + (uint32_t)warp * stage_bytes, sB = sM + 2u * OFS_M * 64u;
                    if (lane == 0) {
                        const __nv_bfloat16 *Amat =
                            Aofs + (amat * (int64_t)P.kblocks + kb) * (int64_t)P.np * 64;
                        mbar_arrive_expect_tx(&full[warp], 2u * b_half);
                        bulk_load(sB, Amat, 2u * b_half, &full[warp]);
                        last_issued = u;
                    }
                    // 128 rows x (4 hi + 4 lo) 16-byte chunks of source coefficients by asynchronous
                    // copies (zero-filled past the tile's pairs and past 2 p^2), all in flight together
                    for (int i = lane; i < OFS_M * 8; i += 32) {
                        const int m = i >> 3, part = i & 7, lohalf = part >> 2, qc = part & 3;
                        const int k0 = kb * KBLK + 8 * qc;
                        const int64_t ro = rowoff[warp][m];
                        const bool valid = ro >= 0 && k0 < twop2;
                        const __nv_bfloat16 *src = valid ? (lohalf ? Clo : Chi) + ro + k0 : Chi;
                        const uint32_t dst = sM + (uint32_t)lohalf * (OFS_M * 64u) + (uint32_t)m * 64u +
                                             (uint32_t)((qc ^ ((m >> 1) & 3)) << 4);
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                                     "r"(valid ? 16 : 0)
                                     : "memory");
                    }
                    asm volatile("cp.async.wait_all;" ::: "memory");
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full[warp])) : "memory");
                }
            }
        }
        // a copy still in flight after an abort: wait (bounded) for this warp's last bulk copy
        if (lane == 0 && last_issued >= 0 && s_abort)
            if (!mbar_wait(&full[warp], (uint32_t)(last_issued >> 2) & 1u)) atomicExch(err, 1);
    } else if (warp == 4) {
        if (lane == 0) {
            // -------------------------------------------------------------- MMA issuer
            const uint32_t idesc = idesc_bf16(P.np);
            bool ok = true;
            int64_t u = 0, t = 0;
            for (int64_t v = blockIdx.x; v < nunit && ok && !s_abort; v += gridDim.x) {
                const int64_t ckl = v % nch;
                const int passes = P.ppp >= 32 ? 1 : (chunk_cnt[chunk0 + ckl] + P.ppp - 1) / P.ppp;
                for (int pass = 0; pass < passes && ok && !s_abort; ++pass, ++t) {
                    const int buf = (int)(t & 1);
                    const uint32_t acc = tmem + (uint32_t)buf * P.tmem_cols;
                    if (t >= 2 && !mbar_wait(&tfree[buf], (uint32_t)((t >> 1) - 1) & 1u)) { ok = false; break; }
                    for (int kb = 0; kb < P.kblocks; ++kb, ++u) {
                        const int s = (int)(u & 3);
                        if (!mbar_wait(&full[s], (uint32_t)(u >> 2) & 1u)) { ok = false; break; }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t sM = sbase + (uint32_t)s * stage_bytes, sB = sM + 2u * OFS_M * 64u;
#pragma unroll
                        for (int j = 0; j < 2; ++j) {  // K = 16 bf16 per MMA, 32 bytes along the 64-byte rows
                            const uint64_t mh = smem_desc_sw64(sM + 32u * j);
                            const uint64_t ml = smem_desc_sw64(sM + OFS_M * 64u + 32u * j);
                            const uint64_t bh = smem_desc_sw64(sB + 32u * j), bl = smem_desc_sw64(sB + b_half + 32u * j);
                            mma_bf16(acc, mh, bh, idesc, (kb > 0 || j > 0) ? 1u : 0u);
                            mma_bf16(acc, mh, bl, idesc, 1u);
                            mma_bf16(acc, ml, bh, idesc, 1u);
                        }
                        mma_commit(&empty[s]);
                    }
                    if (ok) mma_commit(&done[buf]);
                }
            }
            mma_commit(&fin);  // arrives once every MMA issued above has completed
            if (!ok) { atomicExch(err, 1); s_abort = 1; }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------------ epilogue warps 5..8
        const int ew = (warp - 5 + 1) & 3;  // the tensor-memory lane quarter this warp may read
        int64_t t = 0;
        bool stop = false;
        for (int64_t v = blockIdx.x; v < nunit && !stop; v += gridDim.x) {
            const int d = (int)(v / nch);
            const int64_t ck = chunk0 + (v - (int64_t)d * nch);
            float *Yd = Y + (int64_t)d * P.y_dom;
            const int2 pr = chunk_pairs[ck * 32 + lane];
            const int passes = P.ppp >= 32 ? 1 : (chunk_cnt[ck] + P.ppp - 1) / P.ppp;
            for (int pass = 0; pass < passes; ++pass, ++t) {
                const int buf = (int)(t & 1);
                bool ok = !s_abort && mbar_wait(&done[buf], (uint32_t)(t >> 1) & 1u);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) {
                    if (lane == 0) { atomicExch(err, 1); s_abort = 1; }
                    stop = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int m = ew * 32 + lane;
                const int jj = pass * P.ppp + m / P.ncols, c = m % P.ncols;
                const int e = __shfl_sync(0xffffffffu, pr.y, jj & 31);
                const bool valid = m < P.ppp * P.ncols && jj < 32 && e >= 0;
                float *out = valid ? Yd + ((int64_t)e * P.ncols + c) * twop2 : nullptr;
                for (int c0 = 0; c0 < P.np; c0 += 16) {
                    uint32_t v[16];
                    const uint32_t taddr = tmem + (uint32_t)buf * P.tmem_cols + ((uint32_t)(ew * 32) << 16) + (uint32_t)c0;
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                        "[%16];"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                          "=r"(v[15])
                        : "r"(taddr));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (valid)  // 16-byte stores (rows of 2 p^2 floats, p even: 16-byte aligned)
#pragma unroll
                        for (int j = 0; j < 16; j += 4)
                            if (c0 + j < twop2)
                                *reinterpret_cast<float4 *>(out + c0 + j) =
                                    make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]),
                                                __uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]));
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tfree[buf])) : "memory");
            }
        }
    }
    __syncwarp();
    __syncthreads();
    if (threadIdx.x == 0 && any && !mbar_wait(&fin, 0)) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * P.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
}

// per chunk of FF pairs, 32 entries (source box, CSR position of the pair); (-1, -1) past the chunk
__global__ void k_chunk_pairs(int64_t nch, const int32_t *chunk_beg, const int32_t *chunk_cnt, const int32_t *pair_e,
                              const int32_t *ff_src, int2 *out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nch * 32) return;
    const int64_t ck = i >> 5;
    const int j = (int)(i & 31);
    if (j < chunk_cnt[ck]) {
        const int e = pair_e[chunk_beg[ck] + j];
        out[i] = make_int2(ff_src[e], e);
    } else {
        out[i] = make_int2(-1, -1);
    }
}

// bf16 hi/lo images of the S|R matrices for k_m2l_ofs: per matrix and K block, np rows (the
// real-form output rows 2r + a, zero past 2 p^2) x 32 K elements of hi, then of lo, in the
// 64-byte-swizzled K-major layout
__global__ void k_build_ofs_tables(const c64 *T, int64_t nmat, int p2, int np, int kblocks, __nv_bfloat16 *out) {
    const int64_t per = (int64_t)kblocks * np * KBLK;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nmat * per) return;
    const int64_t m = idx / per;
    const int rem = (int)(idx % per);
    const int kb = rem / (np * KBLK), R = (rem % (np * KBLK)) / KBLK, kk = rem % KBLK;
    const int K = kb * KBLK + kk;
    const int r = R >> 1, a = R & 1, k = K >> 1, b = K & 1;
    double x = 0.0;
    if (r < p2 && k < p2) {
        const c64 t = T[(m * p2 + k) * p2 + r];
        x = (a == 0) ? (b == 0 ? t.re : -t.im) : (b == 0 ? t.im : t.re);  // [[Re, -Im], [Im, Re]]
    }
    const __nv_bfloat16 hi = __double2bfloat16(x);
    const __nv_bfloat16 lo = __double2bfloat16(x - (double)__bfloat162float(hi));
    __nv_bfloat16 *blk = out + m * 2 * per + (int64_t)kb * 2 * np * KBLK;
    blk[sw64_index(R, kk)] = hi;
    blk[(int64_t)np * KBLK + sw64_index(R, kk)] = lo;
}

}  // namespace

// 2 p^2 <= 128 fills the 128-row real form; p >= 4 makes a column's 2 p^2 floats at least one
// full 128-byte K block; an even p keeps the rows a multiple of 16 bytes, as a tensor map needs
bool m2l_tc_supported(const fmbem *h) { return h->p >= 4 && h->p <= 8 && h->p % 2 == 0; }

void build_tc_tables(fmbem *h, cudaStream_t s) {
    const int p2 = h->p2, kb = tc_kblocks(p2);
    const int64_t per = (int64_t)kb * TC_M * KBLK;
    const int64_t n_m2l = (int64_t)(h->J + 1) * (h->lmax + 1) * 316, n_oct = (int64_t)(h->J + 1) * (h->lmax + 1) * 8;
    h->Atc = (float *)dev_alloc(h, sizeof(float) * per * n_m2l);
    h->Lltc = (float *)dev_alloc(h, sizeof(float) * per * n_oct);
    const int tb = 256;
    k_build_tc_tables<<<(unsigned)((n_m2l * per + tb - 1) / tb), tb, 0, s>>>(h->T_m2l64, n_m2l, p2, kb, h->Atc);
    CKL("k_build_tc_tables");
    k_build_tc_tables<<<(unsigned)((n_oct * per + tb - 1) / tb), tb, 0, s>>>(h->T_ll64, n_oct, p2, kb, h->Lltc);
    CKL("k_build_tc_tables");
    // the bf16 hi/lo images take the bytes of the TF32 ones
    h->Abf = (float *)dev_alloc(h, sizeof(float) * per * n_m2l);
    h->Llbf = (float *)dev_alloc(h, sizeof(float) * per * n_oct);
    k_build_bf3_tables<<<(unsigned)((n_m2l * per + tb - 1) / tb), tb, 0, s>>>(h->T_m2l64, n_m2l, p2, kb,
                                                                            (__nv_bfloat16 *)h->Abf);
    CKL("k_build_bf3_tables");
    k_build_bf3_tables<<<(unsigned)((n_oct * per + tb - 1) / tb), tb, 0, s>>>(h->T_ll64, n_oct, p2, kb,
                                                                            (__nv_bfloat16 *)h->Llbf);
    CKL("k_build_bf3_tables");
    h->Mmbf = (float *)dev_alloc(h, sizeof(float) * per * n_oct);  // S|S images for M2M (BF16x3)
    k_build_bf3_tables<<<(unsigned)((n_oct * per + tb - 1) / tb), tb, 0, s>>>(h->T_mm64, n_oct, p2, kb,
                                                                            (__nv_bfloat16 *)h->Mmbf);
    CKL("k_build_bf3_tables");
    h->tc_err = (int *)dev_alloc(h, sizeof(int));
    CK(cudaMemsetAsync(h->tc_err, 0, sizeof(int), s));
}

// tile shape: a CTA covers up to 512 columns (the whole tensor memory) as one or two sub-tiles of
// at most 256 columns (one MMA's N), so each A image is loaded once per product for up to 170
// right-hand sides; sub-tiles split the columns evenly, rounded up to 16
void tc_tile_shape(int64_t ncols, int *n, int *nsub, int *ntile) {
    const int64_t t = (ncols + 511) / 512;
    const int64_t per = (ncols + t - 1) / t;
    *ntile = (int)t;
    *nsub = per > 256 ? 2 : 1;
    *n = (int)(((per + *nsub - 1) / *nsub + 15) / 16 * 16);
}

// downward pass for all levels: the multipole expansions C are rounded to TF32 in place first
// (TF32), or split into bf16 hi/lo parts in the second half of their buffer (BF16x3; the handle's
// expansion buffers hold double-precision complex values, so single precision leaves that half
// free); from here on only these products read them.  Then one launch per level.
// launch shape and tensor maps of the tile kernel for nr right-hand sides
struct TcSetup {
    int n, nsub, ntile, stages;
    size_t smem;
    uint32_t tcols;
    CUtensorMap tmC, tmD, tmC2, tmD2;
};
static TcSetup tc_setup(fmbem *h, float *C, float *D, int64_t nr, bool bf3) {
    TcSetup t{};
    const int64_t ncols = 3 * nr;
    const int64_t nfloat = (int64_t)(h->J + 1) * h->nbox * ncols * 2 * h->p2;
    tc_tile_shape(ncols, &t.n, &t.nsub, &t.ntile);
    const int stage = A_KB_BYTES + t.nsub * t.n * 128;
    t.stages = std::min(MAX_STAGES, SMEM_BUDGET / stage);
    t.smem = (size_t)t.stages * stage + 1024;  // + slack to align the stages to 1024 bytes
    t.tcols = 32;
    while ((int)t.tcols < t.nsub * t.n) t.tcols <<= 1;
    const int64_t rows = (int64_t)(h->J + 1) * h->nbox * ncols;
    if (bf3) {
        CK(cudaFuncSetAttribute(k_m2l_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t.smem));
        __nv_bfloat16 *Chi = (__nv_bfloat16 *)(C + nfloat), *Clo = Chi + nfloat;
        __nv_bfloat16 *Dhi = (__nv_bfloat16 *)(D + nfloat), *Dlo = Dhi + nfloat;
        t.tmC = make_column_map_bf16(Chi, rows, h->p2, t.n);
        t.tmC2 = make_column_map_bf16(Clo, rows, h->p2, t.n);
        t.tmD = make_column_map_bf16(Dhi, rows, h->p2, t.n);
        t.tmD2 = make_column_map_bf16(Dlo, rows, h->p2, t.n);
    } else {
        CK(cudaFuncSetAttribute(k_m2l_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t.smem));
        t.tmC = t.tmC2 = make_column_map(C, rows, h->p2, t.n);
        t.tmD = t.tmD2 = make_column_map(D, rows, h->p2, t.n);
    }
    return t;
}

// M2M (Eq. 2.20) on the tensor cores in the BF16x3 form, for the passes that then run M2L + L2L
// there too: the leaves' multipole expansions are split into bf16 hi/lo parts (the whole buffer:
// the other boxes' parts are written below), then one launch per level, l_max - 1 down to 2, in
// which every box sums the S|S products of its children and writes its expansion in FP32 and
// split; the M2L + L2L pass then finds C split (run_m2l_tc with c_split)
// (leaves_split: run_p2m_tc wrote the leaves' expansions split already, and the M2M launches write
// every other box of levels 2 .. l_max - 1, so the split pass is skipped)
void run_m2m_tc(fmbem *h, float *C, int64_t nr, cudaStream_t s, bool leaves_split) {
    const int64_t ncols = 3 * nr;
    const int64_t nfloat = (int64_t)(h->J + 1) * h->nbox * ncols * 2 * h->p2;
    __nv_bfloat16 *Chi = (__nv_bfloat16 *)(C + nfloat), *Clo = Chi + nfloat;
    if (!leaves_split) {
        k_split_bf16<<<152 * 8, 256, 0, s>>>(C, Chi, Clo, nfloat);
        CKL("k_split_bf16");
    }
    const TcSetup t = tc_setup(h, C, C, nr, true);
    for (int l = h->lmax; l >= 3; --l) {
        const LevelInfo &Lv = h->lev[l - 1];  // the parents
        const TcLevel P{Lv.off, l, h->lmax, h->nbox, (int)ncols, h->p2, tc_kblocks(h->p2), t.n, t.nsub, t.stages,
                        t.tcols, 1, 1};
        const dim3 grid((unsigned)Lv.n, h->Jf + 1, (unsigned)t.ntile);
        k_m2l_tc<true><<<grid, 128, t.smem, s>>>(t.tmC, t.tmC, t.tmC2, t.tmC2, P, h->box_parent, h->box_key,
                                                 h->ff_start, h->ff_src, h->ff_off, h->Mmbf, nullptr, C, Chi, Clo,
                                                 h->tc_err, h->box_cbeg, h->box_cend);
        CKL("k_m2l_tc (M2M)");
    }
}

// P2M of the leaves on the tensor cores (k_p2m_tc): BF16x3, 2 p^2 <= 128, 16 or more right-hand
// sides; the second half of C receives the bf16 hi / lo split of the leaves' expansions (run_m2m_tc
// with leaves_split).  The densities come from dens, or from the node-major densS when it is given
// (whole blocks of 32 right-hand sides, dens then unused)
bool p2m_tc_supported(const fmbem *h, int64_t nr) { return 2 * h->p2 <= TC_M && nr >= 16; }

void run_p2m_tc(fmbem *h, const float *dens, const float4 *densS, const float *Bp2m, float *C, int64_t nr,
                cudaStream_t s) {
    if (!p2m_tc_supported(h, nr)) throw fmbem_error{FMBEM_ERR_INVALID_ARGUMENT, "tensor-core P2M: unsupported shape"};
    if (!h->tc_err) throw fmbem_error{FMBEM_ERR_CUDA, "tensor-core P2M: the error flag was not allocated"};
    const int64_t ncols = 3 * nr;
    const int64_t nfloat = (int64_t)(h->J + 1) * h->nbox * ncols * 2 * h->p2;
    __nv_bfloat16 *Chi = (__nv_bfloat16 *)(C + nfloat), *Clo = Chi + nfloat;
    // tiles of whole right-hand sides: 48-column units, up to four (192 columns) per tile
    const int units = (int)((ncols + 47) / 48), ntile = (units + 3) / 4;
    const int nt = 48 * ((units + ntile - 1) / ntile);
    const uint32_t tcols = nt <= 64 ? 64u : nt <= 128 ? 128u : 256u;
    // shared memory: two stages; at least enough that no more CTAs share an SM than its 512 TMEM
    // columns hold (an allocation would otherwise wait for another CTA to free its columns)
    const int per_sm = 512 / (int)tcols;
    const size_t need = 1024 + P2M_TC_STAGES * (P2M_TC_A_BYTES + (size_t)nt * 128);
    const size_t smem = std::max(need, (size_t)(228 * 1024) / (per_sm + 1) + 1024);
    CK(cudaFuncSetAttribute(k_p2m_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const P2mTc P{h->N, nr, h->nbox, h->p2, (int)ncols, nt, ntile, tcols};
    const dim3 grid((unsigned)(h->n_leaves * ntile), (unsigned)(h->Jf + 1));
    // the FP32 copy of the leaves' expansions is not written: M2M and M2L read the split
    k_p2m_tc<<<grid, P2M_TC_THREADS, smem, s>>>(P, h->leaf_box, h->box_nbeg, h->box_nend, h->dom, h->nrm_f,
                                                (const float2 *)dens, densS, (const c64 *)h->dcons,
                                                (const float2 *)Bp2m, nullptr, Chi, Clo, h->tc_err);
    CKL("k_p2m_tc");
}

void run_m2l_tc(fmbem *h, float *C, float *D, int64_t nr, cudaStream_t s, bool bf3, bool c_split) {
    const int64_t ncols = 3 * nr;
    const int64_t nfloat = (int64_t)(h->J + 1) * h->nbox * ncols * 2 * h->p2;
    __nv_bfloat16 *Chi = (__nv_bfloat16 *)(C + nfloat), *Clo = Chi + nfloat;
    __nv_bfloat16 *Dhi = (__nv_bfloat16 *)(D + nfloat), *Dlo = Dhi + nfloat;
    if (bf3) {
        if (!c_split) {
            k_split_bf16<<<152 * 8, 256, 0, s>>>(C, Chi, Clo, nfloat);
            CKL("k_split_bf16");
        }
    } else {
        k_round_tf32<<<152 * 8, 256, 0, s>>>(C, nfloat);
        CKL("k_round_tf32");
    }
    const TcSetup t = tc_setup(h, C, D, nr, bf3);
    for (int l = 2; l <= h->lmax; ++l) {
        const LevelInfo &Lv = h->lev[l];
        const TcLevel P{Lv.off, l, h->lmax, h->nbox, (int)ncols, h->p2, tc_kblocks(h->p2), t.n, t.nsub, t.stages,
                        t.tcols, l < h->lmax ? 1 : 0, 0};
        const dim3 grid((unsigned)Lv.n, h->Jf + 1, (unsigned)t.ntile);
        if (bf3)
            k_m2l_tc<true><<<grid, 128, t.smem, s>>>(t.tmC, t.tmD, t.tmC2, t.tmD2, P, h->box_parent, h->box_key,
                                                     h->ff_start, h->ff_src, h->ff_off, h->Abf, h->Llbf, D, Dhi, Dlo,
                                                     h->tc_err, h->box_cbeg, h->box_cend);
        else
            k_m2l_tc<false><<<grid, 128, t.smem, s>>>(t.tmC, t.tmD, t.tmC2, t.tmD2, P, h->box_parent, h->box_key,
                                                      h->ff_start, h->ff_src, h->ff_off, h->Atc, h->Lltc, D, nullptr,
                                                      nullptr, h->tc_err, h->box_cbeg, h->box_cend);
        CKL("k_m2l_tc");
    }
}

// the offset-stationary few-column M2L runs for even p up to 10 (2 p^2 <= 200 rows of 16-byte
// aligned bf16 coefficient rows, N = 2 p^2 rounded up to 16 <= 256)
bool m2l_ofs_supported(const fmbem *h) { return h->p >= 4 && h->p <= 10 && h->p % 2 == 0; }

static int ofs_np(int p2) { return ((2 * p2 + 15) / 16) * 16; }

void build_ofs_tables(fmbem *h, cudaStream_t s) {
    const int p2 = h->p2, kb = tc_kblocks(p2), np = ofs_np(p2);
    const int64_t nmat = (int64_t)(h->J + 1) * (h->lmax + 1) * 316;
    const int64_t per = (int64_t)kb * np * KBLK;
    h->Aofs = dev_alloc(h, sizeof(__nv_bfloat16) * 2 * per * nmat);
    const int tb = 256;
    k_build_ofs_tables<<<(unsigned)((nmat * per + tb - 1) / tb), tb, 0, s>>>(h->T_m2l64, nmat, p2, np, kb,
                                                                            (__nv_bfloat16 *)h->Aofs);
    CKL("k_build_ofs_tables");
    const int64_t nch = h->h_chunk_first.empty() ? 0 : h->h_chunk_first.back();
    if (nch > 0) {
        h->chunk_pairs = dev_alloc(h, sizeof(int2) * 32 * nch);
        k_chunk_pairs<<<(unsigned)((nch * 32 + tb - 1) / tb), tb, 0, s>>>(nch, h->chunk_beg, h->chunk_cnt, h->pair_e,
                                                                         h->ff_src, (int2 *)h->chunk_pairs);
        CKL("k_chunk_pairs");
    }
    if (!h->tc_err) {
        h->tc_err = (int *)dev_alloc(h, sizeof(int));
        CK(cudaMemsetAsync(h->tc_err, 0, sizeof(int), s));
    }
}

// bf16 hi/lo split of the multipole expansions into the second half of their buffer (see
// run_m2l_tc) before the offset-stationary M2L reads them
void split_expansions_bf16(fmbem *h, float *C, int64_t nr, cudaStream_t s) {
    const int64_t nfloat = (int64_t)(h->J + 1) * h->nbox * 3 * nr * 2 * h->p2;
    __nv_bfloat16 *Chi = (__nv_bfloat16 *)(C + nfloat), *Clo = Chi + nfloat;
    k_split_bf16<<<152 * 8, 256, 0, s>>>(C, Chi, Clo, nfloat);
    CKL("k_split_bf16");
}

// one launch of k_m2l_ofs over every chunk of levels 2..l_max and every domain 0..Jf: the M2L
// of all levels at once (they read only the multipole expansions), into Y[d][CSR position]
// (Y + d * ofs_y_dom(h, nr) floats, the layout k_l2l_reduce reads with e_first = 0)
int64_t ofs_y_dom(const fmbem *h, int64_t nr) { return std::max<int64_t>(h->n_ff, 1) * 3 * nr * 2 * h->p2; }

// (levels l0..l1; reserve_sms SMs left free for work on other streams)
void run_m2l_ofs(fmbem *h, const float *C, float *Y, int64_t nr, cudaStream_t s, int l0, int l1, int reserve_sms) {
    if (h->lmax + 1 > OFS_MAX_LEVELS) throw fmbem_error{FMBEM_ERR_INVALID_ARGUMENT, "too many octree levels"};
    l0 = std::max(l0, 2);
    l1 = std::min(l1, h->lmax);
    if (l1 < l0) return;
    const int64_t c0 = h->h_chunk_first[l0], nch = h->h_chunk_first[l1 + 1] - c0;
    if (nch <= 0) return;
    const int p2 = h->p2, kb = tc_kblocks(p2), np = ofs_np(p2);
    const int64_t nfloat = (int64_t)(h->J + 1) * h->nbox * 3 * nr * 2 * p2;
    const __nv_bfloat16 *Chi = (const __nv_bfloat16 *)(C + nfloat), *Clo = Chi + nfloat;
    uint32_t tcols = 32;  // one accumulator; two are allocated (2 x 256 columns at most)
    while ((int)tcols < np) tcols <<= 1;
    OfsLevel P{};
    P.nbox = h->nbox;
    P.ncols = (int)(3 * nr);
    P.p2 = p2;
    P.kblocks = kb;
    P.np = np;
    P.lmax = h->lmax;
    P.ndom = h->Jf + 1;
    P.ppp = (int)(OFS_M / (3 * nr));
    P.tmem_cols = tcols;
    P.y_dom = ofs_y_dom(h, nr);
    for (int l = 0; l <= OFS_MAX_LEVELS; ++l)
        P.level_first[l] = l <= h->lmax + 1 ? std::max<int64_t>(h->h_chunk_first[std::max(l, 2)] - c0, 0) : nch;
    const size_t smem = (size_t)OFS_STAGES * (2 * OFS_M * 64 + 2 * (size_t)np * 64) + 1024;
    CK(cudaFuncSetAttribute(k_m2l_ofs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int64_t grid = std::min<int64_t>(nch * P.ndom, std::max(1, nsm - reserve_sms));  // one persistent CTA per SM
    k_m2l_ofs<<<(unsigned)grid, OFS_THREADS, smem, s>>>(P, c0, nch, h->chunk_cnt, h->chunk_off,
                                                         (const int2 *)h->chunk_pairs, Chi, Clo,
                                                         (const __nv_bfloat16 *)h->Aofs, Y, h->tc_err);
    CKL("k_m2l_ofs");
}
