// fmm.cu -- the fast multipole matrix-vector product of Section 2.2 (Steps 1-4).
//
// For every domain d (background d = 0 over all nodes with normal n0 = -n; scatterer j over its
// own nodes with normal +n) and every Cartesian component i, Eq. (2.12) is a scalar Helmholtz
// sum over the sources beta of domain d:
//   y_i(alpha) = sum_beta [ Q_i g_d(s_beta, s_alpha) + m_i . grad' g_d(s_beta, s_alpha) ],
//   Q = w q,  m_i = w [ v_i n' + (n'.v) e_i - n'_i v ],
// with v = T_d Phi and q = gamma_d Psi^(d) (Psi^(0) = -Psi): the bracket of Eq. (2.12) applied to
// v, [n' grad'g - (n'.grad'g) I - grad'g n'].v = grad'g . m / w, enters with a minus sign, and
// -(...)_i = m_i . grad'g / w.  Far interactions go through P2M -> M2M -> M2L -> L2L -> L2P
// (Eqs. 2.18-2.21, first term of 2.23); the sources in the node's own leaf and its Neighbor
// leaves are summed directly (second term of Eq. 2.23), beta = alpha excluded and replaced by the
// analytic self block A_self (Appendix B).
#include <algorithm>

#include <cstring>
#include <type_traits>

#include "fmbem_internal.cuh"

namespace {

inline unsigned nblk(int64_t n, int tb) { return (unsigned)((n + tb - 1) / tb); }

struct DomainConsts {  // per domain, device array
    c64 k, t, gamma;
};

// ---------------------------------------------------------------- source densities (a2)
// dens[side][r][i][6] = (w v, w q) for side 0 (background: v = Phi, q = -Psi) and side 1 (own
// scatterer j: v = T_j Phi, q = gamma_j Psi), nodes in sorted order.
// The bodies of k_prep, k_p2m, k_m2m, k_down and k_near take their block coordinates as
// arguments (bx, by, bz), so that the persistent kernel over many problems (k_batch) runs the same
// code on work items; the __global__ wrappers pass blockIdx.
template <typename R>
__device__ __forceinline__ void prep_body(int64_t N, int64_t nr, const c64 *x, const int32_t *perm, const double *nrm,
                                          const double *w, const int32_t *dom, const DomainConsts *dc, cx<R> *dens,
                                          int64_t bx, int64_t by, cx<R> *sj = nullptr) {
    int64_t i = bx * (int64_t)blockDim.x + threadIdx.x;
    int64_t r = by;
    if (i >= N) return;
    // in the working precision R: single precision rounds x, n, w and the constants first (the
    // densities are rounded to it in any case; the FP64 pipe would bound this kernel otherwise)
    const c64 *xi = x + (r * N + perm[i]) * 6;
    const R n[3] = {(R)nrm[3 * i], (R)nrm[3 * i + 1], (R)nrm[3 * i + 2]};
    const R wi = (R)w[i];
    const int j = dom[i];
    const cx<R> Phi[3] = {to<R>(xi[0]), to<R>(xi[1]), to<R>(xi[2])};
    const cx<R> Psi[3] = {to<R>(xi[3]), to<R>(xi[4]), to<R>(xi[5])};
    cx<R> *d0 = dens + ((0 * nr + r) * N + i) * 6;
    cx<R> *d1 = dens + ((1 * nr + r) * N + i) * 6;
    const cx<R> nP = n[0] * Phi[0] + n[1] * Phi[1] + n[2] * Phi[2];
    const cx<R> tn = to<R>(dc[j].t) * nP;
    const cx<R> gw = to<R>(dc[j].gamma) * wi;
    for (int q = 0; q < 3; ++q) {
        d0[q] = wi * Phi[q];
        d0[3 + q] = (-wi) * Psi[q];
        d1[q] = wi * (Phi[q] + n[q] * tn);
        d1[3 + q] = gw * Psi[q];
    }
    if (sj) sj[r * N + i] = wi * tn;  // v_1 - v_0 = s n (see k_near_ws)
}
template <typename R>
__global__ void k_prep(int64_t N, int64_t nr, const c64 *x, const int32_t *perm, const double *nrm, const double *w,
                       const int32_t *dom, const DomainConsts *dc, cx<R> *dens, cx<R> *sj) {
    prep_body<R>(N, nr, x, perm, nrm, w, dom, dc, dens, blockIdx.x, blockIdx.y, sj);
}

// The single-precision densities straight into the node-major layout below (k_dens_node_major's
// densS), for 32 k right-hand sides whose every consumer reads that layout (k_near_r, and P2M on
// the tensor cores, which forms the scatterer side from v_1 = v_0 + s n, q_1 = -gamma_j q_0):
// block = 8 nodes x 32 right-hand sides, lane = right-hand side, so that each warp stores one
// node's 2 KB row whole; arithmetic as in prep_body<float>
__global__ void __launch_bounds__(256) k_prep_node_major(int64_t N, int64_t nr, const c64 *x, const int32_t *perm,
                                                         const double *nrm, const double *w, const int32_t *dom,
                                                         const DomainConsts *dc, float4 *densS) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5), rb = blockIdx.y;
    if (i >= N) return;
    const int64_t r = rb * 32 + lane;
    const c64 *xi = x + (r * N + perm[i]) * 6;
    const float n[3] = {(float)nrm[3 * i], (float)nrm[3 * i + 1], (float)nrm[3 * i + 2]};
    const float wi = (float)w[i];
    const cx<float> Phi[3] = {to<float>(xi[0]), to<float>(xi[1]), to<float>(xi[2])};
    const cx<float> Psi[3] = {to<float>(xi[3]), to<float>(xi[4]), to<float>(xi[5])};
    const cx<float> nP = n[0] * Phi[0] + n[1] * Phi[1] + n[2] * Phi[2];
    const cx<float> tn = to<float>(dc[dom[i]].t) * nP;
    cx<float> v[3], q[3];
    for (int c = 0; c < 3; ++c) {
        v[c] = wi * Phi[c];
        q[c] = (-wi) * Psi[c];
    }
    const cx<float> sj = wi * tn;  // n . (v_1 - v_0)
    float4 *o = densS + ((rb * N + i) * 32 + lane) * 4;
    o[0] = make_float4(v[0].re, v[0].im, v[1].re, v[1].im);
    o[1] = make_float4(v[2].re, v[2].im, q[0].re, q[0].im);
    o[2] = make_float4(q[1].re, q[1].im, q[2].re, q[2].im);
    o[3] = make_float4(sj.re, sj.im, 0.f, 0.f);
}

// The single-precision densities node-major within blocks of 32 right-hand sides, for the
// lane-per-RHS near field (a source's 32 right-hand sides are contiguous):
// densS[block][node][32][4 float4] = (v0x, v0y), (v0z, q0x), (q0y, q0z), (s, 0) of the background
// side, with s = n . (v_1 - v_0) the scatterer side's jump along the normal (v_1 = v_0 + s n, see
// k_near_ws); grid (node tiles of 16, block), 32 x 16 entries through shared memory, written in
// whole rows.
__global__ void __launch_bounds__(256) k_dens_node_major(int64_t N, int64_t nr, const float4 *dens, const float4 *rec,
                                                         float4 *densS) {
    __shared__ float4 t[32][16 * 4 + 1];
    const int64_t i0 = (int64_t)blockIdx.x * 16, rb = blockIdx.y;
    const int ni = (int)min((int64_t)16, N - i0);
    for (int e = threadIdx.x; e < 32 * 16; e += blockDim.x) {  // (right-hand side rl, node il)
        const int rl = e / 16, il = e - rl * 16;
        if (il < ni) {
            const int64_t i = i0 + il;
            const float4 *a = dens + ((rb * 32 + rl) * N + i) * 3;         // background side
            const float4 *b = dens + ((nr + rb * 32 + rl) * N + i) * 3;    // scatterer side
            const float4 a0 = a[0], a1 = a[1], b0 = b[0], b1 = b[1];
            const float4 n1 = rec[3 * i + 1], n2 = rec[3 * i + 2];        // n = (n1.w, n2.x, n2.y)
            const float sre = n1.w * (b0.x - a0.x) + n2.x * (b0.z - a0.z) + n2.y * (b1.x - a1.x);
            const float sim = n1.w * (b0.y - a0.y) + n2.x * (b0.w - a0.w) + n2.y * (b1.y - a1.y);
            t[rl][il * 4] = a0;
            t[rl][il * 4 + 1] = a1;
            t[rl][il * 4 + 2] = a[2];
            t[rl][il * 4 + 3] = make_float4(sre, sim, 0.f, 0.f);
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 16 * 128; e += blockDim.x) {  // node il: 32 right-hand sides x 4 float4
        const int il = e / 128, k = e - il * 128, rl = k / 4, c = k - rl * 4;
        if (il < ni) densS[(rb * N + i0 + il) * 128 + k] = t[rl][il * 4 + c];
    }
}

// ---------------------------------------------------------------- P2M (Eqs. 2.18-2.19)
// grid (leaf, domain, rhs); thread per coefficient nm; C[d][g][3r+i][nm].  The dipole and monopole
// of component c enter as sum_k W_k(c) B_k with the node weights W_0 = q_c and
// W_k = v_c n_k - n_c v_k + (n.v) delta_ck (m_c . grad R + q_c R, Eq. 2.18); the block forms them
// once per node in shared memory, P2M_WN nodes at a time.
constexpr int P2M_WN = 64;
template <typename R>
__device__ __forceinline__ void p2m_body(int64_t g, int64_t N, int64_t nr, int p2, int64_t nbox,
                                         const int32_t *nbeg, const int32_t *nend, const int32_t *dom,
                                         const double *nrm, const cx<R> *dens, const cx<R> *Bp2m, cx<R> *C, int64_t bx,
                                         int by, int64_t bz) {
    __shared__ cx<R> W[P2M_WN][4][3];
    const int d = by;
    const int64_t r = bz;
    const int side = d == 0 ? 0 : 1;
    const R sg = d == 0 ? (R)-1 : (R)1;
    const int i0 = nbeg[g], i1 = nend[g];
    const int q = threadIdx.x;  // one thread per coefficient: blockDim >= p2
    cx<R> acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int ib = i0; ib < i1; ib += P2M_WN) {
        const int nk = min(P2M_WN, i1 - ib);
        __syncthreads();
        for (int e = threadIdx.x; e < 3 * nk; e += blockDim.x) {
            const int il = e / 3, c = e - 3 * il, i = ib + il;
            if (d > 0 && dom[i] != d) {
                for (int k = 0; k < 4; ++k) W[il][k][c] = {0, 0};
                continue;
            }
            const cx<R> *dn = dens + ((side * nr + r) * N + i) * 6;
            const cx<R> v[3] = {dn[0], dn[1], dn[2]};
            const R n[3] = {sg * (R)nrm[3 * i], sg * (R)nrm[3 * i + 1], sg * (R)nrm[3 * i + 2]};
            const cx<R> nv = n[0] * v[0] + n[1] * v[1] + n[2] * v[2];
            W[il][0][c] = dn[3 + c];
            const cx<R> vc = c == 0 ? v[0] : (c == 1 ? v[1] : v[2]);  // selects, not a local-memory index
            const R nc = c == 0 ? n[0] : (c == 1 ? n[1] : n[2]);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                cx<R> t = n[k] * vc - nc * v[k];
                if (k == c) t += nv;
                W[il][1 + k][c] = t;
            }
        }
        __syncthreads();
        if (q < p2)
            for (int il = 0; il < nk; ++il) {
                const cx<R> *B = Bp2m + ((int64_t)side * N + ib + il) * 4 * p2;
                const cx<R> b[4] = {B[q], B[p2 + q], B[2 * p2 + q], B[3 * p2 + q]};
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int k = 0; k < 4; ++k) cfma(acc[c], W[il][k][c], b[k]);
            }
    }
    if (q < p2)
        for (int c = 0; c < 3; ++c) C[(((int64_t)d * nbox + g) * 3 * nr + 3 * r + c) * p2 + q] = acc[c];
}
template <typename R>
__global__ void k_p2m(const int32_t *leaf_box, int64_t N, int64_t nr, int p2, int64_t nbox, const int32_t *nbeg,
                      const int32_t *nend, const int32_t *dom, const double *nrm, const cx<R> *dens, const cx<R> *Bp2m,
                      cx<R> *C) {
    p2m_body<R>(leaf_box[blockIdx.x], N, nr, p2, nbox, nbeg, nend, dom, nrm, dens, Bp2m, C, blockIdx.x, blockIdx.y,
                blockIdx.z);
}

// P2M for blocks of RB right-hand sides: the basis values of a (node, coefficient) are read once
// and applied to every right-hand side of the block; grid (leaf, domain, rhs block), thread per
// coefficient; same arithmetic, order and layout as k_p2m
template <typename R, int RB>
__global__ void k_p2m_rb(const int32_t *leaf_box, int64_t N, int64_t nr, int p2, int64_t nbox, const int32_t *nbeg,
                         const int32_t *nend, const int32_t *dom, const double *nrm, const cx<R> *dens,
                         const cx<R> *Bp2m, cx<R> *C) {
    const int64_t g = leaf_box[blockIdx.x];
    const int d = blockIdx.y;
    const int64_t rb0 = (int64_t)blockIdx.z * RB;
    const int nrb = (int)min((int64_t)RB, nr - rb0);
    const int side = d == 0 ? 0 : 1;
    const R sg = d == 0 ? (R)-1 : (R)1;
    const int i0 = nbeg[g], i1 = nend[g];
    for (int q = threadIdx.x; q < p2; q += blockDim.x) {
        cx<R> acc[RB][3];
#pragma unroll
        for (int rr = 0; rr < RB; ++rr)
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[rr][c] = {0, 0};
        for (int i = i0; i < i1; ++i) {
            if (d > 0 && dom[i] != d) continue;
            const R n[3] = {sg * (R)nrm[3 * i], sg * (R)nrm[3 * i + 1], sg * (R)nrm[3 * i + 2]};
            const cx<R> *B = Bp2m + ((int64_t)side * N + i) * 4 * p2;
            const cx<R> b0 = B[q], G[3] = {B[p2 + q], B[2 * p2 + q], B[3 * p2 + q]};
            const cx<R> nG = n[0] * G[0] + n[1] * G[1] + n[2] * G[2];
#pragma unroll
            for (int rr = 0; rr < RB; ++rr) {
                if (rr >= nrb) break;
                const cx<R> *dn = dens + ((side * nr + rb0 + rr) * N + i) * 6;
                const cx<R> v[3] = {dn[0], dn[1], dn[2]}, qq[3] = {dn[3], dn[4], dn[5]};
                const cx<R> nv = n[0] * v[0] + n[1] * v[1] + n[2] * v[2];
                const cx<R> vG = v[0] * G[0] + v[1] * G[1] + v[2] * G[2];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    // m_c . G = v_c (n.G) + (n.v) G_c - n_c (v.G), plus the monopole q_c R
                    const cx<R> t = v[c] * nG + nv * G[c] - n[c] * vG + qq[c] * b0;
                    acc[rr][c] += t;
                }
            }
        }
#pragma unroll
        for (int rr = 0; rr < RB; ++rr) {
            if (rr >= nrb) break;
            for (int c = 0; c < 3; ++c)
                C[(((int64_t)d * nbox + g) * 3 * nr + 3 * (rb0 + rr) + c) * p2 + q] = acc[rr][c];
        }
    }
}

// P2M for many right-hand sides as a register-tiled product.  For one leaf and domain,
//   C[col][q] = sum over (node i, k = 0..3) of B_k(i, q) W_k(i, col),
// with B_0 = R_n^{-m} (monopole) and B_{1..3} = grad R (the P2M basis rows) and, for column col =
// 3 r + c (right-hand side r, component c), W_0 = q_c and W_k = v_c n_k + (n.v) delta_ck - n_c v_k
// (so that sum_k W_k B_k = m_c . grad R + q_c R, Eqs. 2.18-2.19).  Nodes are taken P2M_KC at a time:
// the block stages their basis rows and weights in shared memory, and each thread accumulates a
// tile of (coefficient, column) outputs: PT pairs of coefficients 2 (rg + nrg a) + {0, 1}
// (a = 0..PT-1; the lanes of a warp read consecutive pairs, free of bank conflicts) and columns
// 4 cgp .. 4 cgp + 3: a 4 x 4 tile (8 x 4 measured slower: fewer resident warps to hide the
// staging's global loads).  Grid (leaf, domain, tile of MT columns); MT = 96 (32 right-hand
// sides) in single precision, 48 in double (register budget).
constexpr int P2M_KC = 8;   // nodes per shared-memory chunk
template <typename R>
__host__ __device__ constexpr int p2m_mt() { return sizeof(R) == 4 ? 96 : 48; }
template <typename R>
__host__ __device__ constexpr int p2m_pt() { return 2; }
template <typename R>
__global__ void k_p2m_gemm(const int32_t *leaf_box, int64_t N, int64_t nr, int p2, int64_t nbox, const int32_t *nbeg,
                           const int32_t *nend, const int32_t *dom, const double *nrm, const cx<R> *dens,
                           const cx<R> *Bp2m, cx<R> *C) {
    constexpr int MT = p2m_mt<R>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<R> *Bs = reinterpret_cast<cx<R> *>(smem_raw);  // [4 P2M_KC][p2]
    cx<R> *Ws = Bs + 4 * P2M_KC * p2;                   // [4 P2M_KC][MT]
    const int64_t g = leaf_box[blockIdx.x];
    const int d = blockIdx.y;
    const int ncols = (int)(3 * nr), col0 = blockIdx.z * MT;
    const int nh = min(MT, ncols - col0);
    const int side = d == 0 ? 0 : 1;
    const R sg = d == 0 ? (R)-1 : (R)1;
    const int i0 = nbeg[g], i1 = nend[g];
    constexpr int PT = p2m_pt<R>();  // coefficient pairs per thread
    const int nrg = (p2 + 2 * PT - 1) / (2 * PT);
    const int rg = threadIdx.x % nrg, cgp = threadIdx.x / nrg;
    const int c0 = 4 * cgp;
    const bool owner = cgp < MT / 4;
    cx<R> acc[2 * PT][4];
#pragma unroll
    for (int a = 0; a < 2 * PT; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = {0, 0};
    for (int ib = i0; ib < i1; ib += P2M_KC) {
        const int nk = min(P2M_KC, i1 - ib);
        __syncthreads();
        if (sizeof(R) == 4 && (p2 & 1) == 0) {  // pairs of coefficients as 16-byte words
            const int hp = p2 >> 1;
            for (int e = threadIdx.x; e < 4 * P2M_KC * hp; e += blockDim.x) {
                const int kk = e / hp, q2 = e - kk * hp, il = kk >> 2;
                const int i = ib + il;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (il < nk && (d == 0 || dom[i] == d))
                    v = reinterpret_cast<const float4 *>(Bp2m + ((int64_t)side * N + i) * 4 * p2 + (int64_t)(kk & 3) * p2)[q2];
                reinterpret_cast<float4 *>(Bs + kk * p2)[q2] = v;
            }
        } else {
            for (int e = threadIdx.x; e < 4 * P2M_KC * p2; e += blockDim.x) {
                const int kk = e / p2, q = e - kk * p2, il = kk >> 2;
                const int i = ib + il;
                cx<R> v = {0, 0};
                if (il < nk && (d == 0 || dom[i] == d)) v = Bp2m[((int64_t)side * N + i) * 4 * p2 + (int64_t)(kk & 3) * p2 + q];
                Bs[e] = v;
            }
        }
        for (int e = threadIdx.x; e < P2M_KC * (MT / 3); e += blockDim.x) {
            const int il = e / (MT / 3), rl = e - il * (MT / 3);
            const int i = ib + il, col = 3 * rl;
            cx<R> w[4][3];
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int c = 0; c < 3; ++c) w[k][c] = {0, 0};
            if (il < nk && col < nh && (d == 0 || dom[i] == d)) {
                const int64_t r = (col0 + col) / 3;
                const cx<R> *dn = dens + ((side * nr + r) * N + i) * 6;
                const cx<R> v[3] = {dn[0], dn[1], dn[2]};
                const R n[3] = {sg * (R)nrm[3 * i], sg * (R)nrm[3 * i + 1], sg * (R)nrm[3 * i + 2]};
                const cx<R> nv = n[0] * v[0] + n[1] * v[1] + n[2] * v[2];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    w[0][c] = dn[3 + c];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        cx<R> t = n[k] * v[c] - n[c] * v[k];
                        if (k == c) t += nv;
                        w[1 + k][c] = t;
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int c = 0; c < 3; ++c) Ws[(4 * il + k) * MT + col + c] = w[k][c];
        }
        __syncthreads();
        // single precision with p2 even: the coefficient pairs and the four columns as 16-byte words
        // (Bs rows and Ws column groups then start 16-byte aligned)
        const bool vec = sizeof(R) == 4 && (p2 & 1) == 0;
        if (owner) {
            for (int kk = 0; kk < 4 * nk; ++kk) {
                cx<R> bq[2 * PT], wc[4];
                if (vec) {
#pragma unroll
                    for (int a = 0; a < PT; ++a) {
                        const int q = 2 * (rg + nrg * a);
                        const float4 v = q < p2 ? reinterpret_cast<const float4 *>(Bs + kk * p2)[q >> 1]
                                                : make_float4(0.f, 0.f, 0.f, 0.f);
                        bq[2 * a] = cx<R>{(R)v.x, (R)v.y};
                        bq[2 * a + 1] = cx<R>{(R)v.z, (R)v.w};
                    }
                    const float4 w0 = reinterpret_cast<const float4 *>(Ws + kk * MT + c0)[0];
                    const float4 w1 = reinterpret_cast<const float4 *>(Ws + kk * MT + c0)[1];
                    wc[0] = cx<R>{(R)w0.x, (R)w0.y};
                    wc[1] = cx<R>{(R)w0.z, (R)w0.w};
                    wc[2] = cx<R>{(R)w1.x, (R)w1.y};
                    wc[3] = cx<R>{(R)w1.z, (R)w1.w};
                } else {
#pragma unroll
                    for (int a = 0; a < PT; ++a) {
                        const int q = 2 * (rg + nrg * a);
                        bq[2 * a] = q < p2 ? Bs[kk * p2 + q] : cx<R>{0, 0};
                        bq[2 * a + 1] = q + 1 < p2 ? Bs[kk * p2 + q + 1] : cx<R>{0, 0};
                    }
#pragma unroll
                    for (int b = 0; b < 4; ++b) wc[b] = Ws[kk * MT + c0 + b];
                }
#pragma unroll
                for (int a = 0; a < 2 * PT; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) cfma(acc[a][b], bq[a], wc[b]);
            }
        }
    }
    if (owner)
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if (c0 + b < nh)
#pragma unroll
                for (int a = 0; a < 2 * PT; ++a) {
                    const int q = 2 * (rg + nrg * (a >> 1)) + (a & 1);
                    if (q < p2) C[(((int64_t)d * nbox + g) * ncols + col0 + c0 + b) * p2 + q] = acc[a][b];
                }
}

// ---------------------------------------------------------------- translation apply helper
// acc[cc] += sum_c T[c][r] X[cc][c] for the thread's output row r; X in shared memory
template <typename R, int CC>
__device__ __forceinline__ void apply_T(const cx<R> *__restrict__ T, const cx<R> *X, int p2, int r, int ncol, cx<R> *acc) {
#pragma unroll 4
    for (int c = 0; c < p2; ++c) {
        cx<R> t = T[(int64_t)c * p2 + r];
#pragma unroll
        for (int cc = 0; cc < CC; ++cc)
            if (cc < ncol) cfma(acc[cc], t, X[cc * p2 + c]);
    }
}

constexpr int CC = 6;  // columns per CTA in the translation kernels
static_assert(CC == BATCH_CHUNK_COLS, "the batch's column chunks are the translation kernels'");

// M2M (Eq. 2.20): parent multipole = sum over children S|S(child octant) child multipole
// grid (parent box at level l-1, domain, chunk of NC columns); NC = 3 for one right-hand side,
// so that no multiply-add of the unrolled column loop is issued for an absent column
template <typename R, int NC>
__device__ __forceinline__ void m2m_body(int64_t par_off, int l, int lmax, int64_t nr, int p2, int64_t nbox,
                                         const int32_t *cbeg, const int32_t *cend, const uint64_t *key, const cx<R> *Tmm,
                                         cx<R> *C, int64_t bx, int by, int bz) {
    extern __shared__ unsigned char smem_raw[];
    cx<R> *X = reinterpret_cast<cx<R> *>(smem_raw);
    int64_t g = par_off + bx;
    if (cbeg[g] == cend[g]) return;  // a leaf of an adaptive tree: its multipole expansion is P2M's
    int d = by;
    int col0 = bz * NC;
    int ncol = min(NC, (int)(3 * nr) - col0);
    int r = threadIdx.x;
    cx<R> acc[NC];
    for (int cc = 0; cc < NC; ++cc) acc[cc] = {0, 0};
    for (int ch = cbeg[g]; ch < cend[g]; ++ch) {
        __syncthreads();
        for (int e = threadIdx.x; e < ncol * p2; e += blockDim.x)
            X[e] = C[(((int64_t)d * nbox + ch) * 3 * nr + col0 + e / p2) * p2 + e % p2];
        __syncthreads();
        int o = (int)(key[ch] & 7);
        if (r < p2) apply_T<R, NC>(Tmm + oct_matrix(d, l, o, lmax) * p2 * p2, X, p2, r, ncol, acc);
    }
    if (r < p2)
        for (int cc = 0; cc < ncol; ++cc) C[(((int64_t)d * nbox + g) * 3 * nr + col0 + cc) * p2 + r] = acc[cc];
}
template <typename R, int NC>
__global__ void k_m2m(int64_t par_off, int l, int lmax, int64_t nr, int p2, int64_t nbox, const int32_t *cbeg,
                      const int32_t *cend, const uint64_t *key, const cx<R> *Tmm, cx<R> *C) {
    m2m_body<R, NC>(par_off, l, lmax, nr, p2, nbox, cbeg, cend, key, Tmm, C, blockIdx.x, blockIdx.y, blockIdx.z);
}

// M2L + L2L (Eq. 2.21): D(l,q) = R|R D(parent) + sum_{FF(l,q)} S|R C(source)
template <typename R>
__device__ __forceinline__ void down_body(int64_t off, int l, int lmax, int64_t nr, int p2, int64_t nbox,
                                          const int32_t *parent, const uint64_t *key, const int32_t *ff_start,
                                          const int32_t *ff_src, const int16_t *ff_off, const cx<R> *Tm2l,
                                          const cx<R> *Tll, const cx<R> *C, cx<R> *D, int64_t bx, int by, int bz) {
    extern __shared__ unsigned char smem_raw[];
    cx<R> *X = reinterpret_cast<cx<R> *>(smem_raw);
    int64_t g = off + bx;
    int d = by;
    int col0 = bz * CC;
    int ncol = min(CC, (int)(3 * nr) - col0);
    int r = threadIdx.x;
    cx<R> acc[CC];
    for (int cc = 0; cc < CC; ++cc) acc[cc] = {0, 0};
    if (l >= 3) {
        int64_t P = parent[g];
        for (int e = threadIdx.x; e < ncol * p2; e += blockDim.x)
            X[e] = D[(((int64_t)d * nbox + P) * 3 * nr + col0 + e / p2) * p2 + e % p2];
        __syncthreads();
        int o = (int)(key[g] & 7);
        if (r < p2) apply_T<R, CC>(Tll + oct_matrix(d, l, o, lmax) * p2 * p2, X, p2, r, ncol, acc);
    }
    for (int e0 = ff_start[g]; e0 < ff_start[g + 1]; ++e0) {
        __syncthreads();
        int src = ff_src[e0];
        for (int e = threadIdx.x; e < ncol * p2; e += blockDim.x)
            X[e] = C[(((int64_t)d * nbox + src) * 3 * nr + col0 + e / p2) * p2 + e % p2];
        __syncthreads();
        if (r < p2) apply_T<R, CC>(Tm2l + m2l_matrix(d, l, ff_off[e0], lmax) * p2 * p2, X, p2, r, ncol, acc);
    }
    if (r < p2)
        for (int cc = 0; cc < ncol; ++cc) D[(((int64_t)d * nbox + g) * 3 * nr + col0 + cc) * p2 + r] = acc[cc];
}
template <typename R>
__global__ void k_down(int64_t off, int l, int lmax, int64_t nr, int p2, int64_t nbox, const int32_t *parent,
                       const uint64_t *key, const int32_t *ff_start, const int32_t *ff_src, const int16_t *ff_off,
                       const cx<R> *Tm2l, const cx<R> *Tll, const cx<R> *C, cx<R> *D) {
    down_body<R>(off, l, lmax, nr, p2, nbox, parent, key, ff_start, ff_src, ff_off, Tm2l, Tll, C, D, blockIdx.x,
                 blockIdx.y, blockIdx.z);
}

// M2L on a chunk of FF pairs that share one offset o (S|R part of Eq. 2.21): the chunk's
// translation matrix is staged once in shared memory and applied to every pair of the chunk,
// Y[e][col][r] = sum_k T_o[k][r] C[src(e)][col0 + col][k], stored at the pair's CSR position e so
// that k_l2l_reduce can sum each target's pairs in a fixed order.
// Threads: rows_pad (= p2 rounded up to a warp multiple) x cg column groups; a warp shares its
// columns, so the gathered inputs are read as shared-memory broadcasts.
// TSM: the translation matrix is staged in shared memory; otherwise (large p in double
// precision) it is read from L2, coalesced across the rows, and shared memory holds the columns.
template <typename R, int MAXC, bool TSM>
__global__ void k_m2l_chunks(int64_t chunk0, int l, int lmax, int d0, int64_t nr, int p2, int64_t nbox, int col0,
                             int ncol, int pc, int cg, const int32_t *chunk_beg, const int32_t *chunk_cnt,
                             const int16_t *chunk_off, const int32_t *pair_e, const int32_t *ff_src,
                             const cx<R> *Tm2l, const cx<R> *C, cx<R> *Y, int64_t e_first, int64_t y_dstride) {
    const int d = d0 + (int)blockIdx.y;  // domain: one grid row per domain, each with its own Y block
    Y += (int64_t)blockIdx.y * y_dstride;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<R> *Tsh = reinterpret_cast<cx<R> *>(smem_raw);  // [k][r]
    cx<R> *Xs = Tsh + (TSM ? p2 * p2 : 0);              // [pair * ncol + col][k]
    const int64_t ck = chunk0 + blockIdx.x;
    const int beg = chunk_beg[ck], cnt = chunk_cnt[ck];
    const cx<R> *__restrict__ T = Tm2l + m2l_matrix(d, l, chunk_off[ck], lmax) * p2 * p2;
    if (TSM)
        for (int i = threadIdx.x; i < p2 * p2; i += blockDim.x) Tsh[i] = T[i];
    const cx<R> *Ts = TSM ? Tsh : T;
    const int rows_pad = blockDim.x / cg;
    const int r = threadIdx.x % rows_pad, grp = threadIdx.x / rows_pad;
    // every column group owns exactly MAXC columns; columns past the sub-batch are zero-filled,
    // so the inner product loop carries no per-column predicate
    const int ncap = cg * MAXC;
    for (int b0 = 0; b0 < cnt; b0 += pc) {
        const int np = min(pc, cnt - b0);
        const int nct = np * ncol;
        __syncthreads();
        for (int i = threadIdx.x; i < ncap * p2; i += blockDim.x) {
            int j = i / p2, k = i - j * p2;
            cx<R> v = {0, 0};
            if (j < nct) {
                int pr = j / ncol, col = j - pr * ncol;
                int src = ff_src[pair_e[beg + b0 + pr]];
                v = C[(((int64_t)d * nbox + src) * 3 * nr + col0 + col) * p2 + k];
            }
            Xs[i] = v;
        }
        __syncthreads();
        const int j0 = grp * MAXC, nj = min(MAXC, nct - j0);
        if (r < p2 && nj > 0) {
            cx<R> acc[MAXC];
#pragma unroll
            for (int q = 0; q < MAXC; ++q) acc[q] = {0, 0};
            const cx<R> *xb = Xs + j0 * p2;
#pragma unroll 2
            for (int k = 0; k < p2; ++k) {
                cx<R> t = Ts[k * p2 + r];
#pragma unroll
                for (int q = 0; q < MAXC; ++q) cfma(acc[q], t, xb[q * p2 + k]);
            }
#pragma unroll
            for (int q = 0; q < MAXC; ++q)
                if (q < nj) {
                    int j = j0 + q, pr = j / ncol, col = j - pr * ncol;
                    int64_t e = pair_e[beg + b0 + pr];
                    Y[((e - e_first) * ncol + col) * p2 + r] = acc[q];
                }
        }
    }
}

// M2L on offset chunks in rotation form (S|R of Eq. 2.21 factored as T_o = B_o Z_{|t|} A_o):
// C' = A_o C rotates each degree block into the frame whose z axis is the translation,
// D' = Z C' translates along z (block-diagonal in the order m), Y = B_o D' rotates back.
// A_o and B_o are a diagonal azimuthal phase and a real polar rotation per degree.  A rotation
// about y commutes with the mirror y -> -y, which maps Y_n^m to Y_n^{-m} in this basis (the
// normalisation depends on |m| only), so a polar block D obeys D[-m'][-m] = D[m'][m]; the coaxial
// translation commutes with it too, so Z^{-m} = Z^m.  In the folded coordinates
//   a_0 = x_0, a_m = x_m + x_{-m}, b_m = x_m - x_{-m}  (m >= 1)
// a polar block splits into two half-size blocks, (D[m'][m] + D[m'][-m]) acting on a and
// (D[m'][m] - D[m'][-m]) acting on b, and Z^m acts on both halves; the back rotation returns
// P +- Q to the orders +-m'.  Per column this costs sum_n ((n+1)^2 + n^2) real-by-complex products
// per rotation instead of sum_n (2n+1)^2, and sum_m (p-|m|)^2 complex products for Z.  The folded
// blocks (pack_rot_factors) and Z are staged in shared memory once per chunk; a thread owns one
// folded coefficient (degree n, slot s in 0..2n: a_s for s <= n, b_{s-n} after) for MAXC columns.
__device__ __host__ __forceinline__ int rot_off(int n) { return n * (2 * n * n + 1) / 3; }  // folded blocks before degree n
// The k-th folded slot (index n^2 + s) in order of its polar row length t = 1..p (stages 1 and 3):
// length t holds the t a-slots of degree t-1 and the t b-slots of degree t.
__device__ __forceinline__ int slot_by_rowlen(int p, int k) {
    for (int t = 1; t <= p; ++t) {
        if (k < t) return (t - 1) * (t - 1) + k;
        k -= t;
        if (t < p) {
            if (k < t) return t * t + t + 1 + k;
            k -= t;
        }
    }
    return 0;
}
// The k-th folded slot in order of its coaxial row length p - |m| (stage 2), longest first: order
// 0 holds the a-slots of degrees 0..p-1, order m >= 1 the a- and b-slots of degrees m..p-1.
__device__ __forceinline__ int slot_by_order(int p, int k) {
    for (int am = 0; am < p; ++am) {
        const int cnt = p - am;
        if (k < cnt) return (am + k) * (am + k) + am;
        k -= cnt;
        if (am > 0) {
            if (k < cnt) return (am + k) * (am + k) + (am + k) + am;
            k -= cnt;
        }
    }
    return 0;
}
template <typename R, int MAXC>
__global__ void __launch_bounds__(512) k_m2l_rot(int64_t chunk0, int l, int lmax, int d0, int64_t nr, int p, int64_t nbox,
                                                 int col0, int ncol, int pc, int cg, const int32_t *chunk_beg,
                                                 const int32_t *chunk_cnt, const int16_t *chunk_off, const int32_t *pair_e,
                                                 const int32_t *ff_src, const int8_t *tidx, int n_tlen, const R *RD,
                                                 const cx<R> *RP, const cx<R> *RZ, const cx<R> *C, cx<R> *Y,
                                                 int64_t e_first, int64_t y_dstride) {
    const int d = d0 + (int)blockIdx.y;  // domain: one grid row per domain, each with its own Y block
    Y += (int64_t)blockIdx.y * y_dstride;
    const int p2 = p * p;
    const int nrot = rot_off(p), ncoax = p * (2 * p * p + 1) / 3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *Df = reinterpret_cast<R *>(smem_raw);  // forward polar rotation, folded real blocks
    R *Db = Df + nrot;                         // back polar rotation, folded
    cx<R> *Pf = reinterpret_cast<cx<R> *>(Db + nrot);  // forward azimuthal phases [p2]
    cx<R> *Pb = Pf + p2;                                // back azimuthal phases [p2]
    cx<R> *Zb = Pb + p2;
    const int ncap = cg * MAXC;
    cx<R> *X = Zb + ncoax;       // [ncap][p2]
    cx<R> *U = X + ncap * p2;    // [ncap][p2]
    short2 *itab = reinterpret_cast<short2 *>(U + ncap * p2);  // fold items: (degree n, order m >= 0)
    const int nitem = p * (p + 1) / 2;
    for (int i = threadIdx.x; i < nitem; i += blockDim.x) {
        int n = 0;
        while ((n + 1) * (n + 2) / 2 <= i) ++n;
        itab[i] = make_short2((short)n, (short)(i - n * (n + 1) / 2));
    }
    const int64_t ck = chunk0 + blockIdx.x;
    const int beg = chunk_beg[ck], cnt = chunk_cnt[ck];
    const int o = chunk_off[ck];
    // packed factors of this offset (pack_rot_factors) and the coaxial blocks of its length
    const R *D2 = RD + (int64_t)o * 2 * nrot;
    const cx<R> *P2 = RP + (int64_t)o * 2 * p2;
    const cx<R> *Z = RZ + (((int64_t)d * (lmax + 1) + l) * n_tlen + tidx[o]) * ncoax;
    for (int i = threadIdx.x; i < 2 * nrot; i += blockDim.x) Df[i] = D2[i];
    for (int i = threadIdx.x; i < 2 * p2; i += blockDim.x) Pf[i] = P2[i];
    for (int i = threadIdx.x; i < ncoax; i += blockDim.x) Zb[i] = Z[i];
    const int rows_pad = blockDim.x / cg;
    const int r = threadIdx.x % rows_pad, grp = threadIdx.x / rows_pad;
    int rn = (int)sqrtf((float)r);  // the natural coefficient (rn, r - rn^2 - rn) of the unfold
    while (rn * rn > r) --rn;
    while ((rn + 1) * (rn + 1) <= r) ++rn;
    // the folded slots of the three stages, ordered by row length so that the lanes of a warp
    // run loops of (nearly) equal length; odd column groups take the order reversed, so that a
    // warp straddling two groups still meets similar lengths
    const int kk = (grp & 1) ? p2 - 1 - r : r;
    const int r13 = r < p2 ? slot_by_rowlen(p, kk) : 0, r2 = r < p2 ? slot_by_order(p, kk) : 0;
    int n1 = (int)sqrtf((float)r13);
    while (n1 * n1 > r13) --n1;
    while ((n1 + 1) * (n1 + 1) <= r13) ++n1;
    const int sl1 = r13 - n1 * n1;
    const bool plus1 = sl1 <= n1;
    const int am1 = plus1 ? sl1 : sl1 - n1;
    // folded polar rows of the stage 1 and 3 slot: a-block rows (n+1 long) or b-block rows (n long)
    const int foff = rot_off(n1) + (plus1 ? sl1 * (n1 + 1) : (n1 + 1) * (n1 + 1) + (am1 - 1) * n1);
    const int flen = plus1 ? n1 + 1 : n1, fin = plus1 ? n1 * n1 : n1 * n1 + n1 + 1;
    int n2 = (int)sqrtf((float)r2);
    while (n2 * n2 > r2) --n2;
    while ((n2 + 1) * (n2 + 1) <= r2) ++n2;
    const bool plus2 = r2 - n2 * n2 <= n2;
    const int am2 = plus2 ? r2 - n2 * n2 : r2 - n2 * n2 - n2;
    // coaxial block of the stage 2 slot's order am2 (Z^{-m} = Z^m): row n' - am2, columns n - am2
    int zbase = 0;
    for (int m = -(p - 1); m < am2; ++m) zbase += (p - abs(m)) * (p - abs(m));
    const int zw = p - am2;
    for (int b0 = 0; b0 < cnt; b0 += pc) {
        const int np = min(pc, cnt - b0);
        const int nct = np * ncol;
        __syncthreads();
        // load with the forward azimuthal phase and fold, one item (n, m >= 0) per thread: with
        // the phase e of order m (that of -m is its conjugate, checked at packing),
        // a_m = x_m e + x_{-m} conj(e) = Re(e) (x_m + x_{-m}) + i Im(e) (x_m - x_{-m}) and
        // b_m = x_m e - x_{-m} conj(e) = Re(e) (x_m - x_{-m}) + i Im(e) (x_m + x_{-m})
        for (int i = threadIdx.x; i < ncap * nitem; i += blockDim.x) {
            const int j = i / nitem, it = i - j * nitem;
            const short2 tn = itab[it];
            const int n = tn.x, mm = tn.y, c0 = n * n + n;
            cx<R> va = {0, 0}, vb = {0, 0};
            if (j < nct) {
                const int pr = j / ncol, c = j - pr * ncol;
                const cx<R> *src = C + (((int64_t)d * nbox + ff_src[pair_e[beg + b0 + pr]]) * 3 * nr + col0 + c) * p2;
                if (mm == 0) {
                    va = src[c0] * Pf[c0];
                } else {
                    const cx<R> xp = src[c0 + mm], xm = src[c0 - mm], e = Pf[c0 + mm];
                    const cx<R> sum = xp + xm, dif = xp - xm;
                    va = cx<R>{e.re * sum.re - e.im * dif.im, e.re * sum.im + e.im * dif.re};
                    vb = cx<R>{e.re * dif.re - e.im * sum.im, e.re * dif.im + e.im * sum.re};
                }
            }
            X[j * p2 + n * n + mm] = va;
            if (mm > 0) X[j * p2 + n * n + n + mm] = vb;
        }
        __syncthreads();
        const int j0 = grp * MAXC, nj = min(MAXC, nct - j0);
        cx<R> acc[MAXC];
        // stage 1: folded polar rotation into the translation frame
        if (r < p2 && nj > 0) {
#pragma unroll
            for (int q = 0; q < MAXC; ++q) acc[q] = {0, 0};
            const R *a = Df + foff;
            for (int jj = 0; jj < flen; ++jj) {
                const R t = a[jj];
#pragma unroll
                for (int q = 0; q < MAXC; ++q) {
                    const cx<R> xv = X[(j0 + q) * p2 + fin + jj];
                    acc[q].re = fma(t, xv.re, acc[q].re);
                    acc[q].im = fma(t, xv.im, acc[q].im);
                }
            }
#pragma unroll
            for (int q = 0; q < MAXC; ++q) U[(j0 + q) * p2 + r13] = acc[q];
        }
        __syncthreads();
        // stage 2: coaxial translation along z of order am2, on the a (or b) half
        if (r < p2 && nj > 0) {
#pragma unroll
            for (int q = 0; q < MAXC; ++q) acc[q] = {0, 0};
            const cx<R> *z = Zb + zbase + (n2 - am2) * zw;
            for (int jj = 0; jj < zw; ++jj) {
                const cx<R> t = z[jj];
                const int n = am2 + jj;
                const int src = n * n + (plus2 ? am2 : n + am2);
#pragma unroll
                for (int q = 0; q < MAXC; ++q) cfma(acc[q], t, U[(j0 + q) * p2 + src]);
            }
#pragma unroll
            for (int q = 0; q < MAXC; ++q) X[(j0 + q) * p2 + r2] = acc[q];
        }
        __syncthreads();
        // stage 3: folded polar rotation back: P (a half) and Q (b half)
        if (r < p2 && nj > 0) {
#pragma unroll
            for (int q = 0; q < MAXC; ++q) acc[q] = {0, 0};
            const R *bb = Db + foff;
            for (int jj = 0; jj < flen; ++jj) {
                const R t = bb[jj];
#pragma unroll
                for (int q = 0; q < MAXC; ++q) {
                    const cx<R> xv = X[(j0 + q) * p2 + fin + jj];
                    acc[q].re = fma(t, xv.re, acc[q].re);
                    acc[q].im = fma(t, xv.im, acc[q].im);
                }
            }
#pragma unroll
            for (int q = 0; q < MAXC; ++q) U[(j0 + q) * p2 + r13] = acc[q];
        }
        __syncthreads();
        // unfold, y_{+-m} = P_m +- Q_m, apply the back azimuthal phase and store at the pairs'
        // CSR positions; here thread r owns the natural coefficient (rn, m = r - rn^2 - rn)
        if (r < p2 && nj > 0) {
            const int m = r - rn * rn - rn, mm = abs(m);
            const cx<R> ph = Pb[r];
#pragma unroll
            for (int q = 0; q < MAXC; ++q)
                if (q < nj) {
                    const cx<R> *u = U + (j0 + q) * p2 + rn * rn;
                    cx<R> v = u[mm];
                    if (mm > 0) v = m > 0 ? v + u[rn + mm] : v - u[rn + mm];
                    const int j = j0 + q, pr = j / ncol, c = j - pr * ncol;
                    const int64_t e = pair_e[beg + b0 + pr];
                    Y[((e - e_first) * ncol + c) * p2 + r] = v * ph;
                }
        }
    }
}

// The same folded rotation form with the columns across the lanes (double precision, where the
// FP64 pipe is the bound): the block takes up to ROTC_N columns (pc pairs x ncol) per pass and a
// warp works one folded slot at a time with one column per lane, so that all lanes of a warp run
// loops of the same length and read the broadcast table entries; the warps deal the slots,
// ordered by loop length, in snake order.  Same arguments and results as k_m2l_rot (cg unused).
constexpr int ROTC_N = 32;      // columns per pass (one per lane)
constexpr int ROTC_S = ROTC_N + 1;  // row stride of the staged coefficients (conflict-free both ways)
constexpr int ROTC_WARPS = 16;
template <typename R>
__global__ void __launch_bounds__(32 * ROTC_WARPS) k_m2l_rot_cols(
    int64_t chunk0, int l, int lmax, int d0, int64_t nr, int p, int64_t nbox, int col0, int ncol, int pc, int cg,
    const int32_t *chunk_beg, const int32_t *chunk_cnt, const int16_t *chunk_off, const int32_t *pair_e,
    const int32_t *ff_src, const int8_t *tidx, int n_tlen, const R *RD, const cx<R> *RP, const cx<R> *RZ,
    const cx<R> *C, cx<R> *Y, int64_t e_first, int64_t y_dstride) {
    const int d = d0 + (int)blockIdx.y;  // domain: one grid row per domain, each with its own Y block
    Y += (int64_t)blockIdx.y * y_dstride;
    const int p2 = p * p;
    const int nrot = rot_off(p), ncoax = p * (2 * p * p + 1) / 3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *Df = reinterpret_cast<R *>(smem_raw);
    R *Db = Df + nrot;
    cx<R> *Pf = reinterpret_cast<cx<R> *>(Db + nrot);
    cx<R> *Pb = Pf + p2;
    cx<R> *Zb = Pb + p2;
    cx<R> *X = Zb + ncoax;         // [p2][ROTC_S]
    cx<R> *U = X + p2 * ROTC_S;    // [p2][ROTC_S]
    short2 *itab = reinterpret_cast<short2 *>(U + p2 * ROTC_S);
    const int nitem = p * (p + 1) / 2;
    for (int i = threadIdx.x; i < nitem; i += blockDim.x) {
        int n = 0;
        while ((n + 1) * (n + 2) / 2 <= i) ++n;
        itab[i] = make_short2((short)n, (short)(i - n * (n + 1) / 2));
    }
    const int64_t ck = chunk0 + blockIdx.x;
    const int beg = chunk_beg[ck], cnt = chunk_cnt[ck];
    const int o = chunk_off[ck];
    const R *D2 = RD + (int64_t)o * 2 * nrot;
    const cx<R> *P2 = RP + (int64_t)o * 2 * p2;
    const cx<R> *Z = RZ + (((int64_t)d * (lmax + 1) + l) * n_tlen + tidx[o]) * ncoax;
    for (int i = threadIdx.x; i < 2 * nrot; i += blockDim.x) Df[i] = D2[i];
    for (int i = threadIdx.x; i < 2 * p2; i += blockDim.x) Pf[i] = P2[i];
    for (int i = threadIdx.x; i < ncoax; i += blockDim.x) Zb[i] = Z[i];
    const int warp = threadIdx.x >> 5, c = threadIdx.x & 31;
    for (int b0 = 0; b0 < cnt; b0 += pc) {
        const int np = min(pc, cnt - b0);
        const int nct = np * ncol;
        __syncthreads();
        // load with the forward phase and fold (as in k_m2l_rot), one (item, column) per thread
        for (int i = threadIdx.x; i < nitem * ROTC_N; i += blockDim.x) {
            const int it = i / ROTC_N, j = i - it * ROTC_N;
            const short2 tn = itab[it];
            const int n = tn.x, mm = tn.y, c0 = n * n + n;
            cx<R> va = {0, 0}, vb = {0, 0};
            if (j < nct) {
                const int pr = j / ncol, cc = j - pr * ncol;
                const cx<R> *src = C + (((int64_t)d * nbox + ff_src[pair_e[beg + b0 + pr]]) * 3 * nr + col0 + cc) * p2;
                if (mm == 0) {
                    va = src[c0] * Pf[c0];
                } else {
                    const cx<R> xp = src[c0 + mm], xm = src[c0 - mm], e = Pf[c0 + mm];
                    const cx<R> sum = xp + xm, dif = xp - xm;
                    va = cx<R>{e.re * sum.re - e.im * dif.im, e.re * sum.im + e.im * dif.re};
                    vb = cx<R>{e.re * dif.re - e.im * sum.im, e.re * dif.im + e.im * sum.re};
                }
            }
            X[(n * n + mm) * ROTC_S + j] = va;
            if (mm > 0) X[(n * n + n + mm) * ROTC_S + j] = vb;
        }
        __syncthreads();
        // stage 1: folded polar rotation; slot k (by loop length) goes to warp k in snake order
        for (int k0 = 0; k0 < p2; k0 += ROTC_WARPS) {
            const int k = k0 + (((k0 / ROTC_WARPS) & 1) ? ROTC_WARPS - 1 - warp : warp);
            if (k >= p2) continue;
            const int r13 = slot_by_rowlen(p, k);
            int n1 = (int)sqrtf((float)r13);
            while (n1 * n1 > r13) --n1;
            while ((n1 + 1) * (n1 + 1) <= r13) ++n1;
            const int sl1 = r13 - n1 * n1;
            const bool plus1 = sl1 <= n1;
            const int am1 = plus1 ? sl1 : sl1 - n1;
            const R *a = Df + rot_off(n1) + (plus1 ? sl1 * (n1 + 1) : (n1 + 1) * (n1 + 1) + (am1 - 1) * n1);
            const int flen = plus1 ? n1 + 1 : n1, fin = plus1 ? n1 * n1 : n1 * n1 + n1 + 1;
            cx<R> acc = {0, 0};
            for (int jj = 0; jj < flen; ++jj) {
                const R t = a[jj];
                const cx<R> xv = X[(fin + jj) * ROTC_S + c];
                acc.re = fma(t, xv.re, acc.re);
                acc.im = fma(t, xv.im, acc.im);
            }
            U[r13 * ROTC_S + c] = acc;
        }
        __syncthreads();
        // stage 2: coaxial translation, slot k by coaxial row length
        for (int k0 = 0; k0 < p2; k0 += ROTC_WARPS) {
            const int k = k0 + (((k0 / ROTC_WARPS) & 1) ? ROTC_WARPS - 1 - warp : warp);
            if (k >= p2) continue;
            const int r2 = slot_by_order(p, k);
            int n2 = (int)sqrtf((float)r2);
            while (n2 * n2 > r2) --n2;
            while ((n2 + 1) * (n2 + 1) <= r2) ++n2;
            const bool plus2 = r2 - n2 * n2 <= n2;
            const int am2 = plus2 ? r2 - n2 * n2 : r2 - n2 * n2 - n2;
            int zbase = 0;
            for (int m = -(p - 1); m < am2; ++m) zbase += (p - abs(m)) * (p - abs(m));
            const int zw = p - am2;
            const cx<R> *z = Zb + zbase + (n2 - am2) * zw;
            cx<R> acc = {0, 0};
            for (int jj = 0; jj < zw; ++jj) {
                const int n = am2 + jj;
                cfma(acc, z[jj], U[(n * n + (plus2 ? am2 : n + am2)) * ROTC_S + c]);
            }
            X[r2 * ROTC_S + c] = acc;
        }
        __syncthreads();
        // stage 3: folded polar rotation back: P (a half) and Q (b half)
        for (int k0 = 0; k0 < p2; k0 += ROTC_WARPS) {
            const int k = k0 + (((k0 / ROTC_WARPS) & 1) ? ROTC_WARPS - 1 - warp : warp);
            if (k >= p2) continue;
            const int r13 = slot_by_rowlen(p, k);
            int n1 = (int)sqrtf((float)r13);
            while (n1 * n1 > r13) --n1;
            while ((n1 + 1) * (n1 + 1) <= r13) ++n1;
            const int sl1 = r13 - n1 * n1;
            const bool plus1 = sl1 <= n1;
            const int am1 = plus1 ? sl1 : sl1 - n1;
            const R *bb = Db + rot_off(n1) + (plus1 ? sl1 * (n1 + 1) : (n1 + 1) * (n1 + 1) + (am1 - 1) * n1);
            const int flen = plus1 ? n1 + 1 : n1, fin = plus1 ? n1 * n1 : n1 * n1 + n1 + 1;
            cx<R> acc = {0, 0};
            for (int jj = 0; jj < flen; ++jj) {
                const R t = bb[jj];
                const cx<R> xv = X[(fin + jj) * ROTC_S + c];
                acc.re = fma(t, xv.re, acc.re);
                acc.im = fma(t, xv.im, acc.im);
            }
            U[r13 * ROTC_S + c] = acc;
        }
        __syncthreads();
        // unfold, back phase, store: one (column, coefficient) per thread, coefficients fastest
        // so that the stores of a warp are contiguous
        for (int i = threadIdx.x; i < p2 * nct; i += blockDim.x) {
            const int j = i / p2, r = i - j * p2;
            int rn = (int)sqrtf((float)r);
            while (rn * rn > r) --rn;
            while ((rn + 1) * (rn + 1) <= r) ++rn;
            const int m = r - rn * rn - rn, mm = abs(m);
            cx<R> v = U[(rn * rn + mm) * ROTC_S + j];
            if (mm > 0) {
                const cx<R> q = U[(rn * rn + rn + mm) * ROTC_S + j];
                v = m > 0 ? v + q : v - q;
            }
            const int pr = j / ncol, cc = j - pr * ncol;
            const int64_t e = pair_e[beg + b0 + pr];
            Y[((e - e_first) * ncol + cc) * p2 + r] = v * Pb[r];
        }
    }
}

// D(l,q) = R|R D(parent) + sum of the target's M2L pair results (Eq. 2.21), columns col0..col0+ncol.
// Threads: rows_pad x ct column groups; a thread owns columns cid * L2L_CPT .. + L2L_CPT - 1.
constexpr int L2L_CPT = 3;
template <typename R>
__global__ void k_l2l_reduce(int64_t off, int l, int lmax, int d0, int64_t nr, int p2, int64_t nbox, int col0, int ncol,
                             int ct, const int32_t *parent, const uint64_t *key, const int32_t *ff_start,
                             const cx<R> *Tll, const cx<R> *Y, int64_t e_first, cx<R> *D, const cx<R> *Yll,
                             const int32_t *ll_entry, int64_t ll_first, int64_t y_dstride, int64_t yll_dstride) {
    const int d = d0 + (int)blockIdx.y;  // domain: one grid row per domain, each with its own Y blocks
    Y += (int64_t)blockIdx.y * y_dstride;
    if (Yll) Yll += (int64_t)blockIdx.y * yll_dstride;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<R> *X = reinterpret_cast<cx<R> *>(smem_raw);
    const int64_t g = off + blockIdx.x;
    const int rows_pad = blockDim.x / ct;
    const int r = threadIdx.x % rows_pad, cid = threadIdx.x / rows_pad;
    const cx<R> *T = nullptr;
    if (l >= 3 && Yll == nullptr) {
        const int64_t P = parent[g];
        for (int e = threadIdx.x; e < ncol * p2; e += blockDim.x)
            X[e] = D[(((int64_t)d * nbox + P) * 3 * nr + col0 + e / p2) * p2 + e % p2];
        T = Tll + oct_matrix(d, l, (int)(key[g] & 7), lmax) * p2 * p2;
        __syncthreads();
    }
    if (r >= p2) return;
    const int e0 = ff_start[g], e1 = ff_start[g + 1];
    // this thread's columns c0 .. c0 + L2L_CPT - 1: one read of T per row k feeds all of them
    const int c0 = cid * L2L_CPT;
    cx<R> lp[L2L_CPT];
#pragma unroll
    for (int j = 0; j < L2L_CPT; ++j) lp[j] = {0, 0};
    if (T)
        for (int k = 0; k < p2; ++k) {
            const cx<R> t = T[(int64_t)k * p2 + r];
#pragma unroll
            for (int j = 0; j < L2L_CPT; ++j)
                if (c0 + j < ncol) cfma(lp[j], t, X[(c0 + j) * p2 + k]);
        }
    if (l >= 3 && Yll != nullptr) {  // R|R already applied in rotation form, per child entry
        const cx<R> *yl = Yll + ((int64_t)(ll_entry[g] - ll_first) * ncol) * p2 + r;
#pragma unroll
        for (int j = 0; j < L2L_CPT; ++j)
            if (c0 + j < ncol) lp[j] = yl[(c0 + j) * p2];
    }
#pragma unroll
    for (int j = 0; j < L2L_CPT; ++j) {
        const int c = c0 + j;
        if (c >= ncol) break;
        cx<R> a0 = lp[j], a1 = {0, 0}, a2 = {0, 0}, a3 = {0, 0};
        const cx<R> *y = Y + ((e0 - e_first) * ncol + c) * p2 + r;
        const int64_t st = (int64_t)ncol * p2;
        int e = e0;
        for (; e + 4 <= e1; e += 4, y += 4 * st) {
            a0 += y[0];
            a1 += y[st];
            a2 += y[2 * st];
            a3 += y[3 * st];
        }
        for (; e < e1; ++e, y += st) a0 += y[0];
        D[(((int64_t)d * nbox + g) * 3 * nr + col0 + c) * p2 + r] = (a0 + a1) + (a2 + a3);
    }
}

// Rotation-form M2M: the parent's multipole is the sum of its children's translated expansions,
// C(g) = sum_{children ch} Y[entry(ch)], columns col0 .. col0 + ncol - 1 (Eq. 2.20).
template <typename R>
__global__ void k_mm_reduce(int64_t par_off, int d0, int64_t nr, int p2, int64_t nbox, int col0, int ncol,
                            const int32_t *cbeg, const int32_t *cend, const int32_t *entry, int64_t e_first,
                            const cx<R> *Y, cx<R> *C, int64_t y_dstride) {
    const int d = d0 + (int)blockIdx.y;  // domain: one grid row per domain, each with its own Y block
    Y += (int64_t)blockIdx.y * y_dstride;
    const int64_t g = par_off + blockIdx.x;
    if (cbeg[g] == cend[g]) return;  // a leaf of an adaptive tree: its multipole expansion is P2M's
    const int64_t nel = (int64_t)ncol * p2;
    for (int64_t e = threadIdx.x; e < nel; e += blockDim.x) {
        cx<R> a = {0, 0};
        for (int ch = cbeg[g]; ch < cend[g]; ++ch) a += Y[(int64_t)(entry[ch] - e_first) * nel + e];
        const int c = (int)(e / p2), q = (int)(e - (int64_t)c * p2);
        C[(((int64_t)d * nbox + g) * 3 * nr + col0 + c) * p2 + q] = a;
    }
}

// M2L + L2L for many columns (Eq. 2.21) as a register-tiled complex GEMM per target box:
// D[t][:, tile] = T_ll(oct) D[parent][:, tile] + sum_FF T_o C[src][:, tile], tile = 64 columns.
// For every translation the CTA stages T (input-major, p2 x p2) and the input columns transposed
// to [k][col]; thread (rg, cgp) accumulates rows 4rg..4rg+3 x columns 4cgp..4cgp+3.
constexpr int MT_COLS = 64;
template <typename R>
__device__ __forceinline__ void mt_stage(const cx<R> *__restrict__ T, const cx<R> *__restrict__ Xg, int p2, int ncol_here,
                                         cx<R> *Ts, cx<R> *Cs) {
    for (int i = threadIdx.x; i < p2 * p2; i += blockDim.x) Ts[i] = T[i];
    // Xg points at column 0 of the tile: element (c, k) at Xg[c * p2 + k]
    for (int i = threadIdx.x; i < p2 * MT_COLS; i += blockDim.x) {
        int c = i / p2, k = i - c * p2;
        Cs[k * MT_COLS + c] = c < ncol_here ? Xg[(int64_t)c * p2 + k] : cx<R>{0, 0};
    }
}
template <typename R>
__device__ __forceinline__ void mt_accumulate(const cx<R> *Ts, const cx<R> *Cs, int p2, int rg, int cgp, cx<R> acc[4][4]) {
    const int r0 = 4 * rg, c0 = 4 * cgp;
#pragma unroll 4
    for (int k = 0; k < p2; ++k) {
        cx<R> t[4], c[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) t[i] = (r0 + i < p2) ? Ts[k * p2 + r0 + i] : cx<R>{0, 0};
#pragma unroll
        for (int j = 0; j < 4; ++j) c[j] = Cs[k * MT_COLS + c0 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) cfma(acc[i][j], t[i], c[j]);
    }
}
template <typename R>
__global__ void k_m2l_multi(int64_t off, int l, int lmax, int64_t nr, int p2, int64_t nbox, const int32_t *parent,
                            const uint64_t *key, const int32_t *ff_start, const int32_t *ff_src, const int16_t *ff_off,
                            const cx<R> *Tm2l, const cx<R> *Tll, const cx<R> *C, cx<R> *D) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<R> *Ts = reinterpret_cast<cx<R> *>(smem_raw);
    cx<R> *Cs = Ts + p2 * p2;
    const int64_t g = off + blockIdx.x;
    const int d = blockIdx.y;
    const int ncols = (int)(3 * nr);
    const int col0 = blockIdx.z * MT_COLS;
    const int nh = min(MT_COLS, ncols - col0);
    const int rg = threadIdx.x % ((p2 + 3) / 4), cgp = threadIdx.x / ((p2 + 3) / 4);
    cx<R> acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = {0, 0};
    if (l >= 3) {
        const int64_t P = parent[g];
        mt_stage<R>(Tll + oct_matrix(d, l, (int)(key[g] & 7), lmax) * p2 * p2,
                    D + (((int64_t)d * nbox + P) * ncols + col0) * p2, p2, nh, Ts, Cs);
        __syncthreads();
        mt_accumulate<R>(Ts, Cs, p2, rg, cgp, acc);
    }
    for (int e = ff_start[g]; e < ff_start[g + 1]; ++e) {
        __syncthreads();
        mt_stage<R>(Tm2l + m2l_matrix(d, l, ff_off[e], lmax) * p2 * p2,
                    C + (((int64_t)d * nbox + ff_src[e]) * ncols + col0) * p2, p2, nh, Ts, Cs);
        __syncthreads();
        mt_accumulate<R>(Ts, Cs, p2, rg, cgp, acc);
    }
    const int r0 = 4 * rg, c0 = 4 * cgp;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (c0 + j < nh)
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (r0 + i < p2) D[(((int64_t)d * nbox + g) * ncols + col0 + c0 + j) * p2 + r0 + i] = acc[i][j];
}

// ---------------------------------------------------------------- near field + L2P + self (Step 4)
template <typename R>
struct __align__(4 * sizeof(R)) V4 {
    R x, y, z, w;
};
template <typename R>
struct __align__(2 * sizeof(R)) V2 {
    R x, y;
};
// one tile of 128 sources, packed so that a pair reads its source with a few vector loads
template <typename R>
struct SrcTile {
    V4<R> pa[128];      // position (high part) and scatterer id
    V4<R> pb[128];      // position low part (double-float only) and n_x
    V2<R> pn[128];      // n_y, n_z
    V4<R> dv[2][3][128];  // densities (v0, v1), (v2, q0), (q1, q2) of the current RHS, both sides
    V2<R> sn[128];        // s = n.(v_side1 - v_side0): the scatterer's dipole density is v_0 + s n
};
template <typename R>
union NearSmem {
    SrcTile<R> tile;
    cx<R> red[6][128];             // partial sums of the source slices
};

// fast single-precision transcendentals, precise double-precision ones.  In single precision the
// PTX approximations of the special-function unit with subnormals flushed (the arguments of the
// near field are distances, R k and -Im k R: never subnormal where the result matters):
// rsqrt.approx (relative error about 2^-23), ex2.approx of x log2(e), sin/cos.approx (absolute
// error about 2^-21 for |x| <= pi; near-field pairs have |k| R well inside that range)
__device__ __forceinline__ float rsqrt_(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
__device__ __forceinline__ float exp_(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x * 1.44269504088896340736f));
    return y;
}
__device__ __forceinline__ double exp_(double x) { return exp(x); }
__device__ __forceinline__ void sincos_(float x, float *s, float *c) {
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(*s) : "f"(x));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(*c) : "f"(x));
}
__device__ __forceinline__ void sincos_(double x, double *s, double *c) { sincos(x, s, c); }

// One (source, target) pair of one domain: acc_i += -(K v)_i + g q_i (Eq. 2.12 for beta != alpha),
// r = s_beta - s_alpha, inv = 1/|r| (0 for the node itself, which then contributes nothing).  With
// grad'g = c r, the bracket applied to v is -c [n (r.v) - (n.r) v - r (n.v)], which by
// a x (b x c) = b (a.c) - c (a.b) equals c [(n x r) x v + (n.r) v]; w = n x r is formed once per
// pair, so each right-hand side costs one real-vector cross product and two complex FMAs per row.
template <typename R>
__device__ __forceinline__ void cross_apply(const R *w, R nr, cx<R> g, cx<R> c, const cx<R> *v, const cx<R> *q,
                                            cx<R> *acc) {
    const cx<R> u[3] = {w[1] * v[2] - w[2] * v[1] + nr * v[0], w[2] * v[0] - w[0] * v[2] + nr * v[1],
                        w[0] * v[1] - w[1] * v[0] + nr * v[2]};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        cfma(acc[i], c, u[i]);
        cfma(acc[i], g, q[i]);
    }
}
template <typename R>
__device__ __forceinline__ void pair_kernel(R rx, R ry, R rz, R inv, R Rr, cx<R> k, R nx, R ny, R nz, const cx<R> *v,
                                            const cx<R> *q, cx<R> *acc) {
    // g = e^{ikR}/(4 pi R), grad'g = c r with c = g (ik - 1/R)/R
    R e = k.im != (R)0 ? exp_(-k.im * Rr) : (R)1;  // warp-uniform: k is per domain
    R sn, cs;
    sincos_(k.re * Rr, &sn, &cs);
    R f = e * inv * (R)(0.25 / FMBEM_PI);
    cx<R> g = {f * cs, f * sn};
    // (i k - 1/R)/R with i k = -Im k + i Re k
    cx<R> c = g * cx<R>{(-k.im - inv) * inv, k.re * inv};
    const R w[3] = {ny * rz - nz * ry, nz * rx - nx * rz, nx * ry - ny * rx};
    const R nr = nx * rx + ny * ry + nz * rz;
    cross_apply<R>(w, nr, g, c, v, q, acc);
}

// Epilogue of one result row of one target node a (row = 3 * side + component): the sum of the
// source slices' partial results red[sl * nt + ti] in slice order, plus the far field (L2P,
// Eq. 2.23 first term) of that side's domain from the leaf's local expansion, plus the row of the
// analytic self block applied to x in double precision; stored in user order.
template <typename R>
__device__ __forceinline__ void near_epilogue(const cx<R> *red, int ti, int nt, int nsl, int a, int row, int64_t r,
                                              int64_t g, int64_t N, int64_t nr, int p2, int64_t nbox,
                                              const int32_t *dom, const int32_t *perm, const cx<R> *Bl2p,
                                              const cx<R> *D, const c64 *Mself, const c64 *x, c64 *y) {
    const int sd = row / 3, c = row % 3;
    cx<R> v = red[ti];
    for (int sl = 1; sl < nsl; ++sl) v += red[sl * nt + ti];
    const int d = sd == 0 ? 0 : dom[a];
    const cx<R> *Dl = D + (((int64_t)d * nbox + g) * 3 * nr + 3 * r + c) * p2;
    const cx<R> *B = Bl2p + ((int64_t)sd * N + a) * p2;
    for (int q = 0; q < p2; ++q) cfma(v, Dl[q], B[q]);
    const int64_t u = perm[a];
    const c64 *M = Mself + 36 * u + 6 * row;
    const c64 *xa = x + (r * N + u) * 6;
    c64 sacc = {(double)v.re, (double)v.im};
    for (int cc = 0; cc < 6; ++cc) cfma(sacc, M[cc], xa[cc]);
    y[(r * N + u) * 6 + row] = sacc;
}

// index of the neighbour range holding source e: the last q with cum[q] <= e (binary search)
__device__ __forceinline__ int source_range(const int *cum, int nnb, int e) {
    int lo = 0, hi = nnb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cum[mid] <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Step 4 for one leaf: near field over the leaf and its Neighbor leaves (both domains), far field
// from the leaf's local expansions (L2P), the analytic self block in double precision, and the
// store of the 6 result rows in user order.  Up to 128 targets per pass; the 128 threads split as
// (target, source slice) with 128 / n_targets slices, reduced in a fixed order.
template <typename R, bool DOUBLE_FLOAT>
__device__ __forceinline__ void near_body(int64_t g, int64_t N, int64_t nr, int p2, int64_t nbox,
                                          const int32_t *nbeg, const int32_t *nend, const int32_t *nbr_start,
                                          const int32_t *nbr_idx, const R *pos_hi, const R *pos_lo, const R *nrm,
                                          const int32_t *dom, const int32_t *perm, const cx<R> *dens,
                                          const DomainConsts *dc, const cx<R> *Bl2p, const cx<R> *D, const c64 *Mself,
                                          const c64 *x, c64 *y, const int64_t *cache_base, const V4<R> *cache,
                                          bool side1, int64_t bx) {
    __shared__ NearSmem<R> S;
    __shared__ int rng_beg[32], rng_cum[33];
    SrcTile<R> &T = S.tile;
    const int nb0 = nbr_start[bx], nnb = nbr_start[bx + 1] - nb0;
    if (threadIdx.x == 0) {
        int cum = 0;
        for (int q = 0; q < nnb; ++q) {
            int b = nbr_idx[nb0 + q];
            rng_beg[q] = nbeg[b];
            rng_cum[q] = cum;
            cum += nend[b] - nbeg[b];
        }
        rng_cum[nnb] = cum;
    }
    __syncthreads();
    const int nsrc = rng_cum[nnb];
    const int t0 = nbeg[g], t1 = nend[g];
    for (int64_t r = 0; r < nr; ++r) {
        for (int tb = t0; tb < t1; tb += 128) {
            const int nt = min(128, t1 - tb);
            const int nsl = 128 / nt;
            const int tg = threadIdx.x % nt, slice = threadIdx.x / nt;
            const bool active = slice < nsl;
            const int a = tb + tg;
            R ax = pos_hi[3 * a], ay = pos_hi[3 * a + 1], az = pos_hi[3 * a + 2], alx = 0, aly = 0, alz = 0;
            if (DOUBLE_FLOAT) { alx = pos_lo[3 * a]; aly = pos_lo[3 * a + 1]; alz = pos_lo[3 * a + 2]; }
            const int adom = dom[a];
            const cx<R> kb = to<R>(dc[0].k), kj = to<R>(dc[adom].k);
            cx<R> acc0[3] = {{0, 0}, {0, 0}, {0, 0}}, acc1[3] = {{0, 0}, {0, 0}, {0, 0}};
            for (int s0 = 0; s0 < nsrc; s0 += 128) {
                __syncthreads();
                {  // stage a tile of sources
                    int e = s0 + threadIdx.x;
                    if (e < nsrc) {
                        const int q = source_range(rng_cum, nnb, e);
                        int i = rng_beg[q] + (e - rng_cum[q]);
                        const int t = threadIdx.x;
                        T.pa[t] = V4<R>{pos_hi[3 * i], pos_hi[3 * i + 1], pos_hi[3 * i + 2], (R)dom[i]};
                        R lo[3] = {0, 0, 0};
                        if (DOUBLE_FLOAT) { lo[0] = pos_lo[3 * i]; lo[1] = pos_lo[3 * i + 1]; lo[2] = pos_lo[3 * i + 2]; }
                        T.pb[t] = V4<R>{lo[0], lo[1], lo[2], nrm[3 * i]};
                        T.pn[t] = V2<R>{nrm[3 * i + 1], nrm[3 * i + 2]};
                        for (int sd = 0; sd < 2; ++sd) {
                            const cx<R> *dn = dens + ((sd * nr + r) * N + i) * 6;
                            for (int c = 0; c < 3; ++c)
                                T.dv[sd][c][t] = V4<R>{dn[2 * c].re, dn[2 * c].im, dn[2 * c + 1].re, dn[2 * c + 1].im};
                        }
                        if (cache) {  // the scatterer side's v differs from the background's along n only
                            const cx<R> *d0 = dens + (r * N + i) * 6, *d1 = dens + ((nr + r) * N + i) * 6;
                            const R nv[3] = {nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2]};
                            cx<R> sv = {0, 0};
                            for (int c = 0; c < 3; ++c) sv += nv[c] * (d1[c] - d0[c]);
                            T.sn[t] = V2<R>{sv.re, sv.im};
                        }
                    }
                }
                __syncthreads();
                const int ns = min(128, nsrc - s0);
                const R adom_r = side1 ? (R)adom : (R)-1;  // -1: no scatterer-side pairs (impedance boundary)
                // cached pair scalars of this target: [side][source][target] within the leaf's block
                const int NT = t1 - t0;
                const V4<R> *cs0 = cache ? cache + 2 * cache_base[bx] + (tb - t0 + tg) : nullptr;
                if (active)
                    for (int u = slice; u < ns; u += nsl) {
                        const V4<R> pa = T.pa[u], pb = T.pb[u];
                        const V2<R> pn = T.pn[u];
                        R rx = pa.x - ax, ry = pa.y - ay, rz = pa.z - az;
                        if (DOUBLE_FLOAT) { rx += pb.x - alx; ry += pb.y - aly; rz += pb.z - alz; }
                        cx<R> v[3], q[3];
                        {
                            const V4<R> a0 = T.dv[0][0][u], a1 = T.dv[0][1][u], a2 = T.dv[0][2][u];
                            v[0] = {a0.x, a0.y}; v[1] = {a0.z, a0.w}; v[2] = {a1.x, a1.y};
                            q[0] = {a1.z, a1.w}; q[1] = {a2.x, a2.y}; q[2] = {a2.z, a2.w};
                        }
                        if (cs0) {
                            // g and c from the cache; only the normal-dependent part here.  With
                            // w = n x r, U = w x v_0 + (n.r) v_0 is the background's bracket up to sign
                            // (its normal is -n), and since (n x r) x n + (n.r) n = r for a unit n,
                            // the scatterer side's bracket for v_0 + s n is U + s r
                            const int64_t e = s0 + u;
                            const R w1[3] = {pn.x * rz - pn.y * ry, pn.y * rx - pb.w * rz, pb.w * ry - pn.x * rx};
                            const R nr1 = pb.w * rx + pn.x * ry + pn.y * rz;
                            const cx<R> U[3] = {w1[1] * v[2] - w1[2] * v[1] + nr1 * v[0],
                                                w1[2] * v[0] - w1[0] * v[2] + nr1 * v[1],
                                                w1[0] * v[1] - w1[1] * v[0] + nr1 * v[2]};
                            const V4<R> s0v = cs0[e * NT];
                            const cx<R> mc0 = {-s0v.z, -s0v.w}, g0 = {s0v.x, s0v.y};
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                cfma(acc0[c], mc0, U[c]);
                                cfma(acc0[c], g0, q[c]);
                            }
                            if (pa.w == adom_r) {
                                const V4<R> a1 = T.dv[1][1][u], a2 = T.dv[1][2][u];
                                const cx<R> q1[3] = {{a1.z, a1.w}, {a2.x, a2.y}, {a2.z, a2.w}};
                                const V2<R> sv = T.sn[u];
                                const cx<R> sc = {sv.x, sv.y};
                                const R rr[3] = {rx, ry, rz};
                                const V4<R> s1v = cs0[((int64_t)nsrc + e) * NT];
                                const cx<R> c1 = {s1v.z, s1v.w}, g1 = {s1v.x, s1v.y};
#pragma unroll
                                for (int c = 0; c < 3; ++c) {
                                    cfma(acc1[c], c1, U[c] + rr[c] * sc);
                                    cfma(acc1[c], g1, q1[c]);
                                }
                            }
                            continue;
                        }
                        R R2 = rx * rx + ry * ry + rz * rz;
                        R inv = R2 > (R)0 ? rsqrt_(R2) : (R)0;  // the node itself drops out
                        R Rr = R2 * inv;
                        pair_kernel<R>(rx, ry, rz, inv, Rr, kb, -pb.w, -pn.x, -pn.y, v, q, acc0);
                        if (pa.w == adom_r) {
                            const V4<R> a0 = T.dv[1][0][u], a1 = T.dv[1][1][u], a2 = T.dv[1][2][u];
                            v[0] = {a0.x, a0.y}; v[1] = {a0.z, a0.w}; v[2] = {a1.x, a1.y};
                            q[0] = {a1.z, a1.w}; q[1] = {a2.x, a2.y}; q[2] = {a2.z, a2.w};
                            pair_kernel<R>(rx, ry, rz, inv, Rr, kj, pb.w, pn.x, pn.y, v, q, acc1);
                        }
                    }
            }
            // reduce the source slices in a fixed order, then far field (L2P), self block and store,
            // one (target, result row) item per thread so that all warps share the epilogue
            __syncthreads();
            for (int c = 0; c < 3; ++c) { S.red[c][threadIdx.x] = acc0[c]; S.red[3 + c][threadIdx.x] = acc1[c]; }
            __syncthreads();
            for (int it = threadIdx.x; it < nt * 6; it += blockDim.x) {
                const int ti = it % nt, row = it / nt;
                near_epilogue<R>(S.red[row], ti, nt, nsl, tb + ti, row, r, g, N, nr, p2, nbox, dom, perm, Bl2p, D,
                                 Mself, x, y);
            }
        }
    }
}
template <typename R, bool DOUBLE_FLOAT>
__global__ void __launch_bounds__(128) k_near(const int32_t *leaf_box, int64_t N, int64_t nr, int p2, int64_t nbox,
                                              const int32_t *nbeg, const int32_t *nend, const int32_t *nbr_start,
                                              const int32_t *nbr_idx, const R *pos_hi, const R *pos_lo, const R *nrm,
                                              const int32_t *dom, const int32_t *perm, const cx<R> *dens,
                                              const DomainConsts *dc, const cx<R> *Bl2p, const cx<R> *D, const c64 *Mself,
                                              const c64 *x, c64 *y, const int64_t *cache_base,
                                              const V4<R> *cache, bool side1) {
    near_body<R, DOUBLE_FLOAT>(leaf_box[blockIdx.x], N, nr, p2, nbox, nbeg, nend, nbr_start, nbr_idx, pos_hi, pos_lo, nrm, dom,
                               perm, dens, dc, Bl2p, D, Mself, x, y, cache_base, cache, side1, blockIdx.x);
}

// ---------------------------------------------------------------- near field for blocks of RHS
// The kernel scalars of a pair and domain (g and c of grad'g = c r) do not depend on the right-
// hand side, so for many right-hand sides they are computed once and applied to RB of them.
template <typename R>
__device__ __forceinline__ void pair_scalars(R inv, R Rr, cx<R> k, cx<R> &g, cx<R> &c) {
    R e = k.im != (R)0 ? exp_(-k.im * Rr) : (R)1;
    R sn, cs;
    sincos_(k.re * Rr, &sn, &cs);
    R f = e * inv * (R)(0.25 / FMBEM_PI);
    g = {f * cs, f * sn};
    c = g * cx<R>{(-k.im - inv) * inv, k.re * inv};
}
// Near-field pair scalars of one leaf for the cache: for side 0 (domain 0) and side 1 (the
// target's scatterer, zero where the source lies in another scatterer), every source e of the
// leaf's Neighbor list (in k_near's order) and every target t of the leaf, g and c of
// grad'g = c r (Eq. 2.12) at entry (side, e, t) of the leaf's block, in double precision.
template <typename R>
__global__ void k_near_cache(const int32_t *leaf_box, const int32_t *nbeg, const int32_t *nend, const int32_t *nbr_start,
                             const int32_t *nbr_idx, const double *pos, const int32_t *dom, const DomainConsts *dc,
                             const int64_t *base, V4<R> *cache) {
    __shared__ int rng_beg[32], rng_cum[33];
    const int64_t g = leaf_box[blockIdx.x];
    const int nb0 = nbr_start[blockIdx.x], nnb = nbr_start[blockIdx.x + 1] - nb0;
    if (threadIdx.x == 0) {
        int cum = 0;
        for (int q = 0; q < nnb; ++q) {
            const int b = nbr_idx[nb0 + q];
            rng_beg[q] = nbeg[b];
            rng_cum[q] = cum;
            cum += nend[b] - nbeg[b];
        }
        rng_cum[nnb] = cum;
    }
    __syncthreads();
    const int nsrc = rng_cum[nnb], t0 = nbeg[g], nt = nend[g] - t0;
    V4<R> *out = cache + 2 * base[blockIdx.x];
    const int64_t total = 2 * (int64_t)nsrc * nt;
    for (int64_t it = threadIdx.x; it < total; it += blockDim.x) {
        const int side = (int)(it / ((int64_t)nsrc * nt));
        const int rem = (int)(it - (int64_t)side * nsrc * nt), e = rem / nt, t = rem - e * nt;
        const int q = source_range(rng_cum, nnb, e);
        const int i = rng_beg[q] + (e - rng_cum[q]), a = t0 + t;
        const double rx = pos[3 * i] - pos[3 * a], ry = pos[3 * i + 1] - pos[3 * a + 1], rz = pos[3 * i + 2] - pos[3 * a + 2];
        const double R2 = rx * rx + ry * ry + rz * rz;
        const double inv = R2 > 0.0 ? rsqrt_(R2) : 0.0;
        const double Rr = R2 * inv;
        c64 gs = {0, 0}, cs = {0, 0};
        if (side == 0 || dom[i] == dom[a]) pair_scalars<double>(inv, Rr, dc[side == 0 ? 0 : dom[a]].k, gs, cs);
        out[it] = V4<R>{(R)gs.re, (R)gs.im, (R)cs.re, (R)cs.im};
    }
}

constexpr int NB_TILE = 64;  // sources per shared-memory tile in the blocked kernel
template <typename R, int RB>
struct SrcTileRB {
    V4<R> pa[NB_TILE];
    V4<R> pb[NB_TILE];
    V2<R> pn[NB_TILE];
    V4<R> dv[2][RB][3][NB_TILE];  // per side and RHS of the block: (v0, v1), (v2, q0), (q1, q2)
};
template <typename R, int RB>
union NearSmemRB {
    SrcTileRB<R, RB> tile;
    cx<R> red[6][RB][128];
};

template <typename R, bool DOUBLE_FLOAT, int RB>
__global__ void __launch_bounds__(128) k_near_rb(const int32_t *leaf_box, int64_t N, int64_t nr, int p2, int64_t nbox,
                                                 const int32_t *nbeg, const int32_t *nend, const int32_t *nbr_start,
                                                 const int32_t *nbr_idx, const R *pos_hi, const R *pos_lo,
                                                 const R *nrm, const int32_t *dom, const int32_t *perm,
                                                 const cx<R> *dens, const DomainConsts *dc, const cx<R> *Bl2p,
                                                 const cx<R> *D, const c64 *Mself, const c64 *x, c64 *y,
                                                 bool side1) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    NearSmemRB<R, RB> &S = *reinterpret_cast<NearSmemRB<R, RB> *>(smem_raw);
    SrcTileRB<R, RB> &T = S.tile;
    __shared__ int rng_beg[32], rng_cum[33];
    const int64_t g = leaf_box[blockIdx.x];
    const int nb0 = nbr_start[blockIdx.x], nnb = nbr_start[blockIdx.x + 1] - nb0;
    if (threadIdx.x == 0) {
        int cum = 0;
        for (int q = 0; q < nnb; ++q) {
            int b = nbr_idx[nb0 + q];
            rng_beg[q] = nbeg[b];
            rng_cum[q] = cum;
            cum += nend[b] - nbeg[b];
        }
        rng_cum[nnb] = cum;
    }
    __syncthreads();
    const int nsrc = rng_cum[nnb];
    const int t0 = nbeg[g], t1 = nend[g];
    {
        const int64_t rb0 = (int64_t)blockIdx.y * RB;  // this block's right-hand sides
        const int nrb = (int)min((int64_t)RB, nr - rb0);
        for (int tb = t0; tb < t1; tb += 128) {
            const int nt = min(128, t1 - tb);
            const int nsl = 128 / nt;
            const int tg = threadIdx.x % nt, slice = threadIdx.x / nt;
            const bool active = slice < nsl;
            const int a = tb + tg;
            R ax = pos_hi[3 * a], ay = pos_hi[3 * a + 1], az = pos_hi[3 * a + 2], alx = 0, aly = 0, alz = 0;
            if (DOUBLE_FLOAT) { alx = pos_lo[3 * a]; aly = pos_lo[3 * a + 1]; alz = pos_lo[3 * a + 2]; }
            const int adom = dom[a];
            const R adom_r = side1 ? (R)adom : (R)-1;
            const cx<R> kb = to<R>(dc[0].k), kj = to<R>(dc[adom].k);
            cx<R> acc0[RB][3], acc1[RB][3];
#pragma unroll
            for (int rr = 0; rr < RB; ++rr)
#pragma unroll
                for (int c = 0; c < 3; ++c) { acc0[rr][c] = {0, 0}; acc1[rr][c] = {0, 0}; }
            for (int s0 = 0; s0 < nsrc; s0 += NB_TILE) {
                __syncthreads();
                for (int e2 = threadIdx.x; e2 < NB_TILE * (1 + 2 * RB); e2 += blockDim.x) {
                    const int t = e2 % NB_TILE, part = e2 / NB_TILE;  // part 0: geometry, 1..: (side, rhs)
                    const int e = s0 + t;
                    if (e >= nsrc) continue;
                    const int q = source_range(rng_cum, nnb, e);
                    const int i = rng_beg[q] + (e - rng_cum[q]);
                    if (part == 0) {
                        T.pa[t] = V4<R>{pos_hi[3 * i], pos_hi[3 * i + 1], pos_hi[3 * i + 2], (R)dom[i]};
                        R lo[3] = {0, 0, 0};
                        if (DOUBLE_FLOAT) { lo[0] = pos_lo[3 * i]; lo[1] = pos_lo[3 * i + 1]; lo[2] = pos_lo[3 * i + 2]; }
                        T.pb[t] = V4<R>{lo[0], lo[1], lo[2], nrm[3 * i]};
                        T.pn[t] = V2<R>{nrm[3 * i + 1], nrm[3 * i + 2]};
                    } else {
                        const int sd = (part - 1) / RB, rr = (part - 1) % RB;
                        if (rr < nrb) {
                            const cx<R> *dn = dens + ((sd * nr + rb0 + rr) * N + i) * 6;
                            for (int c = 0; c < 3; ++c)
                                T.dv[sd][rr][c][t] = V4<R>{dn[2 * c].re, dn[2 * c].im, dn[2 * c + 1].re, dn[2 * c + 1].im};
                        } else {
                            for (int c = 0; c < 3; ++c) T.dv[sd][rr][c][t] = V4<R>{0, 0, 0, 0};
                        }
                    }
                }
                __syncthreads();
                const int ns = min(NB_TILE, nsrc - s0);
                if (active)
                    for (int u = slice; u < ns; u += nsl) {
                        const V4<R> pa = T.pa[u], pb = T.pb[u];
                        const V2<R> pn = T.pn[u];
                        R rv3[3] = {pa.x - ax, pa.y - ay, pa.z - az};
                        if (DOUBLE_FLOAT) { rv3[0] += pb.x - alx; rv3[1] += pb.y - aly; rv3[2] += pb.z - alz; }
                        R R2 = rv3[0] * rv3[0] + rv3[1] * rv3[1] + rv3[2] * rv3[2];
                        R inv = R2 > (R)0 ? rsqrt_(R2) : (R)0;  // the node itself drops out
                        R Rr = R2 * inv;
                        const R n1[3] = {pb.w, pn.x, pn.y};
                        const R nr1 = n1[0] * rv3[0] + n1[1] * rv3[1] + n1[2] * rv3[2];
                        // w = n x r for the scatterer normal; domain 0 (normal reversed) uses -w, -n.r
                        const R w1[3] = {n1[1] * rv3[2] - n1[2] * rv3[1], n1[2] * rv3[0] - n1[0] * rv3[2],
                                         n1[0] * rv3[1] - n1[1] * rv3[0]};
                        const R w0[3] = {-w1[0], -w1[1], -w1[2]};
                        cx<R> gs, cs;
                        pair_scalars<R>(inv, Rr, kb, gs, cs);
#pragma unroll
                        for (int rr = 0; rr < RB; ++rr) {
                            const V4<R> a0 = T.dv[0][rr][0][u], a1 = T.dv[0][rr][1][u], a2 = T.dv[0][rr][2][u];
                            cx<R> v[3] = {{a0.x, a0.y}, {a0.z, a0.w}, {a1.x, a1.y}};
                            cx<R> qv[3] = {{a1.z, a1.w}, {a2.x, a2.y}, {a2.z, a2.w}};
                            cross_apply<R>(w0, -nr1, gs, cs, v, qv, acc0[rr]);
                        }
                        if (pa.w == adom_r) {
                            pair_scalars<R>(inv, Rr, kj, gs, cs);
#pragma unroll
                            for (int rr = 0; rr < RB; ++rr) {
                                const V4<R> a0 = T.dv[1][rr][0][u], a1 = T.dv[1][rr][1][u], a2 = T.dv[1][rr][2][u];
                                cx<R> v[3] = {{a0.x, a0.y}, {a0.z, a0.w}, {a1.x, a1.y}};
                                cx<R> qv[3] = {{a1.z, a1.w}, {a2.x, a2.y}, {a2.z, a2.w}};
                                cross_apply<R>(w1, nr1, gs, cs, v, qv, acc1[rr]);
                            }
                        }
                    }
            }
            // reduce the source slices in a fixed order
            __syncthreads();
#pragma unroll
            for (int rr = 0; rr < RB; ++rr)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    S.red[c][rr][threadIdx.x] = acc0[rr][c];
                    S.red[3 + c][rr][threadIdx.x] = acc1[rr][c];
                }
            __syncthreads();
            for (int it = threadIdx.x; it < nt * 6 * nrb; it += blockDim.x) {
                const int ti = it % nt, rest = it / nt, row = rest % 6, rr = rest / 6;
                near_epilogue<R>(S.red[row][rr], ti, nt, nsl, tb + ti, row, rb0 + rr, g, N, nr, p2, nbox, dom, perm,
                                 Bl2p, D, Mself, x, y);
            }
        }
    }
}

// ---------------------------------------------------------------- warp-independent near field
// Steps 4-5 for many right-hand sides in single precision.  One warp owns one work item: a group
// of tg target nodes of one leaf, split over nsl source slices (tg * nsl <= 32 lanes, nsl a power
// of two; lane = target + tg * slice), for one side (domain 0, or the target's own scatterer) and
// one block of RB right-hand sides.  The items are built once per tree (near_work_items) so that
// leaves of every size keep most lanes busy.
// - Near field: the warp streams the sources of the leaf's Neighbor list through two warp-private
//   shared-memory tiles of NW_TS sources; while it computes on one, asynchronous copies (cp.async,
//   16 bytes each: the 48-byte source record and the RB x 48 bytes of densities) fill the other,
//   and the warp synchronises only itself.  Per (source, target) pair it evaluates the kernel
//   scalars once and applies them to the RB right-hand sides.
// - Far field (L2P, Eq. 2.23 first term): the leaf's local expansions of the block's 3 RB columns
//   are staged in the same shared memory (in chunks of coefficients), and each slice adds the
//   coefficients q = slice (mod nsl) of B_l2p[a][q] D[col][q] to its partial sums.
// - The slices are summed by a fixed shuffle tree; the slice-0 lane of each target adds the side's
//   rows of the analytic self block (App. B) applied to x in double precision and stores the
//   side's three result rows.
constexpr int NW_TS = 16;    // sources per tile
static_assert(NW_TS == 16, "k_near_w stages a tile with two half-warps of 16 lanes");
constexpr int NW_WARPS = 4;  // warps per block, one per SM sub-partition; each fetches its own units
template <int RB>
struct WarpTile {
    float4 geo[3][NW_TS];     // source record: position hi + scatterer id bits, position lo + n_x, n_y n_z
    float4 dv[RB][3][NW_TS];  // densities (v0, v1), (v2, q0), (q1, q2) of the side, per RHS
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <int RB>
__global__ void __launch_bounds__(32 * NW_WARPS, 4) k_near_w(
    const int32_t *leaf_box, const int4 *__restrict__ items, int n_items, int n_units, int *next_unit, int64_t N, int64_t nr,
    int64_t rhs_base, int nsides,
    const int32_t *nbeg, const int32_t *nend, const int32_t *nbr_start, const int32_t *nbr_idx,
    const float4 *__restrict__ rec, const cx<float> *dens, const DomainConsts *dc, const int32_t *perm, int p2,
    int64_t nbox, const cx<float> *__restrict__ Bl2p, const cx<float> *__restrict__ D,
    const c64 *__restrict__ Mself, const c64 *__restrict__ x, c64 *y) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int rng_beg[NW_WARPS][32], rng_cum[NW_WARPS][33];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpTile<RB> *T = reinterpret_cast<WarpTile<RB> *>(smem_raw) + 2 * warp;  // two buffers per warp
    int *rb_ = rng_beg[warp], *rc_ = rng_cum[warp];
    // persistent warps: each takes the next unit (slab of side and RHS block, item) until none is
    // left; units run slab by slab, so that a slab's densities stay in L2, and within a slab
    // longest item first
    for (;;) {
        int unit = 0;
        if (lane == 0) unit = atomicAdd(next_unit, 1);
        unit = __shfl_sync(0xffffffffu, unit, 0);
        if (unit >= n_units) break;
        const int yslab = unit / n_items, item_id = unit - yslab * n_items;
        __syncwarp();  // the previous unit's shared-memory reads are done
        const int4 it = items[item_id];
        const int leaf = it.x, tg = it.z, nsl = it.w;
        const int64_t g = leaf_box[leaf];
        // the Neighbor leaves' node ranges and their running sum (a Neighbor list has at most 27 entries)
        const int nb0 = nbr_start[leaf], nnb = nbr_start[leaf + 1] - nb0;
        {
            int beg = 0, cnt = 0;
            if (lane < nnb) {
                const int b = nbr_idx[nb0 + lane];
                beg = nbeg[b];
                cnt = nend[b] - beg;
            }
            int incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane < nnb) { rb_[lane] = beg; rc_[lane] = incl - cnt; }
            if (lane == nnb - 1) rc_[nnb] = incl;
        }
        // slabs (RHS block, side); with the impedance boundary only the background side (k_local_rows
        // writes the scatterer rows)
        const int side = yslab % nsides;
        const int64_t rb0 = rhs_base + (int64_t)(yslab / nsides) * RB;
        const int nrb = (int)min((int64_t)RB, nr - rb0);
        // densities of the RHS past the block's end stay zero in both tiles
        for (int e = nrb * 3 * NW_TS + lane; e < RB * 3 * NW_TS; e += 32) {
            (&T[0].dv[0][0][0])[e] = make_float4(0.f, 0.f, 0.f, 0.f);
            (&T[1].dv[0][0][0])[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncwarp();
        const int nsrc = rc_[nnb];
        const int ti = lane % tg, sl = lane / tg;
        const bool busy = sl < nsl;
        const int a = nbeg[g] + it.y + ti;  // lanes past tg * nsl shadow a valid target and never store
        const float sgn = side == 0 ? -1.f : 1.f;  // domain 0 sees the scatterer normal reversed
        const float4 ra = rec[3 * a], rla = rec[3 * a + 1];
        const int adom = __float_as_int(ra.w);
        const cx<float> k = to<float>(dc[side == 0 ? 0 : adom].k);
        const cx<float> *dside = dens + (side * nr + rb0) * N * 6;
        // stage the tile of sources s0 .. s0 + NW_TS - 1 into buffer B: lane j (and j + 16) stages
        // source j, the lower half the record and the first RB/2 right-hand sides' densities, the upper
        // half the other RB/2; a lane's sources advance monotonically, so it follows its Neighbor range
        const int j = lane & (NW_TS - 1), hh = lane >> 4;
        const int64_t rstride = N * 6;
        int qcur = 0;
        auto stage = [&](WarpTile<RB> &B, int s0) {
            const int e = s0 + j;
            if (e < nsrc) {
                while (rc_[qcur + 1] <= e) ++qcur;
                const int64_t i = rb_[qcur] + (e - rc_[qcur]);
                if (hh == 0) {
#pragma unroll
                    for (int part = 0; part < 3; ++part) cp_async16(&B.geo[part][j], rec + 3 * i + part);
                }
                const cx<float> *src = dside + hh * (RB / 2) * rstride + 6 * i;
#pragma unroll
                for (int k = 0; k < RB / 2; ++k) {
                    if (hh * (RB / 2) + k < nrb) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) cp_async16(&B.dv[hh * (RB / 2) + k][c][j], src + k * rstride + 2 * c);
                    }
                }
            }
            cp_async_commit();
        };
        cx<float> acc[RB][3];
#pragma unroll
        for (int rr = 0; rr < RB; ++rr)
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[rr][c] = {0, 0};
        const int ntile = (nsrc + NW_TS - 1) / NW_TS;
        stage(T[0], 0);
        for (int t = 0; t < ntile; ++t) {
            if (t + 1 < ntile) stage(T[(t + 1) & 1], (t + 1) * NW_TS);
            else cp_async_commit();  // an empty group keeps "all but the newest group done" meaning tile t
            cp_async_wait1();
            __syncwarp();
            const WarpTile<RB> &B = T[t & 1];
            const int ns = busy ? min(NW_TS, nsrc - t * NW_TS) : 0;
            for (int u = sl; u < ns; u += nsl) {
                const float4 pa = B.geo[0][u], pb = B.geo[1][u], pc = B.geo[2][u];
                if (side == 1 && __float_as_int(pa.w) != adom) continue;  // a scatterer's sum runs over its own nodes
                const float rv3[3] = {(pa.x - ra.x) + (pb.x - rla.x), (pa.y - ra.y) + (pb.y - rla.y),
                                      (pa.z - ra.z) + (pb.z - rla.z)};
                const float R2 = rv3[0] * rv3[0] + rv3[1] * rv3[1] + rv3[2] * rv3[2];
                const float inv = R2 > 0.f ? rsqrt_(R2) : 0.f;  // the node itself drops out
                const float Rr = R2 * inv;
                const float nn[3] = {sgn * pb.w, sgn * pc.x, sgn * pc.y};
                const float nrv = nn[0] * rv3[0] + nn[1] * rv3[1] + nn[2] * rv3[2];
                const float w[3] = {nn[1] * rv3[2] - nn[2] * rv3[1], nn[2] * rv3[0] - nn[0] * rv3[2],
                                    nn[0] * rv3[1] - nn[1] * rv3[0]};
                cx<float> gs, cs;
                pair_scalars<float>(inv, Rr, k, gs, cs);
#pragma unroll
                for (int rr = 0; rr < RB; ++rr) {
                    const float4 a0 = B.dv[rr][0][u], a1 = B.dv[rr][1][u], a2 = B.dv[rr][2][u];
                    const cx<float> v[3] = {{a0.x, a0.y}, {a0.z, a0.w}, {a1.x, a1.y}};
                    const cx<float> qv[3] = {{a1.z, a1.w}, {a2.x, a2.y}, {a2.z, a2.w}};
                    cross_apply<float>(w, nrv, gs, cs, v, qv, acc[rr]);
                }
            }
            __syncwarp();  // the next stage overwrites this buffer
        }
        // far field: the local expansions of this side's domain at the leaf, for the block's columns
        // 3 rb0 .. 3 (rb0 + nrb) - 1, staged through the tiles' shared memory in chunks of qc
        // coefficients; on the scatterer side the warp's targets may lie in several scatterers, which
        // are taken in turn
        {
            cx<float> *Ds = reinterpret_cast<cx<float> *>(T);
            const int qc = min(p2, (int)(2 * sizeof(WarpTile<RB>) / sizeof(cx<float>)) / (3 * RB));
            const int ncol = 3 * nrb;
            const int64_t ncols = 3 * nr;
            const int mydom = side == 0 ? 0 : adom;
            const cx<float> *Ba = Bl2p + ((int64_t)side * N + a) * p2;
            unsigned pending = 0xffffffffu;
            while (pending) {
                const int d = __shfl_sync(0xffffffffu, mydom, __ffs(pending) - 1);
                const bool mine = mydom == d;
                pending &= ~__ballot_sync(0xffffffffu, mine);
                const cx<float> *Dg = D + ((int64_t)d * nbox + g) * ncols * p2 + 3 * rb0 * p2;
                for (int q0 = 0; q0 < p2; q0 += qc) {
                    const int qn = min(qc, p2 - q0);
                    __syncwarp();
                    for (int e = lane; e < ncol * qn; e += 32) {
                        const int col = e / qn, qq = e - col * qn;
                        Ds[col * qc + qq] = Dg[(int64_t)col * p2 + q0 + qq];
                    }
                    __syncwarp();
                    if (busy && mine) {
                        cx<float> bn = Ba[q0 + min(sl, qn - 1)];  // the next coefficient's load is in flight
                        for (int qq = sl; qq < qn; qq += nsl) {
                            const cx<float> bq = bn;
                            if (qq + nsl < qn) bn = Ba[q0 + qq + nsl];
#pragma unroll
                            for (int rr = 0; rr < RB; ++rr) {
                                if (rr < nrb) {
#pragma unroll
                                    for (int c = 0; c < 3; ++c) cfma(acc[rr][c], bq, Ds[(3 * rr + c) * qc + qq]);
                                }
                            }
                        }
                    }
                }
            }
        }
        // sum the slices of each target: lane ti + tg * sl, fixed tree over sl
        for (int off = nsl >> 1; off >= 1; off >>= 1) {
#pragma unroll
            for (int rr = 0; rr < RB; ++rr)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float re = __shfl_down_sync(0xffffffffu, acc[rr][c].re, off * tg);
                    const float im = __shfl_down_sync(0xffffffffu, acc[rr][c].im, off * tg);
                    if (sl < off) { acc[rr][c].re += re; acc[rr][c].im += im; }
                }
        }
        // the near + far sums of the slice-0 lanes go to shared memory (the tiles are free), and the
        // whole warp adds the side's rows of the self block (its Psi columns are diagonal) in double
        // precision and stores them, one (target, RHS, component) per lane and pass
        cx<float> *Ys = reinterpret_cast<cx<float> *>(T);  // [target][RB][3]
        __syncwarp();
        if (sl == 0) {
#pragma unroll
            for (int rr = 0; rr < RB; ++rr)
#pragma unroll
                for (int c = 0; c < 3; ++c) Ys[(ti * RB + rr) * 3 + c] = acc[rr][c];
        }
        __syncwarp();
        for (int o = lane; o < tg * 3 * nrb; o += 32) {
            const int t = o / (3 * nrb), rem = o - t * 3 * nrb, rr = rem / 3, c = rem - 3 * rr;
            const int64_t u = perm[nbeg[g] + it.y + t];
            const c64 *M = Mself + 36 * u + 18 * side + 6 * c;
            const c64 *xa = x + ((rb0 + rr) * N + u) * 6;
            const cx<float> f = Ys[(t * RB + rr) * 3 + c];
            c64 v = {(double)f.re, (double)f.im};
            cfma(v, M[0], xa[0]);
            cfma(v, M[1], xa[1]);
            cfma(v, M[2], xa[2]);
            cfma(v, M[3 + c], xa[3 + c]);
            y[((rb0 + rr) * N + u) * 6 + 3 * side + c] = v;
        }
    }
}

// Steps 4-5 for one to three right-hand sides in single precision, both sides of every pair in
// one pass.  One warp owns one unit: an item of near_work_items (tg targets of one leaf over nsl
// source slices) and one right-hand side.  The densities of k_prep tie the two sides together:
// v_1 = v_0 + s n with s = w t_j (n . Phi) (k_prep writes s beside the densities), and
// q_1 = -gamma_j q_0; on the scatterer side only sources in the target's own scatterer j count,
// so gamma_j is the target's and that side's q-part is -gamma_j times the sum of g_1 q_0.
// With w = n x r and U = w x v_0 + (n . r) v_0 (the bracket of Eq. 2.12 for the source normal n),
// the background's bracket is -U (it sees the normal -n) and the scatterer side's is U + s r,
// since (n x r) x n + (n . r) n = r for a unit n.  So the geometry and U are evaluated once per
// pair, and only the scalars g, c of grad'g = c r once per wavenumber.
// The sources go through two warp-private tiles of NS_TS (one per lane, cp.async) as in
// k_near_w; then the far field (L2P, Eq. 2.23 first term) and the rows of the analytic self block
// (App. B) of both sides, as in k_near_w's epilogue.
constexpr int NS_TS = 32;    // sources per tile, one staged by each lane
constexpr int NS_WARPS = 4;  // warps per block; each fetches its own units
struct SideTile {
    float4 geo[3][NS_TS];  // source record: position hi + scatterer id bits, position lo + n_x, n_y n_z
    float4 dv[3][NS_TS];   // background densities (v0, v1), (v2, q0), (q1, q2)
    float2 sj[NS_TS];      // s of the source
};

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}

__global__ void __launch_bounds__(32 * NS_WARPS, 6) k_near_ws(
    const int32_t *leaf_box, const int4 *__restrict__ items, int n_items, int n_units, int *next_unit, int64_t N,
    int64_t nr, const int32_t *nbeg, const int32_t *nend, const int32_t *nbr_start, const int32_t *nbr_idx,
    const float4 *__restrict__ rec, const cx<float> *dens, const cx<float> *sjump, const DomainConsts *dc,
    const int32_t *perm, int p2, int64_t nbox, const cx<float> *__restrict__ Bl2p, const cx<float> *__restrict__ D,
    const c64 *__restrict__ Mself, const c64 *__restrict__ x, c64 *y, bool side1) {
    __shared__ SideTile tiles[NS_WARPS][2];
    __shared__ int rng_beg[NS_WARPS][32], rng_cum[NS_WARPS][33];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    SideTile *T = tiles[warp];
    int *rb_ = rng_beg[warp], *rc_ = rng_cum[warp];
    for (;;) {
        int unit = 0;
        if (lane == 0) unit = atomicAdd(next_unit, 1);
        unit = __shfl_sync(0xffffffffu, unit, 0);
        if (unit >= n_units) break;
        const int64_t r = unit / n_items;
        const int item_id = unit - (int)r * n_items;
        __syncwarp();  // the previous unit's shared-memory reads are done
        const int4 it = items[item_id];
        const int leaf = it.x, tg = it.z, nsl = it.w;
        const int64_t g = leaf_box[leaf];
        // the Neighbor leaves' node ranges and their running sum (at most 27 entries)
        const int nb0 = nbr_start[leaf], nnb = nbr_start[leaf + 1] - nb0;
        {
            int beg = 0, cnt = 0;
            if (lane < nnb) {
                const int b = nbr_idx[nb0 + lane];
                beg = nbeg[b];
                cnt = nend[b] - beg;
            }
            int incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane < nnb) { rb_[lane] = beg; rc_[lane] = incl - cnt; }
            if (lane == nnb - 1) rc_[nnb] = incl;
        }
        __syncwarp();
        const int nsrc = rc_[nnb];
        const int ti = lane % tg, sl = lane / tg;
        const bool busy = sl < nsl;
        const int a = nbeg[g] + it.y + ti;  // lanes past tg * nsl shadow a valid target and never store
        const float4 ra = rec[3 * a], rla = rec[3 * a + 1];
        const int adom = __float_as_int(ra.w);
        const cx<float> k0 = to<float>(dc[0].k), kj = to<float>(dc[adom].k);
        const cx<float> *d0 = dens + r * N * 6;
        const cx<float> *sr = sjump + r * N;
        int qcur = 0;
        auto stage = [&](SideTile &B, int s0) {
            const int e = s0 + lane;
            if (e < nsrc) {
                while (rc_[qcur + 1] <= e) ++qcur;
                const int64_t i = rb_[qcur] + (e - rc_[qcur]);
#pragma unroll
                for (int part = 0; part < 3; ++part) cp_async16(&B.geo[part][lane], rec + 3 * i + part);
#pragma unroll
                for (int c = 0; c < 3; ++c) cp_async16(&B.dv[c][lane], d0 + 6 * i + 2 * c);
                if (side1) cp_async8(&B.sj[lane], sr + i);
            }
            cp_async_commit();
        };
        cx<float> acc0[3], acc1[3], bq[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) acc0[c] = acc1[c] = bq[c] = {0, 0};
        const int ntile = (nsrc + NS_TS - 1) / NS_TS;
        stage(T[0], 0);
        for (int t = 0; t < ntile; ++t) {
            if (t + 1 < ntile) stage(T[(t + 1) & 1], (t + 1) * NS_TS);
            else cp_async_commit();  // an empty group keeps "all but the newest group done" meaning tile t
            cp_async_wait1();
            __syncwarp();
            const SideTile &B = T[t & 1];
            const int ns = busy ? min(NS_TS, nsrc - t * NS_TS) : 0;
            for (int u = sl; u < ns; u += nsl) {
                const float4 pa = B.geo[0][u], pb = B.geo[1][u], pc = B.geo[2][u];
                const float rv[3] = {(pa.x - ra.x) + (pb.x - rla.x), (pa.y - ra.y) + (pb.y - rla.y),
                                     (pa.z - ra.z) + (pb.z - rla.z)};
                const float R2 = rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2];
                const float inv = R2 > 0.f ? rsqrt_(R2) : 0.f;  // the node itself drops out
                const float Rr = R2 * inv;
                const float nrv = pb.w * rv[0] + pc.x * rv[1] + pc.y * rv[2];
                const float w[3] = {pc.x * rv[2] - pc.y * rv[1], pc.y * rv[0] - pb.w * rv[2], pb.w * rv[1] - pc.x * rv[0]};
                const float4 a0 = B.dv[0][u], a1 = B.dv[1][u], a2 = B.dv[2][u];
                const cx<float> v[3] = {{a0.x, a0.y}, {a0.z, a0.w}, {a1.x, a1.y}};
                const cx<float> q[3] = {{a1.z, a1.w}, {a2.x, a2.y}, {a2.z, a2.w}};
                const cx<float> U[3] = {w[1] * v[2] - w[2] * v[1] + nrv * v[0], w[2] * v[0] - w[0] * v[2] + nrv * v[1],
                                        w[0] * v[1] - w[1] * v[0] + nrv * v[2]};
                cx<float> gs, cs;
                pair_scalars<float>(inv, Rr, k0, gs, cs);
                const cx<float> mc = {-cs.re, -cs.im};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    cfma(acc0[c], mc, U[c]);
                    cfma(acc0[c], gs, q[c]);
                }
                if (side1 && __float_as_int(pa.w) == adom) {
                    const float2 s2 = B.sj[u];
                    const cx<float> sc = {s2.x, s2.y};
                    pair_scalars<float>(inv, Rr, kj, gs, cs);
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        cfma(acc1[c], cs, U[c] + rv[c] * sc);
                        cfma(bq[c], gs, q[c]);
                    }
                }
            }
            __syncwarp();  // the next stage overwrites this buffer
        }
        if (side1) {
            const cx<float> mg = to<float>(dc[adom].gamma);
#pragma unroll
            for (int c = 0; c < 3; ++c) cfma(acc1[c], cx<float>{-mg.re, -mg.im}, bq[c]);
        }
        // far field of each side: the local expansion of the side's domain at the leaf, three
        // columns, staged through the tiles' shared memory in chunks of qc coefficients; on the
        // scatterer side the warp's targets may lie in several scatterers, taken in turn
        cx<float> *Ds = reinterpret_cast<cx<float> *>(T);
        const int qc = min(p2, (int)(2 * sizeof(SideTile) / sizeof(cx<float>)) / 3);
        auto l2p = [&](int side, cx<float>(&acc)[3]) {
            const int mydom = side == 0 ? 0 : adom;
            const cx<float> *Ba = Bl2p + ((int64_t)side * N + a) * p2;
            unsigned pending = 0xffffffffu;
            while (pending) {
                const int d = __shfl_sync(0xffffffffu, mydom, __ffs(pending) - 1);
                const bool mine = mydom == d;
                pending &= ~__ballot_sync(0xffffffffu, mine);
                const cx<float> *Dg = D + (((int64_t)d * nbox + g) * 3 * nr + 3 * r) * p2;
                for (int q0 = 0; q0 < p2; q0 += qc) {
                    const int qn = min(qc, p2 - q0);
                    __syncwarp();
                    for (int e = lane; e < 3 * qn; e += 32) {
                        const int col = e / qn, qq = e - col * qn;
                        Ds[col * qc + qq] = Dg[(int64_t)col * p2 + q0 + qq];
                    }
                    __syncwarp();
                    if (busy && mine) {
                        for (int qq = sl; qq < qn; qq += nsl) {
                            const cx<float> b = Ba[q0 + qq];
#pragma unroll
                            for (int c = 0; c < 3; ++c) cfma(acc[c], b, Ds[c * qc + qq]);
                        }
                    }
                }
            }
        };
        l2p(0, acc0);
        if (side1) l2p(1, acc1);
        // sum the slices of each target: lane ti + tg * sl, fixed tree over sl
        for (int off = nsl >> 1; off >= 1; off >>= 1) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float re = __shfl_down_sync(0xffffffffu, acc0[c].re, off * tg);
                float im = __shfl_down_sync(0xffffffffu, acc0[c].im, off * tg);
                if (sl < off) { acc0[c].re += re; acc0[c].im += im; }
                re = __shfl_down_sync(0xffffffffu, acc1[c].re, off * tg);
                im = __shfl_down_sync(0xffffffffu, acc1[c].im, off * tg);
                if (sl < off) { acc1[c].re += re; acc1[c].im += im; }
            }
        }
        // the slice-0 sums to shared memory (the tiles are free), then the whole warp adds the
        // rows of the self block in double precision and stores, one (target, row) per lane and pass
        cx<float> *Ys = reinterpret_cast<cx<float> *>(T);  // [target][6]
        __syncwarp();
        if (sl == 0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) { Ys[ti * 6 + c] = acc0[c]; Ys[ti * 6 + 3 + c] = acc1[c]; }
        }
        __syncwarp();
        const int nrow = side1 ? 6 : 3;
        for (int o = lane; o < tg * nrow; o += 32) {
            const int t = o / nrow, row = o - t * nrow, side = row / 3, c = row - 3 * side;
            const int64_t u = perm[nbeg[g] + it.y + t];
            const c64 *M = Mself + 36 * u + 18 * side + 6 * c;
            const c64 *xa = x + (r * N + u) * 6;
            const cx<float> f = Ys[t * 6 + row];
            c64 v = {(double)f.re, (double)f.im};
            cfma(v, M[0], xa[0]);
            cfma(v, M[1], xa[1]);
            cfma(v, M[2], xa[2]);
            cfma(v, M[3 + c], xa[3 + c]);
            y[(r * N + u) * 6 + row] = v;
        }
    }
}

// Steps 4-5 for 32 or more right-hand sides in single precision, one lane per right-hand side,
// both sides of every pair in one pass (the relations of k_near_ws: v_1 = v_0 + s n,
// q_1 = -gamma_j q_0).  A warp owns one unit: a group of at most NR_TT targets of one leaf and a
// block of 32 right-hand sides.  The sources of the leaf's Neighbor list go by in tiles of 32:
// - pair phase: lane l takes source l of the tile and evaluates, against every target of the
//   group, w = n x r, n.r and r, the background's scalars (-c_0, g_0) and the scatterer side's
//   (c_1, -gamma_j g_1; zero where the source lies in another scatterer or past the list's end)
//   into shared memory;
// - right-hand-side phase: every lane reads its own (v_0, q_0, s) of each source (node-major copy
//   k_dens_node_major; the next source's loads in flight while the current one is applied) and, per
//   target, U = w x v_0 + (n.r) v_0 once, then acc_0 += -c_0 U + g_0 q_0 and
//   acc_1 += c_1 (U + s r) - gamma_j g_1 q_0; a pair's scalars serve 32 right-hand sides.
// Then L2P (Eq. 2.23 first term) of both sides from the lane's three columns of the leaf's local
// expansions, and the rows of the analytic self block (App. B) in double precision; each lane
// stores its right-hand side's rows.  With the impedance boundary (side1 false) the background
// side only (k_local_rows writes the scatterer rows).
constexpr int NR_TT = 8;   // targets per unit
constexpr int NR_WARPS = 4;
struct RhsTile {
    float4 ps[NR_TT][32][4];  // (w, n.r), (-c_0, g_0), (c_1, -gamma g_1), (r, 0) per target and source
    float4 tp[NR_TT][2];      // target position hi + scatterer id bits, position lo
    float4 tk[NR_TT];         // the target's scatterer wavenumber k_j and -gamma_j
};

__global__ void __launch_bounds__(32 * NR_WARPS, 3) k_near_r(
    const int32_t *leaf_box, const int4 *__restrict__ groups, int n_groups, int n_units, int *next_unit, int64_t N,
    int64_t nr, bool side1, const int32_t *nbeg, const int32_t *nend, const int32_t *nbr_start,
    const int32_t *nbr_idx, const float4 *__restrict__ rec, const float4 *densS, const DomainConsts *dc,
    const int32_t *perm, int p2, int64_t nbox, const cx<float> *__restrict__ Bl2p, const cx<float> *__restrict__ D,
    const c64 *__restrict__ Mself, const c64 *__restrict__ x, c64 *y, int slab0, int slab_lf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int rng_beg[NR_WARPS][32], rng_cum[NR_WARPS][33];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    RhsTile &S = reinterpret_cast<RhsTile *>(smem_raw)[warp];
    int *rb_ = rng_beg[warp], *rc_ = rng_cum[warp];
    const cx<float> k0 = to<float>(dc[0].k);
    for (;;) {
        int unit = 0;
        if (lane == 0) unit = atomicAdd(next_unit, 1);
        unit = __shfl_sync(0xffffffffu, unit, 0);
        if (unit >= n_units) break;
        // slabs of 32 right-hand sides from slab0 on; the launch's last one (slab_lf) takes its
        // groups longest first
        const int slab = slab0 + unit / n_groups, grp = unit - (slab - slab0) * n_groups;
        const int64_t r = (int64_t)slab * 32 + lane;  // this lane's right-hand side
        __syncwarp();  // the previous unit's shared-memory reads are done
        const int4 gi = groups[slab == slab_lf ? n_groups + grp : grp];
        const int leaf = gi.x, ntg = gi.z;
        const int64_t g = leaf_box[leaf];
        const int tbase = nbeg[g] + gi.y;
        const int nb0 = nbr_start[leaf], nnb = nbr_start[leaf + 1] - nb0;
        {
            int beg = 0, cnt = 0;
            if (lane < nnb) {
                const int b = nbr_idx[nb0 + lane];
                beg = nbeg[b];
                cnt = nend[b] - beg;
            }
            int incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane < nnb) { rb_[lane] = beg; rc_[lane] = incl - cnt; }
            if (lane == nnb - 1) rc_[nnb] = incl;
        }
        if (lane < ntg) {
            const int a = tbase + lane;
            const float4 ta = rec[3 * a];
            S.tp[lane][0] = ta;
            S.tp[lane][1] = rec[3 * a + 1];
            const int td = __float_as_int(ta.w);
            const cx<float> kt = to<float>(dc[td].k), gm = to<float>(dc[td].gamma);
            S.tk[lane] = make_float4(kt.re, kt.im, -gm.re, -gm.im);
        }
        __syncwarp();
        const int nsrc = rc_[nnb];
        // node-major (v_0, q_0, s) of this lane's right-hand side: source i at dl + 128 i
        const float4 *dl = densS + ((int64_t)slab * N * 32 + lane) * 4;
        cx<float> acc0[NR_TT][3], acc1[NR_TT][3];
#pragma unroll
        for (int t = 0; t < NR_TT; ++t)
#pragma unroll
            for (int c = 0; c < 3; ++c) acc0[t][c] = acc1[t][c] = {0, 0};
        int qcur = 0;
        for (int s0 = 0; s0 < nsrc; s0 += 32) {
            // pair phase: source s0 + lane against the group's targets
            const int e = s0 + lane;
            const bool valid = e < nsrc;
            int i = rb_[0];
            if (valid) {
                while (rc_[qcur + 1] <= e) ++qcur;
                i = rb_[qcur] + (e - rc_[qcur]);
            }
            const float4 pa = rec[3 * i], pb = rec[3 * i + 1], pc = rec[3 * i + 2];
            const int sdom = __float_as_int(pa.w);
            const float nn[3] = {pb.w, pc.x, pc.y};
#pragma unroll
            for (int t = 0; t < NR_TT; ++t) {
                if (t < ntg) {
                    const float4 ta = S.tp[t][0], tl = S.tp[t][1];
                    const float rv[3] = {(pa.x - ta.x) + (pb.x - tl.x), (pa.y - ta.y) + (pb.y - tl.y),
                                         (pa.z - ta.z) + (pb.z - tl.z)};
                    const float R2 = rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2];
                    const float inv = R2 > 0.f ? rsqrt_(R2) : 0.f;  // the node itself drops out
                    const float Rr = R2 * inv;
                    const float nrv = nn[0] * rv[0] + nn[1] * rv[1] + nn[2] * rv[2];
                    cx<float> g0, c0, g1 = {0, 0}, c1 = {0, 0};
                    pair_scalars<float>(inv, Rr, k0, g0, c0);
                    if (!valid) g0 = c0 = cx<float>{0.f, 0.f};
                    if (side1 && valid && sdom == __float_as_int(ta.w)) {
                        const float4 tk = S.tk[t];
                        pair_scalars<float>(inv, Rr, cx<float>{tk.x, tk.y}, g1, c1);
                        g1 = cx<float>{tk.z, tk.w} * g1;  // -gamma_j g_1: q_1 = -gamma_j q_0
                    }
                    S.ps[t][lane][0] = make_float4(nn[1] * rv[2] - nn[2] * rv[1], nn[2] * rv[0] - nn[0] * rv[2],
                                                   nn[0] * rv[1] - nn[1] * rv[0], nrv);
                    S.ps[t][lane][1] = make_float4(-c0.re, -c0.im, g0.re, g0.im);
                    S.ps[t][lane][2] = make_float4(c1.re, c1.im, g1.re, g1.im);
                    S.ps[t][lane][3] = make_float4(rv[0], rv[1], rv[2], 0.f);
                }
            }
            __syncwarp();
            // right-hand-side phase
            const int nsv = min(32, nsrc - s0);
            int ic = __shfl_sync(0xffffffffu, i, 0);
            float4 d0 = dl[128 * (int64_t)ic], d1 = dl[128 * (int64_t)ic + 1], d2 = dl[128 * (int64_t)ic + 2],
                   d3 = dl[128 * (int64_t)ic + 3];
            for (int sv = 0; sv < nsv; ++sv) {
                float4 n0 = d0, n1 = d1, n2 = d2, n3 = d3;
                const int in = __shfl_sync(0xffffffffu, i, (sv + 1) & 31);
                if (sv + 1 < nsv) {
                    n0 = dl[128 * (int64_t)in];
                    n1 = dl[128 * (int64_t)in + 1];
                    n2 = dl[128 * (int64_t)in + 2];
                    n3 = dl[128 * (int64_t)in + 3];
                }
                const cx<float> v[3] = {{d0.x, d0.y}, {d0.z, d0.w}, {d1.x, d1.y}};
                const cx<float> q[3] = {{d1.z, d1.w}, {d2.x, d2.y}, {d2.z, d2.w}};
                const cx<float> sj = {d3.x, d3.y};
#pragma unroll
                for (int t = 0; t < NR_TT; ++t) {
                    if (t < ntg) {
                        const float4 p0 = S.ps[t][sv][0], p1 = S.ps[t][sv][1];
                        const float w[3] = {p0.x, p0.y, p0.z};
                        const cx<float> U[3] = {w[1] * v[2] - w[2] * v[1] + p0.w * v[0],
                                                w[2] * v[0] - w[0] * v[2] + p0.w * v[1],
                                                w[0] * v[1] - w[1] * v[0] + p0.w * v[2]};
                        const cx<float> mc0 = {p1.x, p1.y}, g0 = {p1.z, p1.w};
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            cfma(acc0[t][c], mc0, U[c]);
                            cfma(acc0[t][c], g0, q[c]);
                        }
                        if (side1) {
                            const float4 p2v = S.ps[t][sv][2], p3 = S.ps[t][sv][3];
                            const cx<float> c1 = {p2v.x, p2v.y}, g1 = {p2v.z, p2v.w};
                            const float rr[3] = {p3.x, p3.y, p3.z};
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                cfma(acc1[t][c], c1, U[c] + rr[c] * sj);
                                cfma(acc1[t][c], g1, q[c]);
                            }
                        }
                    }
                }
                d0 = n0; d1 = n1; d2 = n2; d3 = n3;
            }
            __syncwarp();  // the next tile's pair phase overwrites the scalars
        }
        // far field of each side: this lane's three columns of the leaf's local expansion of the
        // side's domain (on the scatterer side each target's own scatterer: the group's scatterers
        // in turn); the targets' L2P rows are staged in the scalars' shared memory, chunks of qc
        // coefficients, and the lane's expansion coefficients are loaded two coefficients ahead
        auto l2p = [&](int side, cx<float>(&acc)[NR_TT][3]) {
            cx<float> *Bs = reinterpret_cast<cx<float> *>(&S.ps[0][0][0]);
            constexpr int BS_CAP = (int)(sizeof(S.ps) / sizeof(cx<float>));
            const int qc = min(p2, BS_CAP / NR_TT);
            const int64_t ncols = 3 * nr;
            unsigned pending = (1u << ntg) - 1u;
            while (pending) {
                const int d = side == 0 ? 0 : __float_as_int(S.tp[__ffs(pending) - 1][0].w);
                unsigned mine = 0;
                for (int t = 0; t < ntg; ++t)
                    if (side == 0 || __float_as_int(S.tp[t][0].w) == d) mine |= 1u << t;
                pending &= ~mine;
                const cx<float> *Dr = D + (((int64_t)d * nbox + g) * ncols + 3 * r) * p2;
                for (int q0 = 0; q0 < p2; q0 += qc) {
                    const int qn = min(qc, p2 - q0);
                    __syncwarp();
                    for (int e = lane; e < ntg * qn; e += 32) {
                        const int t = e / qn, qq = e - t * qn;
                        Bs[t * qc + qq] = Bl2p[((int64_t)side * N + tbase + t) * p2 + q0 + qq];
                    }
                    __syncwarp();
                    cx<float> e1[3], e2[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        e1[c] = Dr[c * p2 + q0];
                        e2[c] = Dr[c * p2 + q0 + min(1, qn - 1)];
                    }
                    for (int qq = 0; qq < qn; ++qq) {
                        const cx<float> dq[3] = {e1[0], e1[1], e1[2]};
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            e1[c] = e2[c];
                            if (qq + 2 < qn) e2[c] = Dr[c * p2 + q0 + qq + 2];
                        }
#pragma unroll
                        for (int t = 0; t < NR_TT; ++t) {
                            if ((mine >> t) & 1u) {
                                const cx<float> b = Bs[t * qc + qq];
#pragma unroll
                                for (int c = 0; c < 3; ++c) cfma(acc[t][c], b, dq[c]);
                            }
                        }
                    }
                }
            }
        };
        l2p(0, acc0);
        if (side1) l2p(1, acc1);
        // the rows of the self block (Psi columns diagonal) in double precision, stored
#pragma unroll
        for (int t = 0; t < NR_TT; ++t) {
            if (t < ntg) {
                const int64_t u = perm[tbase + t];
                const c64 *xa = x + (r * N + u) * 6;
                c64 *ya = y + (r * N + u) * 6;
                const c64 x0 = xa[0], x1 = xa[1], x2 = xa[2];
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    if (side == 1 && !side1) break;
                    const c64 *M = Mself + 36 * u + 18 * side;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const cx<float> a = side == 0 ? acc0[t][c] : acc1[t][c];
                        c64 v = {(double)a.re, (double)a.im};
                        cfma(v, M[6 * c], x0);
                        cfma(v, M[6 * c + 1], x1);
                        cfma(v, M[6 * c + 2], x2);
                        cfma(v, M[6 * c + 3 + c], xa[3 + c]);
                        ya[3 * side + c] = v;
                    }
                }
            }
        }
    }
}

// Packed rotation-form tables, in the order k_m2l_rot reads them.  Polar rotations (per offset,
// forward then back): per degree n = 0..p-1 the folded blocks (see k_m2l_rot) one after the
// other, each row-major, real: the a-block, (n+1) x (n+1) with rows m' = 0..n and columns
// m = 0..n, then the b-block, n x n with rows and columns 1..n.  With D the dense polar block
// (row = output order, column = input order):
//   forward a-block: row 0: D[0][0], (D[0][m] + D[0][-m]) / 2; rows m' >= 1: 2 D[m'][0],
//                    D[m'][m] + D[m'][-m];   b-block: D[m'][m] - D[m'][-m];
//   back a-block:    row 0 as forward; rows m' >= 1: D[m'][0], (D[m'][m] + D[m'][-m]) / 2;
//                    b-block: (D[m'][m] - D[m'][-m]) / 2,
// so that the back rotation returns P + Q and P - Q for the orders +m' and -m'.  Azimuthal phases
// (per offset, forward then back): the diagonal, p2 complex.  Coaxial Z (per domain, level and
// offset length): the order blocks m = -(p-1)..p-1, each (p-|m|) x (p-|m|) row-major with the row
// the output degree n' - |m| and the column the input degree n - |m|.  The dense projected tables
// are stored input-major, T[c][r] at c * p2 + r.  The polar factors must be real, mirror
// symmetric (D[-m'][-m] = D[m'][m]) and the azimuthal ones diagonal (to rounding); the largest
// departures are recorded in dev[0] (imaginary parts), dev[1] (off-diagonal entries), dev[2]
// (mirror asymmetry) and dev[3] (phases of orders -m that are not the conjugates of those of m)
// as the bit patterns of non-negative doubles, so that atomicMax orders them.
__global__ void k_pack_rot_d(int p, const c64 *Tf, const c64 *Tb, double *D64, float *D32, unsigned long long *dev) {
    const int p2 = p * p, nrot = rot_off(p);
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)316 * 2 * nrot) return;
    const int64_t o = idx / (2 * nrot);
    const int within = (int)(idx - o * 2 * nrot), fb = within / nrot, i = within - fb * nrot;
    int n = 0;
    while (rot_off(n + 1) <= i) ++n;
    const int loc = i - rot_off(n);
    const bool ablk = loc < (n + 1) * (n + 1);
    const int mp = ablk ? loc / (n + 1) : 1 + (loc - (n + 1) * (n + 1)) / n;
    const int m = ablk ? loc % (n + 1) : 1 + (loc - (n + 1) * (n + 1)) % n;
    const c64 *T = (fb == 0 ? Tf : Tb) + o * p2 * p2;
    auto Dv = [&](int row, int col) { return T[(int64_t)(n * n + n + col) * p2 + n * n + n + row]; };
    const c64 d1 = Dv(mp, m), d2 = Dv(mp, -m);
    double v;
    if (ablk && mp == 0) v = m == 0 ? d1.re : 0.5 * (d1.re + d2.re);
    else if (ablk && m == 0) v = fb == 0 ? 2.0 * d1.re : d1.re;
    else if (ablk) v = (fb == 0 ? 1.0 : 0.5) * (d1.re + d2.re);
    else v = (fb == 0 ? 1.0 : 0.5) * (d1.re - d2.re);
    D64[idx] = v;
    D32[idx] = (float)v;
    const c64 e1 = Dv(-mp, -m), e2 = Dv(-mp, m);
    const double asym = fmax(fabs(e1.re - d1.re), fabs(e2.re - d2.re));
    atomicMax(&dev[0], (unsigned long long)__double_as_longlong(fmax(fabs(d1.im), fabs(d2.im))));
    atomicMax(&dev[2], (unsigned long long)__double_as_longlong(asym));
}
__global__ void k_pack_rot_p(int p, const c64 *Tf, const c64 *Tb, c64 *P64, c32 *P32, unsigned long long *dev) {
    const int p2 = p * p;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)316 * 2 * p2 * p2) return;
    const int64_t o = idx / (2 * p2 * p2);
    const int within = (int)(idx - o * 2 * p2 * p2), fb = within / (p2 * p2), e = within - fb * p2 * p2;
    const int c = e / p2, r = e - c * p2;
    const c64 v = (fb == 0 ? Tf : Tb)[o * p2 * p2 + e];
    if (c == r) {
        P64[(o * 2 + fb) * p2 + r] = v;
        P32[(o * 2 + fb) * p2 + r] = c32{(float)v.re, (float)v.im};
        int n = 0;  // the phase of order -m must be the conjugate of that of m
        while ((n + 1) * (n + 1) <= r) ++n;
        const int rm = 2 * (n * n + n) - r;
        const c64 w = (fb == 0 ? Tf : Tb)[o * p2 * p2 + (int64_t)rm * p2 + rm];
        atomicMax(&dev[3], (unsigned long long)__double_as_longlong(fmax(fabs(v.re - w.re), fabs(v.im + w.im))));
    } else {
        atomicMax(&dev[1], (unsigned long long)__double_as_longlong(sqrt(v.re * v.re + v.im * v.im)));
    }
}
template <typename R>
__global__ void k_pack_rot_z(int p, int64_t nz, const cx<R> *Z, cx<R> *Zp) {
    const int p2 = p * p, ncoax = p * (2 * p * p + 1) / 3;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nz * ncoax) return;
    const int64_t t = idx / ncoax;
    const int i = (int)(idx - t * ncoax);
    int m = -(p - 1), base = 0;
    while (base + (p - abs(m)) * (p - abs(m)) <= i) { base += (p - abs(m)) * (p - abs(m)); ++m; }
    const int am = abs(m), w = p - am, loc = i - base, row = loc / w, col = loc - row * w;
    const int np = am + row, n = am + col;  // output degree n', input degree n
    Zp[idx] = Z[t * p2 * p2 + (int64_t)(n * n + n + m) * p2 + np * np + np + m];
}

// Mirror check of the packed coaxial blocks (the folded rotation form applies Z^m to both
// halves): k_z_scale records each table's largest |Z| in zmax[t], k_check_z_mirror the largest
// |Z^{-m} - Z^m| / zmax[t]; both as bit patterns of non-negative doubles.
template <typename R>
__global__ void k_z_scale(int p, int64_t nz, const cx<R> *Zp, unsigned long long *zmax) {
    const int ncoax = p * (2 * p * p + 1) / 3;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nz * ncoax) return;
    const cx<R> a = Zp[idx];
    atomicMax(&zmax[idx / ncoax], (unsigned long long)__double_as_longlong(sqrt((double)a.re * a.re + (double)a.im * a.im)));
}
template <typename R>
__global__ void k_check_z_mirror(int p, int64_t nz, const cx<R> *Zp, const unsigned long long *zmax,
                                 unsigned long long *dev) {
    const int ncoax = p * (2 * p * p + 1) / 3;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nz * ncoax) return;
    const int64_t t = idx / ncoax;
    const int i = (int)(idx - t * ncoax);
    int m = -(p - 1), base = 0;
    while (base + (p - abs(m)) * (p - abs(m)) <= i) { base += (p - abs(m)) * (p - abs(m)); ++m; }
    if (m >= 0) return;
    int bm = base;  // block of order -m
    for (int k = m; k < -m; ++k) bm += (p - abs(k)) * (p - abs(k));
    const cx<R> a = Zp[t * ncoax + i], b = Zp[t * ncoax + bm + (i - base)];
    const double dr = (double)a.re - (double)b.re, di = (double)a.im - (double)b.im;
    const double scale = __longlong_as_double((long long)zmax[t]);
    const double rel = scale > 0 ? sqrt(dr * dr + di * di) / scale : 0.0;
    atomicMax(dev, (unsigned long long)__double_as_longlong(rel));
}

// ---------------------------------------------------------------- adjoint (transposed) product
// y = A^T x for the operator of Eq. (2.12) (complex bilinear transpose).  Gathering the transposed
// pair blocks at a column node b gives, for each domain d of b's two equations (d = 0 and d = the
// scatterer j of b),
//   Phi rows:  w_b T_d(b) u,   u = -sum_i n'_i grad phi_i + n' div phi + (n'.grad) phi   at s_b,
//   Psi rows:  w_b sigma_d phi(s_b),   sigma_0 = -1, sigma_j = gamma_j,
// with n' = -n_b (d = 0) or n_b (d = j), T_0 = I, and phi_i(s) = sum_{a != b} g_d(|s - s_a|) x_{a,i}
// the potential of unweighted monopoles taken from the d rows of x (rows 0-2 of every node for
// d = 0, rows 3-5 of the nodes of scatterer j).  grad phi at s_b is sum_a c_d (s_b - s_a) x_a with
// the c of grad'g = c r.  The far part of phi and grad phi comes from a monopole P2M, the usual
// M2M, M2L and L2L, and L2P with the basis and its gradient; the transposed self block is added
// in double precision.

// dens[side][r][i][0..2] = x_{perm(i), 3 side + c}, unweighted, sorted order
template <typename R>
__global__ void k_prep_adj(int64_t N, int64_t nr, const c64 *x, const int32_t *perm, int sides, cx<R> *dens) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t r = blockIdx.y;
    if (i >= N) return;
    const c64 *xa = x + (r * N + perm[i]) * 6;
    for (int side = 0; side < 2; ++side) {
        cx<R> *dn = dens + ((side * nr + r) * N + i) * 6;
        for (int c = 0; c < 3; ++c) dn[c] = side < sides ? to<R>(xa[3 * side + c]) : cx<R>{0, 0};
    }
}

// monopole P2M: C[d][leaf][3 r + c][q] = sum over the leaf's nodes of domain d of b0(i, q) x_{i,c},
// with b0 the monopole row of the P2M basis (Eqs. 2.18-2.19)
template <typename R>
__global__ void k_p2m_adj(const int32_t *leaf_box, int64_t N, int64_t nr, int p2, int64_t nbox, const int32_t *nbeg,
                          const int32_t *nend, const int32_t *dom, const cx<R> *dens, const cx<R> *Bp2m, cx<R> *C) {
    const int64_t g = leaf_box[blockIdx.x];
    const int d = blockIdx.y;
    const int64_t r = blockIdx.z;
    const int side = d == 0 ? 0 : 1;
    const int i0 = nbeg[g], i1 = nend[g];
    for (int q = threadIdx.x; q < p2; q += blockDim.x) {
        cx<R> acc[3] = {{0, 0}, {0, 0}, {0, 0}};
        for (int i = i0; i < i1; ++i) {
            if (d > 0 && dom[i] != d) continue;
            const cx<R> b0 = Bp2m[((int64_t)side * N + i) * 4 * p2 + q];
            const cx<R> *dn = dens + ((side * nr + r) * N + i) * 6;
#pragma unroll
            for (int c = 0; c < 3; ++c) cfma(acc[c], dn[c], b0);
        }
        for (int c = 0; c < 3; ++c) C[(((int64_t)d * nbox + g) * 3 * nr + 3 * r + c) * p2 + q] = acc[c];
    }
}

template <typename R>
struct AdjTile {
    V4<R> pa[128];      // position (high part) and scatterer id
    V4<R> pb[128];      // position low part (double-float only)
    cx<R> xv[3][128];   // the side's monopole strengths
};
template <typename R>
union AdjSmem {
    AdjTile<R> tile;
    cx<R> red[12][128];  // per source slice: phi (3) and grad phi (9)
};

// near field, L2P (value and gradient), assembly and the transposed self block for one leaf;
// threads split as (target, source slice) like k_near, both domains one after the other; grid
// (leaf, right-hand side)
template <typename R, bool DOUBLE_FLOAT>
__global__ void __launch_bounds__(128) k_near_adj(const int32_t *leaf_box, int64_t N, int64_t nr, int p2, int64_t nbox,
                                                  const int32_t *nbeg, const int32_t *nend, const int32_t *nbr_start,
                                                  const int32_t *nbr_idx, const R *pos_hi, const R *pos_lo,
                                                  const double *nrm, const double *w, const int32_t *dom,
                                                  const int32_t *perm, const cx<R> *dens, const DomainConsts *dc,
                                                  const cx<R> *Bl2p, const cx<R> *Bl2pg, const cx<R> *D,
                                                  const c64 *Mself, const c64 *x, c64 *y, const int64_t *cache_base,
                                                  const V4<R> *cache) {
    __shared__ AdjSmem<R> S;
    __shared__ int rng_beg[32], rng_cum[33];
    AdjTile<R> &T = S.tile;
    const int64_t g = leaf_box[blockIdx.x];
    const int nb0 = nbr_start[blockIdx.x], nnb = nbr_start[blockIdx.x + 1] - nb0;
    if (threadIdx.x == 0) {
        int cum = 0;
        for (int q = 0; q < nnb; ++q) {
            const int b = nbr_idx[nb0 + q];
            rng_beg[q] = nbeg[b];
            rng_cum[q] = cum;
            cum += nend[b] - nbeg[b];
        }
        rng_cum[nnb] = cum;
    }
    __syncthreads();
    const int nsrc = rng_cum[nnb];
    const int t0 = nbeg[g], t1 = nend[g], NT = t1 - t0;
    for (int64_t r = blockIdx.y; r < nr; r += gridDim.y) {  // right-hand sides across the grid
        for (int tb = t0; tb < t1; tb += 128) {
            const int nt = min(128, t1 - tb);
            const int nsl = 128 / nt;
            const int tg = threadIdx.x % nt, slice = threadIdx.x / nt;
            const bool active = slice < nsl;
            const int a = tb + tg;
            const R ax = pos_hi[3 * a], ay = pos_hi[3 * a + 1], az = pos_hi[3 * a + 2];
            R alx = 0, aly = 0, alz = 0;
            if (DOUBLE_FLOAT) { alx = pos_lo[3 * a]; aly = pos_lo[3 * a + 1]; alz = pos_lo[3 * a + 2]; }
            const int adom = dom[a];
            const R adom_r = (R)adom;
            const V4<R> *cs0 = cache ? cache + 2 * cache_base[blockIdx.x] + (tb - t0 + tg) : nullptr;
            c64 yacc[6] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
            for (int side = 0; side < 2; ++side) {
                const int d = side == 0 ? 0 : adom;
                const cx<R> k = to<R>(dc[d].k);
                cx<R> phi[3], gphi[3][3];  // gphi[k][c] = d phi_c / d s_k
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    phi[c] = {0, 0};
#pragma unroll
                    for (int kk = 0; kk < 3; ++kk) gphi[kk][c] = {0, 0};
                }
                for (int s0 = 0; s0 < nsrc; s0 += 128) {
                    __syncthreads();
                    {
                        const int e = s0 + threadIdx.x;
                        if (e < nsrc) {
                            const int q = source_range(rng_cum, nnb, e);
                            const int i = rng_beg[q] + (e - rng_cum[q]);
                            T.pa[threadIdx.x] = V4<R>{pos_hi[3 * i], pos_hi[3 * i + 1], pos_hi[3 * i + 2], (R)dom[i]};
                            R lo[3] = {0, 0, 0};
                            if (DOUBLE_FLOAT) { lo[0] = pos_lo[3 * i]; lo[1] = pos_lo[3 * i + 1]; lo[2] = pos_lo[3 * i + 2]; }
                            T.pb[threadIdx.x] = V4<R>{lo[0], lo[1], lo[2], 0};
                            const cx<R> *dn = dens + ((side * nr + r) * N + i) * 6;
                            for (int c = 0; c < 3; ++c) T.xv[c][threadIdx.x] = dn[c];
                        }
                    }
                    __syncthreads();
                    const int ns = min(128, nsrc - s0);
                    if (active)
                        for (int u = slice; u < ns; u += nsl) {
                            const V4<R> pa = T.pa[u];
                            if (side == 1 && pa.w != adom_r) continue;  // scatterer d sums over its own nodes
                            const V4<R> pb = T.pb[u];
                            R rx = pa.x - ax, ry = pa.y - ay, rz = pa.z - az;
                            if (DOUBLE_FLOAT) { rx += pb.x - alx; ry += pb.y - aly; rz += pb.z - alz; }
                            cx<R> gs, cs;
                            if (cs0) {
                                const V4<R> sv = cs0[((int64_t)side * nsrc + s0 + u) * NT];
                                gs = {sv.x, sv.y};
                                cs = {sv.z, sv.w};
                            } else {
                                const R R2 = rx * rx + ry * ry + rz * rz;
                                const R inv = R2 > (R)0 ? rsqrt_(R2) : (R)0;  // the node itself drops out
                                pair_scalars<R>(inv, R2 * inv, k, gs, cs);
                            }
                            // grad phi at the target: c (s_target - s_source) = -c r
                            const cx<R> cr[3] = {-rx * cs, -ry * cs, -rz * cs};
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                const cx<R> xc = T.xv[c][u];
                                cfma(phi[c], gs, xc);
#pragma unroll
                                for (int kk = 0; kk < 3; ++kk) cfma(gphi[kk][c], cr[kk], xc);
                            }
                        }
                }
                // sum the source slices in a fixed order
                __syncthreads();
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    S.red[c][threadIdx.x] = phi[c];
#pragma unroll
                    for (int kk = 0; kk < 3; ++kk) S.red[3 + 3 * kk + c][threadIdx.x] = gphi[kk][c];
                }
                __syncthreads();
                if (threadIdx.x < nt) {
                    c64 ph[3], gp[3][3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        cx<R> v = S.red[c][threadIdx.x];
                        for (int sl = 1; sl < nsl; ++sl) v += S.red[c][sl * nt + threadIdx.x];
                        ph[c] = c64{(double)v.re, (double)v.im};
#pragma unroll
                        for (int kk = 0; kk < 3; ++kk) {
                            cx<R> t = S.red[3 + 3 * kk + c][threadIdx.x];
                            for (int sl = 1; sl < nsl; ++sl) t += S.red[3 + 3 * kk + c][sl * nt + threadIdx.x];
                            gp[kk][c] = c64{(double)t.re, (double)t.im};
                        }
                    }
                    // far field: L2P of phi and grad phi from the leaf's local expansions
                    const cx<R> *Dl = D + (((int64_t)d * nbox + g) * 3 * nr + 3 * r) * p2;
                    const cx<R> *B = Bl2p + ((int64_t)side * N + a) * p2;
                    const cx<R> *G = Bl2pg + ((int64_t)side * N + a) * 3 * p2;
                    cx<R> fp[3] = {{0, 0}, {0, 0}, {0, 0}}, fg[3][3];
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int kk = 0; kk < 3; ++kk) fg[kk][c] = {0, 0};
                    for (int q = 0; q < p2; ++q) {
                        const cx<R> b = B[q], gx = G[q], gy = G[p2 + q], gz = G[2 * p2 + q];
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            const cx<R> dq = Dl[c * p2 + q];
                            cfma(fp[c], dq, b);
                            cfma(fg[0][c], dq, gx);
                            cfma(fg[1][c], dq, gy);
                            cfma(fg[2][c], dq, gz);
                        }
                    }
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        ph[c] += c64{(double)fp[c].re, (double)fp[c].im};
#pragma unroll
                        for (int kk = 0; kk < 3; ++kk) gp[kk][c] += c64{(double)fg[kk][c].re, (double)fg[kk][c].im};
                    }
                    // assembly in double precision
                    const double sg = side == 0 ? -1.0 : 1.0;
                    const double nb[3] = {nrm[3 * a], nrm[3 * a + 1], nrm[3 * a + 2]};
                    const double np_[3] = {sg * nb[0], sg * nb[1], sg * nb[2]};
                    const c64 div = gp[0][0] + gp[1][1] + gp[2][2];
                    c64 u[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        c64 v = np_[c] * div;
#pragma unroll
                        for (int i = 0; i < 3; ++i) v -= np_[i] * gp[c][i];
#pragma unroll
                        for (int kk = 0; kk < 3; ++kk) v += np_[kk] * gp[kk][c];
                        u[c] = v;
                    }
                    if (side == 1) {  // T_j u = u + t_j n (n.u), n the scatterer normal
                        const c64 nu = nb[0] * u[0] + nb[1] * u[1] + nb[2] * u[2];
                        const c64 tn = dc[d].t * nu;
#pragma unroll
                        for (int c = 0; c < 3; ++c) u[c] += nb[c] * tn;
                    }
                    const double wa = w[a];
                    const c64 sig = side == 0 ? c64{-1.0, 0.0} : dc[d].gamma;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        yacc[c] += wa * u[c];
                        yacc[3 + c] += (sig * ph[c]) * wa;
                    }
                }
            }
            if (threadIdx.x < nt) {  // transposed self block, stored in user order
                const int64_t uu = perm[a];
                const c64 *M = Mself + 36 * uu;
                const c64 *xa = x + (r * N + uu) * 6;
                c64 *ya = y + (r * N + uu) * 6;
#pragma unroll
                for (int pc = 0; pc < 6; ++pc) {
                    c64 acc = yacc[pc];
                    for (int q = 0; q < 6; ++q) cfma(acc, M[q * 6 + pc], xa[q]);
                    ya[pc] = acc;
                }
            }
        }
    }
}

// ---------------------------------------------------------------- one launch over many problems
// A persistent kernel over the work items of many independent problems (one product y_i = A_i x_i
// each): densities, P2M per (leaf, domain, right-hand side), M2M per (parent, domain, column chunk)
// level by level, M2L + L2L per (box, domain, column chunk) level by level, near field + L2P + self
// per leaf.  Blocks take items in queue order from one counter; the items are sorted by stage
// rank, and an item only waits for stages of its own problem that rank lower, so with every block
// resident (the grid is sized by the occupancy) the lowest unfinished item can always proceed.
// Each block waits for its item's inputs on per-problem completion counters with a bounded spin
// (%globaltimer); when a wait runs out it raises the error flag and every block leaves at its next
// item.  stall_problem >= 0 (fault injection for tests) withholds the completion of that problem's
// P2M items, so that its later items wait until the limit.
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t batch_clock() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ bool batch_wait(const unsigned *c, unsigned target, uint64_t wait_ns, const int *err) {
    if (ld_acquire_u32(c) >= target) return true;
    const uint64_t t0 = batch_clock();
    for (;;) {
        for (int i = 0; i < 32; ++i) {
            if (ld_acquire_u32(c) >= target) return true;
            __nanosleep(64);
        }
        if (*(const volatile int *)err) return false;  // another block gave up already
        if (batch_clock() - t0 > wait_ns) return false;
    }
}

template <typename R>
__global__ void __launch_bounds__(128) k_batch(const BatchProblem *probs, const BatchItem *items, int64_t n_items,
                                               int64_t nr, unsigned long long *next, unsigned *cnt,
                                               const unsigned *tgt, int *err, uint64_t wait_ns, int stall_problem) {
    __shared__ int64_t s_it;
    __shared__ int s_go;
    for (;;) {
        if (threadIdx.x == 0) {
            const int64_t it = (int64_t)atomicAdd(next, 1ull);
            int go = it < n_items && !*(volatile int *)err;
            if (go) {
                const BatchItem w = items[it];
                const int lmax = probs[w.prob].lmax;
                const unsigned *c = cnt + (int64_t)w.prob * BATCH_COUNTERS;
                const unsigned *t = tgt + (int64_t)w.prob * BATCH_COUNTERS;
                int k1 = -1, k2 = -1;
                if (w.kind == BK_P2M) k1 = 0;
                else if (w.kind == BK_M2M) k1 = 1 + w.level;
                else if (w.kind == BK_DOWN) { k1 = 1 + w.level; if (w.level >= 3) k2 = 12 + w.level - 1; }
                else if (w.kind == BK_NEAR) k1 = 12 + lmax;
                bool ok = (k1 < 0 || batch_wait(c + k1, t[k1], wait_ns, err)) &&
                          (k2 < 0 || batch_wait(c + k2, t[k2], wait_ns, err));
                if (!ok) {
                    atomicExch(err, 1);
                    go = 0;
                }
                __threadfence();
            }
            s_it = it;
            s_go = go;
        }
        __syncthreads();
        if (!s_go) break;
        const BatchItem w = items[s_it];
        const BatchProblem &P = probs[w.prob];
        const int lmax = P.lmax;
        switch (w.kind) {
            case BK_PREP:
                prep_body<R>(P.N, nr, P.x, P.perm, P.nrm64, P.w, P.dom, (const DomainConsts *)P.dc, (cx<R> *)P.dens,
                             w.a, w.c);
                break;
            case BK_P2M:
                p2m_body<R>(P.lev_off[lmax] + w.a, P.N, nr, P.p2, P.nbox, P.nbeg, P.nend, P.dom, P.nrm64,
                            (const cx<R> *)P.dens, (const cx<R> *)P.Bp2m, (cx<R> *)P.C, w.a, w.b, w.c);
                break;
            case BK_M2M:
                m2m_body<R, CC>(P.lev_off[w.level - 1], w.level, lmax, nr, P.p2, P.nbox, P.cbeg, P.cend, P.key,
                                (const cx<R> *)P.Tmm, (cx<R> *)P.C, w.a, w.b, w.c);
                break;
            case BK_DOWN:
                down_body<R>(P.lev_off[w.level], w.level, lmax, nr, P.p2, P.nbox, P.parent, P.key, P.ff_start,
                             P.ff_src, P.ff_off, (const cx<R> *)P.Tm2l, (const cx<R> *)P.Tll, (const cx<R> *)P.C,
                             (cx<R> *)P.D, w.a, w.b, w.c);
                break;
            default:
                near_body<R, sizeof(R) == 4>(P.lev_off[lmax] + w.a, P.N, nr, P.p2, P.nbox, P.nbeg, P.nend, P.nbr_start,
                                             P.nbr_idx, (const R *)P.pos_hi, (const R *)P.pos_lo, (const R *)P.nrm,
                                             P.dom, P.perm, (const cx<R> *)P.dens, (const DomainConsts *)P.dc,
                                             (const cx<R> *)P.Bl2p, (const cx<R> *)P.D, P.Mself, P.x, P.y, nullptr,
                                             nullptr, true, w.a);
                break;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (!(w.prob == stall_problem && w.kind == BK_P2M))
                atomicAdd(cnt + (int64_t)w.prob * BATCH_COUNTERS + batch_done_counter(w.kind, w.level, lmax), 1u);
        }
    }
}

}  // namespace

// ------------------------------------------------------------------------------------------
// replace dense coaxial tables (nz of them, p2 x p2 input-major) by their packed order blocks and
// check Z^{-m} = Z^m, on which the folded rotation form relies
static void pack_coax(fmbem *h, c64 *&Z64, c32 *&Z32, int64_t nz, cudaStream_t s) {
    const int p = h->p;
    const int64_t ncoax = p * (2 * p * p + 1) / 3;
    auto pack = [&](auto *&Zd) {
        using T = std::remove_reference_t<decltype(*Zd)>;
        T *Zp = (T *)dev_alloc(h, sizeof(T) * nz * ncoax);
        k_pack_rot_z<<<(unsigned)((nz * ncoax + 255) / 256), 256, 0, s>>>(p, nz, Zd, Zp);
        CKL("k_pack_rot_z");
        CK(cudaStreamSynchronize(s));
        dev_free(h, Zd);
        Zd = Zp;
    };
    pack(Z64);
    pack(Z32);
    unsigned long long *dev = (unsigned long long *)dev_alloc(h, sizeof(unsigned long long) * (nz + 1));
    CK(cudaMemsetAsync(dev, 0, sizeof(unsigned long long) * (nz + 1), s));
    const unsigned nb = (unsigned)((nz * ncoax + 255) / 256);
    k_z_scale<<<nb, 256, 0, s>>>(p, nz, Z64, dev + 1);
    CKL("k_z_scale");
    k_check_z_mirror<<<nb, 256, 0, s>>>(p, nz, Z64, dev + 1, dev);
    CKL("k_check_z_mirror");
    unsigned long long hd = 0;
    CK(cudaMemcpyAsync(&hd, dev, sizeof(hd), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    dev_free(h, dev);
    double zmax;
    std::memcpy(&zmax, &hd, sizeof(double));
    // the projected tables carry quadrature rounding of about 1e-12..1e-6 of their largest entry
    // (the upper end for p >= 11 in a strongly damped domain); a convention error would show as an
    // O(1) asymmetry
    if (!(zmax < 1e-4)) {
        char buf[64];
        std::snprintf(buf, sizeof(buf), "%.3e", zmax);
        throw fmbem_error{FMBEM_ERR_CUDA, std::string("coaxial translations: Z^-m differs from Z^m (relative ") + buf + ")"};
    }
}

// the coaxial S|R tables R_Z (per domain, level and offset length)
void pack_rot_tables(fmbem *h, cudaStream_t s) {
    pack_coax(h, h->R_Z64, h->R_Z32, (int64_t)(h->J + 1) * (h->lmax + 1) * h->n_tlen, s);
}

// the coaxial S|S and R|R tables (per domain and level) and the octant-grouped child lists of the
// rotation-form M2M and L2L
void pack_rot_tables_mm(fmbem *h, cudaStream_t s) {
    const int64_t nzl = (int64_t)(h->J + 1) * (h->lmax + 1);
    pack_coax(h, h->R_Zmm64, h->R_Zmm32, nzl, s);
    pack_coax(h, h->R_Zll64, h->R_Zll32, nzl, s);
    build_rot_mm_lists(h, s);
}

// the packed rotation factors from the projected ones: forward T(Rz^T) (azimuthal), T(Ry^T)
// (polar), back T(Ry) (polar), T(Rz) (azimuthal), each [316][p2][p2] input-major; fails loudly if
// the polar factors are not real or not mirror symmetric, or the azimuthal ones not diagonal
void pack_rot_factors(fmbem *h, const c64 *Tzf, const c64 *Tyf, const c64 *Tyb, const c64 *Tzb, cudaStream_t s) {
    const int p = h->p, p2 = h->p2;
    const int64_t nrot = rot_off(p);  // folded polar entries per offset and direction
    h->R_D64 = (double *)dev_alloc(h, sizeof(double) * 316 * 2 * nrot);
    h->R_D32 = (float *)dev_alloc(h, sizeof(float) * 316 * 2 * nrot);
    h->R_P64 = (c64 *)dev_alloc(h, sizeof(c64) * 316 * 2 * p2);
    h->R_P32 = (c32 *)dev_alloc(h, sizeof(c32) * 316 * 2 * p2);
    unsigned long long *dev = (unsigned long long *)dev_alloc(h, 4 * sizeof(unsigned long long));
    CK(cudaMemsetAsync(dev, 0, 4 * sizeof(unsigned long long), s));
    k_pack_rot_d<<<(unsigned)((316 * 2 * nrot + 255) / 256), 256, 0, s>>>(p, Tyf, Tyb, h->R_D64, h->R_D32, dev);
    CKL("k_pack_rot_d");
    const int64_t np = (int64_t)316 * 2 * p2 * p2;
    k_pack_rot_p<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(p, Tzf, Tzb, h->R_P64, h->R_P32, dev);
    CKL("k_pack_rot_p");
    unsigned long long hd[4];
    CK(cudaMemcpyAsync(hd, dev, sizeof(hd), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    dev_free(h, dev);
    double im_max, off_max, asym_max, conj_max;
    std::memcpy(&im_max, &hd[0], sizeof(double));
    std::memcpy(&off_max, &hd[1], sizeof(double));
    std::memcpy(&asym_max, &hd[2], sizeof(double));
    std::memcpy(&conj_max, &hd[3], sizeof(double));
    if (!(im_max < 1e-9) || !(off_max < 1e-9) || !(asym_max < 1e-9) || !(conj_max < 1e-9))
        throw fmbem_error{FMBEM_ERR_CUDA, "rotation factors: polar part not real (" + std::to_string(im_max) +
                                              "), not mirror symmetric (" + std::to_string(asym_max) +
                                              "), azimuthal part not diagonal (" + std::to_string(off_max) +
                                              ") or its orders -m not conjugate to m (" + std::to_string(conj_max) + ")"};
}

// near-field pair-scalar cache (see k_near_cache): per leaf nt x nsrc pairs per side, double
// precision (the single-precision kernels evaluate g and c faster than they could read them), built
// when option near_cache asks for it (or, automatically, when it fits in a quarter of the free
// device memory)
void build_near_cache(fmbem *h, cudaStream_t s) {
    if (h->opt.near_cache == 0) return;
    const int64_t nl = h->n_leaves, nrng = h->nbox + h->n_range_boxes;
    std::vector<int32_t> nb(nrng), ne(nrng), ns(nl + 1);
    CK(cudaMemcpyAsync(nb.data(), h->box_nbeg, sizeof(int32_t) * nrng, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ne.data(), h->box_nend, sizeof(int32_t) * nrng, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ns.data(), h->nbr_start, sizeof(int32_t) * (nl + 1), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<int32_t> idx(std::max(ns[nl], 1));
    CK(cudaMemcpyAsync(idx.data(), h->nbr_idx, sizeof(int32_t) * ns[nl], cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<int64_t> base(nl + 1, 0);
    for (int64_t lf = 0; lf < nl; ++lf) {
        int64_t nsrc = 0;
        for (int q = ns[lf]; q < ns[lf + 1]; ++q) nsrc += ne[idx[q]] - nb[idx[q]];
        const int32_t g = h->h_leaf_box[lf];
        base[lf + 1] = base[lf] + nsrc * (ne[g] - nb[g]);
    }
    const size_t pairs = (size_t)base[nl];
    const size_t bytes = 2 * pairs * sizeof(V4<double>);
    if (h->opt.near_cache == -1) {
        size_t freeb = 0, totb = 0;
        CK(cudaMemGetInfo(&freeb, &totb));
        if (bytes > freeb / 4) return;
    }
    h->near_base = (int64_t *)dev_alloc(h, sizeof(int64_t) * (nl + 1));
    CK(cudaMemcpyAsync(h->near_base, base.data(), sizeof(int64_t) * (nl + 1), cudaMemcpyHostToDevice, s));
    h->near_cache64 = dev_alloc(h, 2 * pairs * sizeof(V4<double>));
    const DomainConsts *dc = (const DomainConsts *)h->dcons;
    k_near_cache<double><<<(unsigned)nl, 256, 0, s>>>(h->leaf_box, h->box_nbeg, h->box_nend, h->nbr_start, h->nbr_idx,
                                                       h->pos, h->dom, dc, h->near_base, (V4<double> *)h->near_cache64);
    CKL("k_near_cache");
    CK(cudaStreamSynchronize(s));
}

// warp work items of the near field (see k_near_w): per leaf of nt targets, the layout of W
// warps x (tg targets x nsl slices) with the least lane time W / nsl, tg = ceil(nt / W) <= 32,
// nsl the largest power of two with tg * nsl <= 32, up to 8 warps per leaf
void near_work_items(fmbem *h, cudaStream_t s) {
    if (h->near_items) return;
    const int64_t nl = h->n_leaves, nrng = h->nbox + h->n_range_boxes;
    std::vector<int32_t> nbA(nrng), neA(nrng), ns(nl + 1), ni;
    CK(cudaMemcpyAsync(nbA.data(), h->box_nbeg, sizeof(int32_t) * nrng, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(neA.data(), h->box_nend, sizeof(int32_t) * nrng, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ns.data(), h->nbr_start, sizeof(int32_t) * (nl + 1), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ni.resize(std::max(ns[nl], 1));
    CK(cudaMemcpyAsync(ni.data(), h->nbr_idx, sizeof(int32_t) * ns[nl], cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // the leaves' own node ranges, in leaf order
    std::vector<int32_t> nb(nl), ne(nl);
    for (int64_t lf = 0; lf < nl; ++lf) { nb[lf] = nbA[h->h_leaf_box[lf]]; ne[lf] = neA[h->h_leaf_box[lf]]; }
    std::vector<int4> items;
    std::vector<int64_t> cost;  // a lane's pair count: the leaf's Neighbor sources over the slices
    for (int64_t leaf = 0; leaf < nl; ++leaf) {
        const int nt = ne[leaf] - nb[leaf];
        if (nt <= 0) continue;
        int bestW = (nt + 31) / 32, bestP = 1;
        double best = bestW;
        for (int W = 1; W <= std::max(8, (nt + 31) / 32); ++W) {
            const int tg = (nt + W - 1) / W;
            if (tg > 32) continue;
            int p = 1;
            while (2 * p * tg <= 32) p *= 2;
            if ((double)W / p < best - 1e-12) { best = (double)W / p; bestW = W; bestP = p; }
        }
        const int tg = (nt + bestW - 1) / bestW;
        int64_t nsrc = 0;
        for (int q = ns[leaf]; q < ns[leaf + 1]; ++q) nsrc += neA[ni[q]] - nbA[ni[q]];
        for (int t = 0; t < nt; t += tg) {
            items.push_back(int4{(int)leaf, t, std::min(tg, nt - t), bestP});
            cost.push_back((nsrc + bestP - 1) / bestP);
        }
    }
    // longest items first: blocks start in index order, so the last ones to start are short
    std::vector<int> order(items.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
    std::stable_sort(order.begin(), order.end(), [&](int u, int v) { return cost[u] > cost[v]; });
    std::vector<int4> sorted(items.size());
    for (size_t k = 0; k < order.size(); ++k) sorted[k] = items[order[k]];
    items.swap(sorted);
    h->n_near_items = (int)items.size();
    h->near_items = (int4 *)dev_alloc(h, sizeof(int4) * items.size());
    h->near_next = (int *)dev_alloc(h, sizeof(int));
    CK(cudaMemcpyAsync(h->near_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, s));
    // target groups of at most NR_TT targets per leaf for k_near_r, near-equal sizes: in leaf
    // (Morton) order, so that concurrent units share sources in L2, and again with the most pair
    // work first, for the last slab
    std::vector<int4> groups;
    std::vector<int64_t> gcost;
    for (int64_t leaf = 0; leaf < nl; ++leaf) {
        const int nt = ne[leaf] - nb[leaf];
        if (nt <= 0) continue;
        int64_t nsrc = 0;
        for (int q = ns[leaf]; q < ns[leaf + 1]; ++q) nsrc += neA[ni[q]] - nbA[ni[q]];
        const int ng = (nt + NR_TT - 1) / NR_TT;
        for (int k = 0, t0 = 0; k < ng; ++k) {
            const int cnt = nt / ng + (k < nt % ng ? 1 : 0);
            groups.push_back(int4{(int)leaf, t0, cnt, 0});
            gcost.push_back(nsrc * cnt);
            t0 += cnt;
        }
    }
    std::vector<int> gorder(groups.size());
    for (size_t k = 0; k < gorder.size(); ++k) gorder[k] = (int)k;
    std::stable_sort(gorder.begin(), gorder.end(), [&](int u, int v) { return gcost[u] > gcost[v]; });
    std::vector<int4> gsorted(groups.size());
    for (size_t k = 0; k < gorder.size(); ++k) gsorted[k] = groups[gorder[k]];
    h->n_near_groups = (int)groups.size();
    h->near_groups = (int4 *)dev_alloc(h, sizeof(int4) * 2 * std::max<size_t>(groups.size(), 1));
    CK(cudaMemcpyAsync(h->near_groups, groups.data(), sizeof(int4) * groups.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->near_groups + groups.size(), gsorted.data(), sizeof(int4) * gsorted.size(),
                       cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
}

// The child boxes of every level l >= 3 for the rotation-form M2M and L2L: entries grouped by
// octant (the child-parent direction), in chunks of at most M2L_CHUNK that share it; each chunk
// carries the far-field offset code of the same direction for M2M (child to parent, offset
// (4o-2) per axis) and for L2L (parent to child, the opposite one).
void build_rot_mm_lists(fmbem *h, cudaStream_t s) {
    const int lmax = h->lmax;
    std::vector<uint64_t> key(h->nbox);
    std::vector<int32_t> par(h->nbox);
    CK(cudaMemcpyAsync(key.data(), h->box_key, sizeof(uint64_t) * h->nbox, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(par.data(), h->box_parent, sizeof(int32_t) * h->nbox, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<int32_t> child, parent, entry(h->nbox, -1), cbeg, ccnt;
    std::vector<int16_t> cmm, cll;
    h->h_rmm_first.assign(lmax + 2, 0);
    h->h_rmm_chunk_first.assign(lmax + 2, 0);
    for (int l = 0; l <= lmax + 1; ++l) {
        h->h_rmm_first[l] = (int64_t)child.size();
        h->h_rmm_chunk_first[l] = (int64_t)cbeg.size();
        if (l < 3 || l > lmax) continue;
        const LevelInfo &Lv = h->lev[l];
        for (int o = 0; o < 8; ++o) {
            const int ox = (o >> 2) & 1, oy = (o >> 1) & 1, oz = o & 1;  // Morton bit order x, y, z
            const int16_t mm = (int16_t)m2l_offset_code(4 * ox - 2, 4 * oy - 2, 4 * oz - 2);
            const int16_t ll = (int16_t)m2l_offset_code(2 - 4 * ox, 2 - 4 * oy, 2 - 4 * oz);
            int in_chunk = M2L_CHUNK;
            for (int64_t g = Lv.off; g < Lv.off + Lv.n; ++g) {
                if ((int)(key[g] & 7) != o) continue;
                if (in_chunk == M2L_CHUNK) {
                    cbeg.push_back((int32_t)child.size());
                    ccnt.push_back(0);
                    cmm.push_back(mm);
                    cll.push_back(ll);
                    in_chunk = 0;
                }
                entry[g] = (int32_t)child.size();
                child.push_back((int32_t)g);
                parent.push_back(par[g]);
                ++ccnt.back();
                ++in_chunk;
            }
        }
    }
    h->n_rmm = (int64_t)child.size();
    if (h->n_rmm == 0) return;
    std::vector<int32_t> iota(child.size());
    for (size_t k = 0; k < iota.size(); ++k) iota[k] = (int32_t)k;
    std::vector<int8_t> zero(316, 0);
    auto up = [&](auto *&dst, const auto &v) {
        using T = std::remove_reference_t<decltype(*dst)>;
        dst = (T *)dev_alloc(h, sizeof(T) * std::max<size_t>(v.size(), 1));
        CK(cudaMemcpyAsync(dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s));
    };
    up(h->rmm_iota, iota);
    up(h->rmm_child, child);
    up(h->rmm_par, parent);
    up(h->rmm_entry, entry);
    up(h->rmm_chunk_beg, cbeg);
    up(h->rmm_chunk_cnt, ccnt);
    up(h->rmm_chunk_mm, cmm);
    up(h->rmm_chunk_ll, cll);
    up(h->rot_zero, zero);
    CK(cudaStreamSynchronize(s));
}

// Columns per window of the FP64 rotation-form M2L when a call has more than 24 columns: one
// column per lane of k_m2l_rot_cols (32), unless the per-target reduction k_l2l_reduce would then
// need more than 1024 threads (p > 8), where it stays at 24.
static int rot_many_cols(const fmbem *h) {
    const int rows_pad = ((h->p2 + 31) / 32) * 32;
    return rows_pad * ((ROTC_N + L2L_CPT - 1) / L2L_CPT) <= 1024 ? ROTC_N : 24;
}
// FP64 calls with more than 24 columns run the rotation form in column windows when its tables
// were built (the dense target-major kernel otherwise)
static bool rot_many_path(const fmbem *h, int64_t nr, bool fp64) {
    return fp64 && 3 * nr > 24 && h->m2l_rotation && h->R_D64 != nullptr;
}
// bytes of the per-pair M2L result buffer for ncol columns: the largest level's pair results,
// then (rotation form) its child entries
// per level, every multipole domain's pair results and rotation-form child entries (the passes
// run the domains of a level in one launch each)
static size_t ybuf_need(const fmbem *h, int64_t ncol, size_t elem) {
    int64_t mp = 1;
    for (int l = 2; l <= h->lmax; ++l) {
        const int64_t ne = h->h_rmm_first.empty() ? 0 : h->h_rmm_first[l + 1] - h->h_rmm_first[l];
        mp = std::max(mp, h->h_pair_first[l + 1] - h->h_pair_first[l] + ne);
    }
    return elem * (size_t)(h->Jf + 1) * (size_t)mp * (size_t)ncol * h->p2;
}

// per-pair results of the one-launch offset-stationary M2L (BF16x3, few columns): every level's
// pairs for every multipole domain, then one level's rotation-form L2L entries
static size_t ofs_ybuf_need(const fmbem *h, int64_t nr) {
    int64_t ne = 1;
    for (int l = 2; l <= h->lmax; ++l)
        if (!h->h_rmm_first.empty()) ne = std::max(ne, h->h_rmm_first[l + 1] - h->h_rmm_first[l]);
    return sizeof(float) * (size_t)(h->Jf + 1) * (ofs_y_dom(h, nr) + (size_t)ne * 3 * nr * 2 * h->p2);
}

static void ensure_scratch(fmbem *h, int64_t nr, int precision, bool pair_results = true) {
    const size_t cb = sizeof(c64);
    if (h->scratch_rhs < nr) {
        if (h->dens) { dev_free(h, h->dens); dev_free(h, h->Cexp); dev_free(h, h->Dexp); }
        h->dens = dev_alloc(h, cb * 2 * nr * h->N * 6);
        h->Cexp = dev_alloc(h, cb * (size_t)(h->J + 1) * h->nbox * 3 * nr * h->p2);
        h->Dexp = dev_alloc(h, cb * (size_t)(h->J + 1) * h->nbox * 3 * nr * h->p2);
        h->scratch_rhs = nr;
    }
    // per-pair M2L results of one level, one domain and up to 24 columns (chunked path only;
    // one column window of the FP64 rotation form for more columns); sized by the columns of
    // this call, so that a few-column call after a many-column one still takes the chunked path
    const bool many = rot_many_path(h, nr, precision == FMBEM_FP64);
    if (pair_results && (3 * nr <= 24 || many)) {
        size_t need = ybuf_need(h, many ? rot_many_cols(h) : 3 * nr, cb);
        if (precision == FMBEM_BF16X3 && h->Aofs != nullptr && 3 * nr <= 24) need = std::max(need, ofs_ybuf_need(h, nr));
        if (h->ybuf == nullptr || h->ybuf_bytes < need) {
            if (h->ybuf) dev_free(h, h->ybuf);
            h->ybuf = nullptr;
            h->ybuf = dev_alloc(h, need);
            h->ybuf_bytes = need;
        }
    }
}

// Launch shape of the rotation-form kernel k_m2l_rot for ncol columns: in double precision
// groups of exactly p2 threads (a warp may straddle two column groups), so that no lane idles on
// a padded row in the FP64-bound stages; in single precision, where the kernel is latency-bound,
// rows padded to whole warps (more threads).  ok is false when the rotation tables were not built
// or the shape does not fit.
constexpr int ROT_MAXC = 12;
struct RotLaunch {
    bool ok = false, cols = false;  // cols: the column-parallel kernel (double precision)
    int rows = 0, cg = 1, pc = 0;
    size_t bytes = 0;
};
template <typename R>
static RotLaunch rot_launch(fmbem *h, int ncol, size_t budget) {
    RotLaunch rl;
    if (!h->m2l_rotation || h->R_D64 == nullptr || ncol > (sizeof(R) == 8 ? ROTC_N : 24)) return rl;
    const int p = h->p, p2 = h->p2, nrot = rot_off(p), ncoax = p * (2 * p * p + 1) / 3;
    if (sizeof(R) == 8) {  // FP64-bound: one column per lane, loops of equal length in a warp
        const size_t b = sizeof(R) * 2 * (size_t)nrot + sizeof(cx<R>) * ((size_t)(2 * p2 + ncoax) + 2 * (size_t)p2 * ROTC_S) +
                         sizeof(short2) * (size_t)(p * (p + 1) / 2);
        if (b <= budget) {
            rl.ok = rl.cols = true;
            rl.rows = 32;
            rl.cg = ROTC_WARPS;
            rl.pc = std::min(M2L_CHUNK, ROTC_N / ncol);
            rl.bytes = b;
            CK(cudaFuncSetAttribute(k_m2l_rot_cols<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b));
            return rl;
        }
    }
    if (ncol > 24) return rl;  // wider windows only in the column-parallel kernel
    cudaFuncAttributes fa{};
    CK(cudaFuncGetAttributes(&fa, k_m2l_rot<R, ROT_MAXC>));
    auto bytes = [&](int c) {
        return sizeof(R) * 2 * (size_t)nrot + sizeof(cx<R>) * ((size_t)(2 * p2 + ncoax) + 2 * (size_t)c * ROT_MAXC * p2) +
               sizeof(short2) * (size_t)(p * (p + 1) / 2);
    };
    rl.rows = sizeof(R) == 4 ? ((p2 + 31) / 32) * 32 : p2;
    rl.cg = std::max(1, std::min(4, fa.maxThreadsPerBlock / rl.rows));
    while (rl.cg > 1 && bytes(rl.cg) > budget) --rl.cg;
    rl.pc = std::min(M2L_CHUNK, rl.cg * ROT_MAXC / ncol);
    rl.bytes = bytes(rl.cg);
    rl.ok = rl.pc >= 1 && rl.bytes <= budget && rl.rows * rl.cg <= fa.maxThreadsPerBlock;
    if (rl.ok) CK(cudaFuncSetAttribute(k_m2l_rot<R, ROT_MAXC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rl.bytes));
    return rl;
}
// one launch of the rotation-form kernel chosen by rot_launch over nch chunks, for domains
// 0 .. ndom - 1 (grid rows), domain d's results at Y + d * y_dstride
template <typename R>
static void launch_rot(const RotLaunch &rl, int64_t nch, cudaStream_t s, int64_t c0, int l, int lmax, int ndom,
                       int64_t nr, int p, int64_t nbox, int col0, int nc, const int32_t *cbeg, const int32_t *ccnt,
                       const int16_t *coff, const int32_t *pair_e, const int32_t *src, const int8_t *tidx, int n_tlen,
                       const R *RD, const cx<R> *RP, const cx<R> *RZ, const cx<R> *C, cx<R> *Y, int64_t e_first,
                       int64_t y_dstride) {
    if (nch <= 0) return;
    const dim3 grid((unsigned)nch, (unsigned)ndom);
    if (rl.cols)
        k_m2l_rot_cols<R><<<grid, 32 * ROTC_WARPS, rl.bytes, s>>>(c0, l, lmax, 0, nr, p, nbox, col0, nc, rl.pc, 1, cbeg,
                                                                  ccnt, coff, pair_e, src, tidx, n_tlen, RD, RP, RZ, C,
                                                                  Y, e_first, y_dstride);
    else
        k_m2l_rot<R, ROT_MAXC><<<grid, rl.rows * rl.cg, rl.bytes, s>>>(c0, l, lmax, 0, nr, p, nbox, col0, nc, rl.pc,
                                                                       rl.cg, cbeg, ccnt, coff, pair_e, src, tidx,
                                                                       n_tlen, RD, RP, RZ, C, Y, e_first, y_dstride);
}

// M2M (Eq. 2.20) from level l_max up to level 2, on the multipole expansions in h->Cexp
template <typename R>
static void upward_m2m(fmbem *h, int64_t nr, cudaStream_t s) {
    const int p2 = h->p2, lmax = h->lmax, J = h->Jf;
    const bool f32 = sizeof(R) == 4;
    cx<R> *C = (cx<R> *)h->Cexp;
    const cx<R> *Tmm = f32 ? (const cx<R> *)h->T_mm32 : (const cx<R> *)h->T_mm64;
    const int rows_pad = ((p2 + 31) / 32) * 32;
    // rotation form (p >= 9, few columns): the children of each level, by octant, translated to
    // their parents' centres (folded rotation, coaxial S|S, rotation back), then summed per parent
    const int ncol = (int)std::min<int64_t>(3 * nr, 24);
    if (3 * nr <= 24 && h->rmm_chunk_beg != nullptr && h->ybuf != nullptr) {
        const RotLaunch rl = rot_launch<R>(h, ncol, 200 * 1024);
        if (rl.ok) {
            const R *RD = f32 ? (const R *)h->R_D32 : (const R *)h->R_D64;
            const cx<R> *RP = f32 ? (const cx<R> *)h->R_P32 : (const cx<R> *)h->R_P64;
            const cx<R> *RZmm = f32 ? (const cx<R> *)h->R_Zmm32 : (const cx<R> *)h->R_Zmm64;
            cx<R> *Y = (cx<R> *)h->ybuf;
            for (int l = lmax; l >= 3; --l) {
                const LevelInfo &P = h->lev[l - 1];
                const int64_t c0 = h->h_rmm_chunk_first[l], nch = h->h_rmm_chunk_first[l + 1] - c0;
                const int64_t e_first = h->h_rmm_first[l];
                // all domains in one launch each: domain d's child entries at Y + d * ystr
                const int64_t ystr = (h->h_rmm_first[l + 1] - e_first) * ncol * p2;
                launch_rot<R>(rl, nch, s, c0, l, lmax, J + 1, nr, h->p, h->nbox, 0, ncol, h->rmm_chunk_beg,
                              h->rmm_chunk_cnt, h->rmm_chunk_mm, h->rmm_iota, h->rmm_child, h->rot_zero, 1, RD, RP,
                              RZmm, C, Y, e_first, ystr);
                CKL("k_m2l_rot (M2M)");
                k_mm_reduce<R><<<dim3((unsigned)P.n, (unsigned)(J + 1)), 128, 0, s>>>(
                    P.off, 0, nr, p2, h->nbox, 0, ncol, h->box_cbeg, h->box_cend, h->rmm_entry, e_first, Y, C, ystr);
                CKL("k_mm_reduce");
            }
            return;
        }
    }
    for (int l = lmax; l >= 3; --l) {
        const LevelInfo &P = h->lev[l - 1];
        if (nr == 1)
            k_m2m<R, 3><<<dim3((unsigned)P.n, J + 1, 1), rows_pad, sizeof(cx<R>) * 3 * p2, s>>>(
                P.off, l, lmax, nr, p2, h->nbox, h->box_cbeg, h->box_cend, h->box_key, Tmm, C);
        else
            k_m2m<R, CC><<<dim3((unsigned)P.n, J + 1, (unsigned)((3 * nr + CC - 1) / CC)), rows_pad,
                           sizeof(cx<R>) * CC * p2, s>>>(P.off, l, lmax, nr, p2, h->nbox, h->box_cbeg, h->box_cend,
                                                         h->box_key, Tmm, C);
        CKL("k_m2m");
    }
}

// downward pass (Eq. 2.21): M2L over the FF lists and L2L, h->Cexp -> h->Dexp, all levels
template <typename R>
// tensor_mode: 0 CUDA cores, 1 TF32 tensor cores, 2 BF16x3 tensor cores (many columns)
// c_split: the BF16x3 tensor-core path finds C already split into bf16 hi/lo parts (run_m2m_tc)
static void downward_pass(fmbem *h, int64_t nr, cudaStream_t s, int tensor_mode, bool c_split = false) {
    const int p2 = h->p2, lmax = h->lmax, J = h->Jf;
    const bool f32 = sizeof(R) == 4;
    cx<R> *C = (cx<R> *)h->Cexp, *D = (cx<R> *)h->Dexp;
    const cx<R> *Tm2l = f32 ? (const cx<R> *)h->T_m2l32 : (const cx<R> *)h->T_m2l64;
    const cx<R> *Tll = f32 ? (const cx<R> *)h->T_ll32 : (const cx<R> *)h->T_ll64;
    const int rows_pad = ((p2 + 31) / 32) * 32;
    const int ncc = (int)((3 * nr + CC - 1) / CC);  // column chunks of the fallback kernel
    const size_t sm = sizeof(cx<R>) * CC * p2;
    // downward pass: offset-chunked M2L with a per-target reduction for few columns, the
    // target-major kernel (translation matrices reused across many columns) otherwise
    constexpr int MAXC = 24;
    // FP64 with more than MAXC columns and rotation tables: the rotation form in column windows
    const bool rot_many = rot_many_path(h, nr, !f32);
    const int ncol = rot_many ? rot_many_cols(h) : (int)std::min<int64_t>(3 * nr, MAXC);
    const size_t tbytes = sizeof(cx<R>) * p2 * p2;
    const size_t budget = 200 * 1024;
    auto xs_bytes = [&](int c) { return sizeof(cx<R>) * c * MAXC * p2; };
    // threads per block are capped by the kernel's register use
    cudaFuncAttributes fa_t{}, fa_g{};
    CK(cudaFuncGetAttributes(&fa_t, k_m2l_chunks<R, MAXC, true>));
    CK(cudaFuncGetAttributes(&fa_g, k_m2l_chunks<R, MAXC, false>));
    const int max_thr = std::min(fa_t.maxThreadsPerBlock, fa_g.maxThreadsPerBlock);
    int cg = std::max(1, std::min(4, max_thr / rows_pad));
    // stage T in shared memory when it fits beside the full column groups; otherwise read T from
    // L2 and keep the column groups (occupancy matters more than T reuse from shared memory)
    const bool tsm = tbytes + xs_bytes(cg) <= budget;
    while (cg > 1 && (tsm ? tbytes : 0) + xs_bytes(cg) > budget) --cg;
    const size_t smc = (tsm ? tbytes : 0) + xs_bytes(cg);
    const int pc = std::min(M2L_CHUNK, cg * MAXC / ncol);
    // rotation form of the chunked S|R (when its tables were built)
    const int pp = h->p;
    const RotLaunch rl = rot_launch<R>(h, ncol, budget);
    const bool chunked =
        (3 * nr <= MAXC ? pc >= 1 && smc <= budget
                        : rot_many && rl.ok && h->ybuf_bytes >= ybuf_need(h, ncol, sizeof(cx<R>))) &&
        h->ybuf != nullptr && rows_pad <= max_thr;
    const bool use_rot = chunked && rl.ok;
    if (tensor_mode && f32 && h->Atc != nullptr && 3 * nr >= 48) {
        run_m2l_tc(h, (float *)C, (float *)D, nr, s, tensor_mode == 2, c_split);
    } else if (chunked) {
        if (tsm) CK(cudaFuncSetAttribute(k_m2l_chunks<R, MAXC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc));
        else CK(cudaFuncSetAttribute(k_m2l_chunks<R, MAXC, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc));
        const R *RD = f32 ? (const R *)h->R_D32 : (const R *)h->R_D64;
        const cx<R> *RP = f32 ? (const cx<R> *)h->R_P32 : (const cx<R> *)h->R_P64;
        const cx<R> *RZ = f32 ? (const cx<R> *)h->R_Z32 : (const cx<R> *)h->R_Z64;
        const cx<R> *RZll = f32 ? (const cx<R> *)h->R_Zll32 : (const cx<R> *)h->R_Zll64;
        const bool use_rot_mm = use_rot && h->rmm_chunk_beg != nullptr;
        cx<R> *Y = (cx<R> *)h->ybuf;
        // BF16x3 with few columns: the S|R products of each offset chunk on the tensor cores
        // (all levels and domains in one launch first: the S|R products read only C; the pair
        // results of every level then wait in Y[d][CSR position], and the rotation form's L2L
        // results go after them)
        const bool ofs = tensor_mode == 2 && f32 && h->Aofs != nullptr && h->chunk_pairs != nullptr && 3 * nr <= MAXC &&
                         h->ybuf_bytes >= ofs_ybuf_need(h, nr);
        // With a second stream the coarse levels' M2L (levels 2..l_max-1) runs first; then, while
        // the leaf level's M2L occupies all but OFS_AUX_SMS SMs, the second stream runs those
        // levels' L2L + reductions and the leaf level's L2L, which are latency-bound chains of
        // small launches; the leaf level's reduction joins both.
        constexpr int OFS_AUX_SMS = 8;
        const bool overlap = ofs && h->aux_stream != nullptr && lmax >= 3;
        if (ofs) {
            split_expansions_bf16(h, (float *)C, nr, s);
            if (overlap) {
                run_m2l_ofs(h, (const float *)C, (float *)Y, nr, s, 2, lmax - 1, 0);
                CK(cudaEventRecord(h->ev_fork, s));
                CK(cudaStreamWaitEvent(h->aux_stream, h->ev_fork, 0));
                run_m2l_ofs(h, (const float *)C, (float *)Y, nr, s, lmax, lmax, OFS_AUX_SMS);
            } else {
                run_m2l_ofs(h, (const float *)C, (float *)Y, nr, s, 2, lmax, 0);
            }
        }
        const int64_t y_dom = ofs ? ofs_y_dom(h, nr) / 2 : 0;  // in complex values
        // per level and column window, all domains in one launch each (grid rows): domain d's pair
        // results at Y + d * ystr, its rotation-form L2L entries after every domain's pair results
        for (int l = 2; l <= lmax; ++l) {
            const LevelInfo &Lv = h->lev[l];
            const int64_t c0 = h->h_chunk_first[l], nch = h->h_chunk_first[l + 1] - c0;
            const int64_t nchild = h->h_rmm_first.empty() ? 0 : h->h_rmm_first[l + 1] - h->h_rmm_first[l];
            for (int col0 = 0; col0 < 3 * nr; col0 += ncol) {
                const int nc = (int)std::min<int64_t>(ncol, 3 * nr - col0);
                const int64_t e_first = ofs ? 0 : h->h_pair_first[l];
                const int64_t ystr = ofs ? y_dom : (h->h_pair_first[l + 1] - e_first) * nc * p2;
                const dim3 grid((unsigned)nch, (unsigned)(J + 1));
                if (nch > 0 && !ofs) {  // (the offset-stationary products ran above)
                    if (use_rot)
                        launch_rot<R>(rl, nch, s, c0, l, lmax, J + 1, nr, pp, h->nbox, col0, nc, h->chunk_beg,
                                      h->chunk_cnt, h->chunk_off, h->pair_e, h->ff_src, h->rot_tidx, h->n_tlen, RD, RP,
                                      RZ, C, Y, e_first, ystr);
                    else if (tsm)
                        k_m2l_chunks<R, MAXC, true><<<grid, rows_pad * cg, smc, s>>>(
                            c0, l, lmax, 0, nr, p2, h->nbox, col0, nc, pc, cg, h->chunk_beg, h->chunk_cnt, h->chunk_off,
                            h->pair_e, h->ff_src, Tm2l, C, Y, e_first, ystr);
                    else
                        k_m2l_chunks<R, MAXC, false><<<grid, rows_pad * cg, smc, s>>>(
                            c0, l, lmax, 0, nr, p2, h->nbox, col0, nc, pc, cg, h->chunk_beg, h->chunk_cnt, h->chunk_off,
                            h->pair_e, h->ff_src, Tm2l, C, Y, e_first, ystr);
                    CKL("k_m2l_chunks");
                }
                // L2L in rotation form: the children of level l, by octant, from their parents'
                // local expansions
                cx<R> *Yll = nullptr;
                int64_t ll_first = 0;
                const int64_t yll_str = nchild * nc * p2;
                cudaStream_t sl = overlap ? h->aux_stream : s;  // this level's L2L
                if (use_rot_mm && l >= 3) {
                    const int64_t lc0 = h->h_rmm_chunk_first[l], lnch = h->h_rmm_chunk_first[l + 1] - lc0;
                    ll_first = h->h_rmm_first[l];
                    Yll = Y + (J + 1) * ystr;
                    launch_rot<R>(rl, lnch, sl, lc0, l, lmax, J + 1, nr, pp, h->nbox, col0, nc, h->rmm_chunk_beg,
                                  h->rmm_chunk_cnt, h->rmm_chunk_ll, h->rmm_iota, h->rmm_par, h->rot_zero, 1, RD, RP,
                                  RZll, D, Yll, ll_first, yll_str);
                    CKL("k_m2l_rot (L2L)");
                }
                if (overlap && l == lmax) {  // join: the leaf level's reduction on the caller's stream
                    CK(cudaEventRecord(h->ev_join, h->aux_stream));
                    CK(cudaStreamWaitEvent(s, h->ev_join, 0));
                }
                cudaStream_t sr = overlap && l < lmax ? h->aux_stream : s;  // this level's reduction
                const int ct = (nc + L2L_CPT - 1) / L2L_CPT;
                k_l2l_reduce<R><<<dim3((unsigned)Lv.n, (unsigned)(J + 1)), rows_pad * ct, sizeof(cx<R>) * nc * p2, sr>>>(
                    Lv.off, l, lmax, 0, nr, p2, h->nbox, col0, nc, ct, h->box_parent, h->box_key, h->ff_start, Tll, Y,
                    e_first, D, Yll, h->rmm_entry, ll_first, ystr, yll_str);
                CKL("k_l2l_reduce");
            }
        }
    } else if (sizeof(cx<R>) * (size_t)(p2 * p2 + p2 * MT_COLS) <= budget &&
               ((p2 + 3) / 4) * (MT_COLS / 4) <= [] {
                   cudaFuncAttributes fa{};
                   CK(cudaFuncGetAttributes(&fa, k_m2l_multi<R>));
                   return fa.maxThreadsPerBlock;
               }()) {
        const size_t smm = sizeof(cx<R>) * (size_t)(p2 * p2 + p2 * MT_COLS);
        CK(cudaFuncSetAttribute(k_m2l_multi<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smm));
        const int nt = ((p2 + 3) / 4) * (MT_COLS / 4);
        const unsigned ntile = (unsigned)((3 * nr + MT_COLS - 1) / MT_COLS);
        for (int l = 2; l <= lmax; ++l) {
            const LevelInfo &Lv = h->lev[l];
            k_m2l_multi<R><<<dim3((unsigned)Lv.n, J + 1, ntile), nt, smm, s>>>(Lv.off, l, lmax, nr, p2, h->nbox,
                                                                             h->box_parent, h->box_key, h->ff_start,
                                                                             h->ff_src, h->ff_off, Tm2l, Tll, C, D);
            CKL("k_m2l_multi");
        }
    } else {
        for (int l = 2; l <= lmax; ++l) {
            const LevelInfo &Lv = h->lev[l];
            k_down<R><<<dim3((unsigned)Lv.n, J + 1, ncc), rows_pad, sm, s>>>(Lv.off, l, lmax, nr, p2, h->nbox,
                                                                             h->box_parent, h->box_key, h->ff_start,
                                                                             h->ff_src, h->ff_off, Tm2l, Tll, C, D);
            CKL("k_down");
        }
    }
}

// Impedance boundary (Section 2.3): the scatterer rows of every node are the local relation of
// Eq. (2.24), y_s = M_s x with M_s the scatterer rows of the node's 6x6 block (Psi - zeta (Phi -
// n (n.Phi))); they replace what the near-field kernel wrote there.  Thread per (rhs, node), user
// order [nr][N][6].
__global__ void k_local_rows(int64_t N, int64_t nr, const c64 *Mself, const c64 *x, c64 *y) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N * nr) return;
    const c64 *M = Mself + 36 * (i % N) + 18;
    const c64 *xi = x + 6 * i;
    for (int q = 0; q < 3; ++q) {
        c64 acc = {0, 0};
        for (int c = 0; c < 6; ++c) cfma(acc, M[6 * q + c], xi[c]);
        y[6 * i + 3 + q] = acc;
    }
}

// zero the local expansions of the domains Jf+1..J (not computed with an impedance boundary) in
// the layout of an nr-column call, so that the near-field kernels read zeros there
static void clear_unused_domains(fmbem *h, int64_t nr, size_t real_bytes, cudaStream_t s) {
    const size_t per = 2 * real_bytes * (size_t)h->nbox * 3 * nr * h->p2;
    if (h->J > h->Jf) CK(cudaMemsetAsync((char *)h->Dexp + per * (h->Jf + 1), 0, per * (h->J - h->Jf), s));
}

template <typename R>
static void matvec_impl(fmbem *h, const c64 *x, c64 *y, int64_t nr, cudaStream_t s, const DomainConsts *dc,
                        int tensor_mode = 0) {
    const int64_t N = h->N;
    const int p2 = h->p2, J = h->Jf;  // multipole passes over domains 0..Jf
    const bool f32 = sizeof(R) == 4;
    cx<R> *dens = (cx<R> *)h->dens, *C = (cx<R> *)h->Cexp, *D = (cx<R> *)h->Dexp;
    const cx<R> *Bp2m = f32 ? (const cx<R> *)h->B_p2m32 : (const cx<R> *)h->B_p2m64;
    const cx<R> *Bl2p = f32 ? (const cx<R> *)h->B_l2p32 : (const cx<R> *)h->B_l2p64;
    const bool timing = h->profile && h->ev[0] != nullptr;
    if (timing) CK(cudaEventRecord(h->ev[0], s));

    // single precision with 32 or more right-hand sides: a node-major copy of the background
    // densities and the normal jumps for k_near_r in the half of the density buffer that double
    // precision would use (64 bytes per node and RHS, within its 96)
    const int64_t nrT = f32 ? (nr / 32) * 32 : 0;
    cx<R> *densT = nrT > 0 ? dens + 2 * nr * N * 6 : nullptr;
    // and with fewer than 4, the normal jump s of the densities (k_near_ws) in the same place
    cx<R> *sj = f32 && nr < 4 ? dens + 2 * nr * N * 6 : nullptr;
    if (h->ibc) clear_unused_domains(h, nr, sizeof(R), s);
    // BF16x3 with many columns: P2M and M2M on the tensor cores as well (their products then leave
    // C split for M2L); otherwise on the CUDA cores
    const bool tc_up = f32 && tensor_mode == 2 && h->Mmbf != nullptr && 3 * nr >= 48;
    const bool tc_p2m = tc_up && p2m_tc_supported(h, nr);
    // whole blocks of 32 right-hand sides with P2M on the tensor cores: every consumer reads the
    // node-major densities, which are then the only ones formed
    const bool node_major_only = tc_p2m && nrT == nr;
    if (node_major_only) {
        k_prep_node_major<<<dim3((unsigned)((N + 7) / 8), (unsigned)(nr / 32)), 256, 0, s>>>(
            N, nr, x, h->perm, h->nrm, h->w, h->dom, dc, (float4 *)densT);
        CKL("k_prep_node_major");
    } else {
        k_prep<R><<<dim3(nblk(N, 128), (unsigned)nr), 128, 0, s>>>(N, nr, x, h->perm, h->nrm, h->w, h->dom, dc, dens,
                                                                    sj);
        CKL("k_prep");
        if (densT != nullptr) {
            k_dens_node_major<<<dim3((unsigned)((N + 15) / 16), (unsigned)(nrT / 32)), 256, 0, s>>>(
                N, nr, (const float4 *)dens, h->src_rec, (float4 *)densT);
            CKL("k_dens_node_major");
        }
    }
    const int tbc = std::min(256, ((p2 + 31) / 32) * 32);
    constexpr int P2M_RB = sizeof(R) == 4 ? 8 : 4;
    if (tc_p2m) {
        run_p2m_tc(h, (const float *)dens, node_major_only ? (const float4 *)densT : nullptr, (const float *)Bp2m,
                   (float *)C, nr, s);
    } else if (nr >= 16) {
        constexpr int MT = p2m_mt<R>(), PT = p2m_pt<R>();
        const int nthr = ((p2 + 2 * PT - 1) / (2 * PT)) * (MT / 4);
        const size_t smp = sizeof(cx<R>) * 4 * P2M_KC * (p2 + MT);
        CK(cudaFuncSetAttribute(k_p2m_gemm<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smp));
        k_p2m_gemm<R><<<dim3((unsigned)h->n_leaves, J + 1, (unsigned)((3 * nr + MT - 1) / MT)), nthr, smp, s>>>(
            h->leaf_box, N, nr, p2, h->nbox, h->box_nbeg, h->box_nend, h->dom, h->nrm, dens, Bp2m, C);
    } else if (nr >= 4)
        k_p2m_rb<R, P2M_RB><<<dim3((unsigned)h->n_leaves, J + 1, (unsigned)((nr + P2M_RB - 1) / P2M_RB)), tbc, 0, s>>>(
            h->leaf_box, N, nr, p2, h->nbox, h->box_nbeg, h->box_nend, h->dom, h->nrm, dens, Bp2m, C);
    else  // one thread per coefficient
        k_p2m<R><<<dim3((unsigned)h->n_leaves, J + 1, (unsigned)nr), ((p2 + 31) / 32) * 32, 0, s>>>(
            h->leaf_box, N, nr, p2, h->nbox, h->box_nbeg, h->box_nend, h->dom, h->nrm, dens, Bp2m, C);
    CKL("k_p2m");
    if (timing) CK(cudaEventRecord(h->ev[1], s));
    if (tc_up) run_m2m_tc(h, (float *)C, nr, s, tc_p2m);
    else upward_m2m<R>(h, nr, s);
    if (timing) CK(cudaEventRecord(h->ev[2], s));
    downward_pass<R>(h, nr, s, tensor_mode, tc_up);
    if (timing) CK(cudaEventRecord(h->ev[3], s));
    const R *ph = f32 ? (const R *)h->pos_hi : (const R *)h->pos;
    const R *pl = f32 ? (const R *)h->pos_lo : nullptr;
    const R *nn = f32 ? (const R *)h->nrm_f : (const R *)h->nrm;
    // near field: in single precision the warp-independent kernel with blocks of RB right-hand
    // sides (the pair scalars are shared by the block); for fewer than 4 right-hand sides, and in
    // double precision, the block-cooperative kernels (more threads per leaf, FP64 pipe busier)
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    // the scatterer side's near field is not needed with the impedance boundary (k_local_rows)
    const int nsides = h->ibc ? 1 : 2;
    // k_near_w over the right-hand sides rhs_base .. nr - 1 in blocks of rb
    auto launch_w = [&](auto kern, int rb, size_t tile_bytes, int64_t rhs_base) {
        if (h->near_items == nullptr) throw fmbem_error{FMBEM_ERR_CUDA, "near-field work items were not built"};
        const size_t smw = 2 * tile_bytes * NW_WARPS;  // two tiles per warp
        const int64_t units = (int64_t)h->n_near_items * nsides * ((nr - rhs_base + rb - 1) / rb);
        if (units >= INT32_MAX) throw fmbem_error{FMBEM_ERR_INVALID_ARGUMENT, "too many near-field work units"};
        CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw));
        int per_sm = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * NW_WARPS, smw));
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((units + NW_WARPS - 1) / NW_WARPS,
                                                                    (int64_t)std::max(per_sm, 1) * nsm));
        CK(cudaMemsetAsync(h->near_next, 0, sizeof(int), s));
        kern<<<(unsigned)grid, 32 * NW_WARPS, smw, s>>>(
            h->leaf_box, h->near_items, h->n_near_items, (int)units, h->near_next, N, nr, rhs_base, nsides, h->box_nbeg,
            h->box_nend, h->nbr_start, h->nbr_idx, h->src_rec, (const cx<float> *)dens, dc, h->perm, p2, h->nbox,
            (const cx<float> *)Bl2p, (const cx<float> *)D, h->Mself, x, y);
        CKL("k_near_w");
    };
    // k_near_r over the right-hand sides 32 slab0 .. 32 (slab0 + nslab) - 1
    auto launch_r = [&](int64_t slab0, int64_t nslab) {
        const int64_t units = (int64_t)h->n_near_groups * nslab;
        if (units >= INT32_MAX) throw fmbem_error{FMBEM_ERR_INVALID_ARGUMENT, "too many near-field work units"};
        const size_t smr = sizeof(RhsTile) * NR_WARPS;
        CK(cudaFuncSetAttribute(k_near_r, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr));
        int per_sm = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_near_r, 32 * NR_WARPS, smr));
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((units + NR_WARPS - 1) / NR_WARPS,
                                                                    (int64_t)std::max(per_sm, 1) * nsm));
        CK(cudaMemsetAsync(h->near_next, 0, sizeof(int), s));
        k_near_r<<<(unsigned)grid, 32 * NR_WARPS, smr, s>>>(
            h->leaf_box, h->near_groups, h->n_near_groups, (int)units, h->near_next, N, nr, nsides == 2, h->box_nbeg,
            h->box_nend, h->nbr_start, h->nbr_idx, h->src_rec, (const float4 *)densT, dc, h->perm, p2, h->nbox,
            (const cx<float> *)Bl2p, (const cx<float> *)D, h->Mself, x, y, (int)slab0, (int)(slab0 + nslab - 1));
        CKL("k_near_r");
    };
    if constexpr (sizeof(R) == 4) {
        if (nr >= 4) {  // whole blocks of 32 right-hand sides one per lane, the rest by k_near_w
            const int64_t nblk = nr / 32, rest = nr - 32 * nblk;
            // a host-buffer product (fmbem_matvec_host) whose rows are final after the near field:
            // one launch per slab, each slab's rows copied back beside the next slab's launch
            auto &io = h->io_rows;
            const bool per_slab = io.y_host != nullptr && nblk > 1 && rest == 0 && !h->ibc && h->ns_pairs <= 0 &&
                                  nblk <= (int64_t)(sizeof(io.ev) / sizeof(io.ev[0]));
            if (per_slab) {
                for (int64_t b = 0; b < nblk; ++b) {
                    launch_r(b, 1);
                    CK(cudaEventRecord(io.ev[b], s));
                    CK(cudaStreamWaitEvent(io.down, io.ev[b], 0));
                    const int64_t off = b * 32 * N * 6;
                    CK(cudaMemcpyAsync(io.y_host + off, y + off, sizeof(c64) * 32 * N * 6, cudaMemcpyDeviceToHost,
                                       io.down));
                }
                io.copied = true;
            } else if (nblk > 0) {
                launch_r(0, nblk);
            }
            if (rest >= 8) launch_w(k_near_w<8>, 8, sizeof(WarpTile<8>), 32 * nblk);
            else if (rest > 0) launch_w(k_near_w<4>, 4, sizeof(WarpTile<4>), 32 * nblk);
        } else {  // few right-hand sides: both sides of a pair in one pass, one unit per item and RHS
            if (h->near_items == nullptr) throw fmbem_error{FMBEM_ERR_CUDA, "near-field work items were not built"};
            const int64_t units = (int64_t)h->n_near_items * nr;
            int per_sm = 0;
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_near_ws, 32 * NS_WARPS, 0));
            const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((units + NS_WARPS - 1) / NS_WARPS,
                                                                        (int64_t)std::max(per_sm, 1) * nsm));
            CK(cudaMemsetAsync(h->near_next, 0, sizeof(int), s));
            k_near_ws<<<(unsigned)grid, 32 * NS_WARPS, 0, s>>>(
                h->leaf_box, h->near_items, h->n_near_items, (int)units, h->near_next, N, nr, h->box_nbeg, h->box_nend,
                h->nbr_start, h->nbr_idx, h->src_rec, (const cx<float> *)dens, (const cx<float> *)sj, dc, h->perm, p2,
                h->nbox, (const cx<float> *)Bl2p, (const cx<float> *)D, h->Mself, x, y, !h->ibc);
            CKL("k_near_ws");
        }
    } else if (nr >= 4) {
        constexpr int RBLK = 2;
        const size_t smn = sizeof(NearSmemRB<R, RBLK>);
        CK(cudaFuncSetAttribute(k_near_rb<R, false, RBLK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smn));
        k_near_rb<R, false, RBLK><<<dim3((unsigned)h->n_leaves, (unsigned)((nr + RBLK - 1) / RBLK)), 128, smn, s>>>(
            h->leaf_box, N, nr, p2, h->nbox, h->box_nbeg, h->box_nend, h->nbr_start, h->nbr_idx, ph, pl, nn, h->dom, h->perm,
            dens, dc, Bl2p, D, h->Mself, x, y, !h->ibc);
    } else {
        k_near<R, false><<<(unsigned)h->n_leaves, 128, 0, s>>>(h->leaf_box, N, nr, p2, h->nbox, h->box_nbeg, h->box_nend, h->nbr_start,
                                                       h->nbr_idx, ph, pl, nn, h->dom, h->perm, dens, dc, Bl2p, D,
                                                       h->Mself, x, y, h->near_base, (const V4<R> *)h->near_cache64,
                                                       !h->ibc);
    }
    CKL("k_near");
    if (h->ibc) {  // impedance boundary: the scatterer rows are the local relation of Eq. (2.24)
        k_local_rows<<<nblk(N * nr, 128), 128, 0, s>>>(N, nr, h->Mself, x, y);
        CKL("k_local_rows");
    }
    apply_near_singular(h, x, y, nr, s, false);  // near-singular pair corrections (option), FP64
    if (timing) CK(cudaEventRecord(h->ev[4], s));
}

// y = A^T x (see k_near_adj): monopole P2M, M2M, the downward pass, near field and assembly
template <typename R>
static void adjoint_impl(fmbem *h, const c64 *x, c64 *y, int64_t nr, cudaStream_t s, const DomainConsts *dc,
                         int tensor_mode = 0) {
    const int64_t N = h->N;
    const int p2 = h->p2, J = h->Jf;  // multipole passes over domains 0..Jf
    const bool f32 = sizeof(R) == 4;
    cx<R> *dens = (cx<R> *)h->dens, *C = (cx<R> *)h->Cexp, *D = (cx<R> *)h->Dexp;
    const cx<R> *Bp2m = f32 ? (const cx<R> *)h->B_p2m32 : (const cx<R> *)h->B_p2m64;
    const cx<R> *Bl2p = f32 ? (const cx<R> *)h->B_l2p32 : (const cx<R> *)h->B_l2p64;
    const cx<R> *Bl2pg = f32 ? (const cx<R> *)h->B_l2pg32 : (const cx<R> *)h->B_l2pg64;
    // impedance boundary: the scatterer rows of A are local (Eq. 2.24), so the transposed product
    // takes them from the transposed self blocks alone; the scatterer sources are zero, and so are
    // the unused local expansions of the scatterer domains that the near-field kernel reads
    if (h->ibc) clear_unused_domains(h, nr, sizeof(R), s);
    k_prep_adj<R><<<dim3(nblk(N, 128), (unsigned)nr), 128, 0, s>>>(N, nr, x, h->perm, h->ibc ? 1 : 2, dens);
    CKL("k_prep_adj");
    const int tbc = std::min(256, ((p2 + 31) / 32) * 32);
    k_p2m_adj<R><<<dim3((unsigned)h->n_leaves, J + 1, (unsigned)nr), tbc, 0, s>>>(h->leaf_box, N, nr, p2, h->nbox, h->box_nbeg,
                                                                           h->box_nend, h->dom, dens, Bp2m, C);
    CKL("k_p2m_adj");
    upward_m2m<R>(h, nr, s);
    downward_pass<R>(h, nr, s, tensor_mode);
    const R *ph = f32 ? (const R *)h->pos_hi : (const R *)h->pos;
    const R *pl = f32 ? (const R *)h->pos_lo : nullptr;
    const V4<R> *cache = f32 ? nullptr : (const V4<R> *)h->near_cache64;
    if constexpr (sizeof(R) == 4)
        k_near_adj<R, true><<<dim3((unsigned)h->n_leaves, (unsigned)std::min<int64_t>(nr, 65535)), 128, 0, s>>>(h->leaf_box, N, nr, p2, h->nbox, h->box_nbeg, h->box_nend,
                                                          h->nbr_start, h->nbr_idx, ph, pl, h->nrm, h->w, h->dom,
                                                          h->perm, dens, dc, Bl2p, Bl2pg, D, h->Mself, x, y,
                                                          h->near_base, cache);
    else
        k_near_adj<R, false><<<dim3((unsigned)h->n_leaves, (unsigned)std::min<int64_t>(nr, 65535)), 128, 0, s>>>(h->leaf_box, N, nr, p2, h->nbox, h->box_nbeg, h->box_nend,
                                                           h->nbr_start, h->nbr_idx, ph, pl, h->nrm, h->w, h->dom,
                                                           h->perm, dens, dc, Bl2p, Bl2pg, D, h->Mself, x, y,
                                                           h->near_base, cache);
    CKL("k_near_adj");
    apply_near_singular(h, x, y, nr, s, true);  // transposed near-singular pair corrections (option)
}

// the bounded mbarrier waits of the tensor-core kernel report time-outs in h->tc_err
static void check_tc_err(fmbem *h, cudaStream_t s) {
    if (!h->tc_err) return;
    int e = 0;
    CK(cudaMemcpyAsync(&e, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (e) {
        CK(cudaMemsetAsync(h->tc_err, 0, sizeof(int), s));
        throw fmbem_error{FMBEM_ERR_DEVICE_TIMEOUT, "tensor-core M2L: an mbarrier wait timed out"};
    }
}

// a handle that keeps only single-precision tables runs FP32 passes only
static void check_fp32_only(const fmbem *h, int precision) {
    if (h->opt.fp32_only && precision != FMBEM_FP32)
        throw fmbem_error{FMBEM_ERR_INVALID_ARGUMENT,
                          "this handle keeps single-precision tables only (fp32_only): FP32 passes only"};
}

void run_adjoint_matvec(fmbem *h, const c64 *x, c64 *y, int64_t nr, int precision, cudaStream_t s) {
    check_fp32_only(h, precision);
    ensure_scratch(h, nr, precision);
    const DomainConsts *dc = (const DomainConsts *)h->dcons;
    if (precision == FMBEM_TF32 || precision == FMBEM_BF16X3) {
        adjoint_impl<float>(h, x, y, nr, s, dc, precision == FMBEM_TF32 ? 1 : 2);
        check_tc_err(h, s);
    } else if (precision == FMBEM_FP32) {
        adjoint_impl<float>(h, x, y, nr, s, dc);
    } else {
        adjoint_impl<double>(h, x, y, nr, s, dc);
    }
}

void run_matvec(fmbem *h, const c64 *x, c64 *y, int64_t nr, int precision, cudaStream_t s) {
    check_fp32_only(h, precision);
    ensure_scratch(h, nr, precision);
    static_assert(sizeof(DomainConsts) == 3 * sizeof(c64), "layout");
    DomainConsts *dc = (DomainConsts *)h->dcons;
    if (precision == FMBEM_TF32 || precision == FMBEM_BF16X3) {
        matvec_impl<float>(h, x, y, nr, s, dc, precision == FMBEM_TF32 ? 1 : 2);
        check_tc_err(h, s);
    } else if (precision == FMBEM_FP32) {
        matvec_impl<float>(h, x, y, nr, s, dc);
    } else {
        matvec_impl<double>(h, x, y, nr, s, dc);
    }
    h->have_times = h->profile && h->ev[0] != nullptr;
}

// ------------------------------------------------------------------------------------------
// Allocation-free matvec.  Some callers cannot allocate device memory at the time they need a
// product: code running inside a CUDA stream capture (where cudaMalloc is not allowed), code
// under a framework allocator that owns all device memory, or callbacks that must not block
// on an implicit device synchronisation.  fmbem_matvec_noalloc runs the same kernels as
// fmbem_matvec, but takes its scratch (source densities, multipole and local coefficients,
// per-pair M2L results) from the file-scope device array below instead of the handle's
// grow-on-demand buffers, so it never calls cudaMalloc or cudaFree.
//
// The array is STATIC_SCRATCH_BYTES (32 MiB) on every GPU that loads the library and stays
// resident until the process exits.  All calls share it and it keeps the last call's contents:
// every element a call reads is written earlier in the same call, so nothing needs clearing,
// but two calls that overlap on the GPU (different streams, no ordering) race on it.
constexpr size_t STATIC_SCRATCH_BYTES = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

#include <mutex>

// Device address of g_static_scratch on the current device.  In host code the symbol is only a
// host-side stand-in, so the address is looked up once per device with cudaGetSymbolAddress (the
// first allocation-free call on a device does this; it should come before any stream capture).
static void *static_scratch_address() {
    static std::mutex mu;
    static void *addr[128] = {nullptr};
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) throw fmbem_error{FMBEM_ERR_CUDA, "device index out of range"};
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        CK(cudaGetSymbolAddress(&p, g_static_scratch));
        addr[dev] = p;
    }
    return addr[dev];
}

template <typename R>
static void matvec_static_scratch(fmbem *h, const c64 *x, c64 *y, int64_t nr, cudaStream_t s) {
    const size_t S = sizeof(cx<R>);
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    // single precision with 32 or more right-hand sides also keeps the node-major density copy,
    // with fewer than 4 the densities' normal jump, both after the densities
    const size_t extra = sizeof(R) == 4 ? (nr >= 32 ? 2 * nr * h->N * 6 : nr < 4 ? nr * h->N : 0) : 0;
    const size_t b_dens = up(S * (2 * nr * h->N * 6 + extra));
    const size_t b_exp = up(S * (size_t)(h->J + 1) * h->nbox * 3 * nr * h->p2);
    size_t b_y = 0;
    if (3 * nr <= 24) {
        b_y = up(ybuf_need(h, 3 * nr, S));  // as ensure_scratch: every domain's pair results and child entries
    }
    const size_t need = b_dens + 2 * b_exp + b_y;
    if (need > STATIC_SCRATCH_BYTES)
        throw fmbem_error{FMBEM_ERR_INVALID_ARGUMENT,
                          "fmbem_matvec_noalloc needs " + std::to_string(need) + " bytes of scratch for this problem and n_rhs; "
                          "its static array holds " + std::to_string(STATIC_SCRATCH_BYTES) + " bytes (use fmbem_matvec)"};
    unsigned char *base = (unsigned char *)static_scratch_address();
    // run the regular passes on pointers into the static array; the handle's own scratch
    // pointers are restored afterwards, so fmbem_matvec is unaffected
    void *sv_dens = h->dens, *sv_C = h->Cexp, *sv_D = h->Dexp, *sv_y = h->ybuf;
    h->dens = base;
    h->Cexp = base + b_dens;
    h->Dexp = base + b_dens + b_exp;
    h->ybuf = b_y ? base + b_dens + 2 * b_exp : nullptr;
    try {
        matvec_impl<R>(h, x, y, nr, s, (const DomainConsts *)h->dcons);
    } catch (...) {
        h->dens = sv_dens; h->Cexp = sv_C; h->Dexp = sv_D; h->ybuf = sv_y;
        throw;
    }
    h->dens = sv_dens; h->Cexp = sv_C; h->Dexp = sv_D; h->ybuf = sv_y;
}

void run_matvec_noalloc(fmbem *h, const c64 *x, c64 *y, int64_t nr, int precision, cudaStream_t s) {
    check_fp32_only(h, precision);
    if (precision == FMBEM_FP32) matvec_static_scratch<float>(h, x, y, nr, s);
    else matvec_static_scratch<double>(h, x, y, nr, s);
    h->have_times = h->profile && h->ev[0] != nullptr;
}

// one launch of the persistent many-problem kernel (see k_batch); the grid is the number of
// blocks that can be resident at once, so that no item waits for an item that is not running
void run_batch_kernel(int precision, const BatchProblem *probs, const BatchItem *items, int64_t n_items,
                      unsigned long long *next, unsigned *cnt, const unsigned *tgt, int *err, uint64_t wait_ns,
                      int stall_problem, int p2max, int64_t nr, cudaStream_t s) {
    int dev = 0, nsm = 0, per_sm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    // single precision only: the double-precision bodies together need more than 48 KiB of static
    // shared memory
    if (precision != FMBEM_FP32) throw fmbem_error{FMBEM_ERR_INVALID_ARGUMENT, "the batch runs in FP32"};
    const size_t smem = sizeof(c32) * CC * p2max;
    CK(cudaFuncSetAttribute(k_batch<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<float>, 128, smem));
    if (per_sm < 1) throw fmbem_error{FMBEM_ERR_CUDA, "the batch kernel cannot be resident"};
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(n_items, (int64_t)per_sm * nsm));
    k_batch<float><<<(unsigned)grid, 128, smem, s>>>(probs, items, n_items, nr, next, cnt, tgt, err, wait_ns,
                                                     stall_problem);
    CKL("k_batch");
}

// scratch of a handle for an n_rhs product in the given precision (batch.cu): densities and
// expansions only, the batch's dense translation items keep no per-pair results
void batch_ensure_scratch(fmbem *h, int64_t nr, int precision) { ensure_scratch(h, nr, precision, false); }
