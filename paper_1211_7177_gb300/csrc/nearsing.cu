// nearsing.cu -- near-singular correction of the pair terms of Eq. (2.12) (option
// near_singular_radius; the paper's operator, radius 0, applies the one-point rule of Eq. (2.8)
// to every pair beta != alpha).
//
// With a radius rho > 0, a source node beta within R = |s_beta - s_alpha| < rho sqrt(w_beta) of
// the target alpha contributes the integral of the pair kernel over its patch, with its density
// (and normal) held constant, instead of w_beta times the kernel at s_beta.  The patch is the
// surface its weight stands for: the triangle itself for centroid nodes; for vertex nodes the
// barycentric dual cell, two flat pieces (A, mid(AB), G) and (A, G, mid(AC)) in every incident
// triangle (A the vertex, G the centroid).  Each piece is cut into 4^L congruent triangles (the
// 2^L x 2^L barycentric grid) and integrated with the centroid rule.
//
// Because the bracket of Eq. (2.12), n'(a.v) - (n'.a) v - a (n'.v), is linear in a = grad'g, the
// correction of a pair and domain is fully described by
//   dS = int_patch g dA' - w g(s_beta),   dA = int_patch grad'g dA' - w grad'g(s_beta)
// (complex scalar and complex 3-vector), computed once at create in FP64 for the background and,
// when both nodes belong to the same scatterer, for the scatterer domain.  Each product then adds
//   background rows:  -[n0 (dA0.v) - (n0.dA0) v - dA0 (n0.v)] + dS0 (-Psi_beta),   v = Phi_beta, n0 = -n_beta
//   scatterer rows:   -[n (dAj.v) - (n.dAj) v - dAj (n.v)] + gamma_j dSj Psi_beta,  v = T_j Phi_beta, n = n_beta
// (and the transposed blocks for A^T), in FP64 whatever the precision of the multipole passes.
// The target's search runs over its leaf and the Neighbor leaves, so rho sqrt(w) must not exceed
// the leaf width; create rejects larger radii.
#include <algorithm>
#include <string>
#include <vector>

#include "fmbem_internal.cuh"

namespace {

constexpr double NS_PI = 3.14159265358979323846;

// pieces of vertex v's dual cell: for its k-th incident triangle t (corner a at v, B and C next in
// the triangle's counter-clockwise order) pieces 2(vt_start[v] + k) and 2(vt_start[v] + k) + 1
__global__ void k_ns_pieces_vertex(int64_t nv, const double *V, const int32_t *F, const int32_t *vt_start,
                                   const int32_t *vt_tri, double *pc) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= nv) return;
    for (int32_t k = vt_start[v]; k < vt_start[v + 1]; ++k) {
        const int32_t t = vt_tri[k];
        int a = 0;
        while (a < 2 && F[3 * t + a] != (int32_t)v) ++a;
        const double *A = V + 3 * F[3 * t + a], *B = V + 3 * F[3 * t + (a + 1) % 3], *C = V + 3 * F[3 * t + (a + 2) % 3];
        double *p1 = pc + 18 * (int64_t)k, *p2 = p1 + 9;
        for (int q = 0; q < 3; ++q) {
            const double mab = 0.5 * (A[q] + B[q]), mac = 0.5 * (A[q] + C[q]), g = (A[q] + B[q] + C[q]) / 3.0;
            p1[q] = A[q];
            p1[3 + q] = mab;
            p1[6 + q] = g;
            p2[q] = A[q];
            p2[3 + q] = g;
            p2[6 + q] = mac;
        }
    }
}

// piece of centroid node t: the triangle itself
__global__ void k_ns_pieces_centroid(int64_t nt, const double *V, const int32_t *F, double *pc) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    for (int a = 0; a < 3; ++a)
        for (int q = 0; q < 3; ++q) pc[9 * t + 3 * a + q] = V[3 * F[3 * t + a] + q];
}

// does source j (sorted) qualify for target i (sorted)?
__device__ __forceinline__ bool ns_pair(const double *pos, const double *w, int64_t i, int64_t j, double rho) {
    if (i == j) return false;
    const double dx = pos[3 * j] - pos[3 * i], dy = pos[3 * j + 1] - pos[3 * i + 1], dz = pos[3 * j + 2] - pos[3 * i + 2];
    return dx * dx + dy * dy + dz * dz < rho * rho * w[j];
}

// pass 1 (start == NULL): count the qualifying sources of every target; pass 2: write them at
// start[target] (user indices of target and source), in the order of the Neighbor list.
// node_leaf holds global box ids; nbr_start is indexed by the leaf's position (box_leafpos)
__global__ void k_ns_pairs(int64_t N, double rho, const int32_t *box_leafpos, const int32_t *node_leaf, const int32_t *nbr_start,
                           const int32_t *nbr_idx, const int32_t *box_nbeg, const int32_t *box_nend, const double *pos,
                           const double *w, const int32_t *perm, int32_t *cnt, const int64_t *start, int32_t *tgt,
                           int32_t *src) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t leaf = box_leafpos[node_leaf[i]];
    const int32_t ui = perm[i];
    int64_t k = start ? start[ui] : 0;
    int32_t c = 0;
    for (int32_t e = nbr_start[leaf]; e < nbr_start[leaf + 1]; ++e) {
        const int32_t bx = nbr_idx[e];
        for (int32_t j = box_nbeg[bx]; j < box_nend[bx]; ++j)
            if (ns_pair(pos, w, i, j, rho)) {
                if (start) {
                    tgt[k] = ui;
                    src[k] = perm[j];
                    ++k;
                }
                ++c;
            }
    }
    if (!start) cnt[ui] = c;
}

// int g dA' and int grad'g dA' minus the one-point terms, per pair and domain side, one warp per
// pair: the lanes share the (piece, grid cell) items; each cell (a, b) of the 2^L x 2^L grid
// holds the "up" triangle when a + b <= n - 1 and the "down" triangle when a + b <= n - 2, with
// centroids at barycentric (a + 1/3, b + 1/3)/n and (a + 2/3, b + 2/3)/n.
// coef [pair][2][4] complex: (dS, dA_x, dA_y, dA_z) for the background (side 0) and the target's
// scatterer (side 1, zero when the source belongs to another scatterer).
__global__ void k_ns_coef(int64_t npair, int L, const int32_t *tgt, const int32_t *src, const int32_t *pc_start,
                          const double *pc, const double *upos, const double *uw, const int32_t *udom, const c64 *dc,
                          c64 *coef) {
    const int64_t pr = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (pr >= npair) return;
    const int32_t a = tgt[pr], b = src[pr];
    const bool same = udom[a] == udom[b];
    const c64 k[2] = {dc[0], dc[3 * udom[a]]};
    const int nsides = same ? 2 : 1;
    const int n = 1 << L, cells = n * n;
    const double *sa = upos + 3 * a;
    double acc[2][8];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[s][q] = 0;
    const int32_t p0 = pc_start[b], p1 = pc_start[b + 1];
    const int64_t items = (int64_t)(p1 - p0) * cells;
    for (int64_t it = lane; it < items; it += 32) {
        const int32_t piece = p0 + (int32_t)(it / cells);
        const int cell = (int)(it % cells), ca = cell / n, cb = cell % n;
        if (ca + cb > n - 1) continue;
        const double *P = pc + 9 * (int64_t)piece;
        const double e1[3] = {P[3] - P[0], P[4] - P[1], P[5] - P[2]}, e2[3] = {P[6] - P[0], P[7] - P[1], P[8] - P[2]};
        const double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        const double sub = 0.5 * sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]) / (double)cells;
        for (int down = 0; down < 2; ++down) {
            if (down && ca + cb > n - 2) break;
            const double u = (ca + (down ? 2.0 : 1.0) / 3.0) / n, v = (cb + (down ? 2.0 : 1.0) / 3.0) / n;
            double r[3];
            for (int q = 0; q < 3; ++q) r[q] = P[q] + u * e1[q] + v * e2[q] - sa[q];
            const double R = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            for (int s = 0; s < nsides; ++s) {
                // g = exp(i k R) / (4 pi R), grad'g = g (i k - 1/R) r / R
                const c64 e = cexpd(c64{-k[s].im * R, k[s].re * R});
                const c64 g = (1.0 / (4 * NS_PI * R)) * e;
                const c64 cc = (1.0 / R) * (g * c64{-1.0 / R, 0.0} + g * c64{0.0, 1.0} * k[s]);
                acc[s][0] += sub * g.re;
                acc[s][1] += sub * g.im;
                for (int q = 0; q < 3; ++q) {
                    acc[s][2 + 2 * q] += sub * r[q] * cc.re;
                    acc[s][3 + 2 * q] += sub * r[q] * cc.im;
                }
            }
        }
    }
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[s][q] += __shfl_xor_sync(0xffffffffu, acc[s][q], o);
    if (lane != 0) return;
    // minus the one-point term w g(s_beta), w grad'g(s_beta)
    double r[3];
    for (int q = 0; q < 3; ++q) r[q] = upos[3 * b + q] - sa[q];
    const double R = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    const double wb = uw[b];
    c64 *out = coef + 8 * pr;
    for (int s = 0; s < 2; ++s) {
        if (s >= nsides) {
            for (int q = 0; q < 4; ++q) out[4 * s + q] = c64{0, 0};
            continue;
        }
        const c64 e = cexpd(c64{-k[s].im * R, k[s].re * R});
        const c64 g = (1.0 / (4 * NS_PI * R)) * e;
        const c64 cc = (1.0 / R) * (g * c64{-1.0 / R, 0.0} + g * c64{0.0, 1.0} * k[s]);
        out[4 * s] = c64{acc[s][0] - wb * g.re, acc[s][1] - wb * g.im};
        for (int q = 0; q < 3; ++q)
            out[4 * s + 1 + q] = c64{acc[s][2 + 2 * q] - wb * r[q] * cc.re, acc[s][3 + 2 * q] - wb * r[q] * cc.im};
    }
}

// bracket of Eq. (2.12): n (a.v) - (n.a) v - a (n.v), and its transpose a (n.u) - (n.a) u - n (a.u)
__device__ __forceinline__ void ns_bracket(const double *n, const c64 *a, const c64 *v, c64 *out) {
    c64 av = {0, 0}, na = {0, 0}, nv = {0, 0};
    for (int q = 0; q < 3; ++q) {
        cfma(av, a[q], v[q]);
        na += n[q] * a[q];
        nv += n[q] * v[q];
    }
    for (int q = 0; q < 3; ++q) out[q] = n[q] * av - na * v[q] - a[q] * nv;
}
__device__ __forceinline__ void ns_bracket_t(const double *n, const c64 *a, const c64 *u, c64 *out) {
    c64 nu = {0, 0}, na = {0, 0}, au = {0, 0};
    for (int q = 0; q < 3; ++q) {
        nu += n[q] * u[q];
        na += n[q] * a[q];
        cfma(au, a[q], u[q]);
    }
    for (int q = 0; q < 3; ++q) out[q] = a[q] * nu - na * u[q] - n[q] * au;
}
// T_j v = v + t_j n (n.v), Eq. (2.13)
__device__ __forceinline__ void ns_T(const double *n, c64 t, const c64 *v, c64 *out) {
    c64 nv = {0, 0};
    for (int q = 0; q < 3; ++q) nv += n[q] * v[q];
    const c64 tn = t * nv;
    for (int q = 0; q < 3; ++q) out[q] = v[q] + n[q] * tn;
}

// y += correction x, thread per (target, right-hand side), user order [nr][N][6]
__global__ void k_ns_apply(int64_t N, int64_t nr, const int64_t *start, const int32_t *src, const c64 *coef,
                           const double *unrm, const int32_t *udom, const c64 *dc, const c64 *x, c64 *y) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= N * nr) return;
    const int64_t a = idx % N, r = idx / N;
    const int64_t p0 = start[a], p1 = start[a + 1];
    if (p0 == p1) return;
    const int j = udom[a];
    const c64 tj = dc[3 * j + 1], gj = dc[3 * j + 2];
    c64 acc[6] = {};
    for (int64_t p = p0; p < p1; ++p) {
        const int32_t b = src[p];
        const c64 *cf = coef + 8 * p;
        const c64 *xb = x + (r * N + b) * 6;
        const double nb[3] = {unrm[3 * b], unrm[3 * b + 1], unrm[3 * b + 2]};
        const double n0[3] = {-nb[0], -nb[1], -nb[2]};
        c64 v[3] = {xb[0], xb[1], xb[2]}, B[3];
        ns_bracket(n0, cf + 1, v, B);
        for (int q = 0; q < 3; ++q) acc[q] += cf[0] * (-xb[3 + q]) - B[q];
        if (udom[b] == j) {
            c64 Tv[3];
            ns_T(nb, tj, v, Tv);
            ns_bracket(nb, cf + 5, Tv, B);
            const c64 gs = gj * cf[4];
            for (int q = 0; q < 3; ++q) acc[3 + q] += gs * xb[3 + q] - B[q];
        }
    }
    c64 *ya = y + (r * N + a) * 6;
    for (int q = 0; q < 6; ++q) ya[q] += acc[q];
}

// y += correction^T x, thread per (source, right-hand side): the pairs of source b are
// tpair[tstart[b] .. tstart[b + 1]), each with its target tgt[p]
__global__ void k_ns_apply_t(int64_t N, int64_t nr, const int64_t *tstart, const int64_t *tpair, const int32_t *tgt,
                             const c64 *coef, const double *unrm, const int32_t *udom, const c64 *dc, const c64 *x,
                             c64 *y) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= N * nr) return;
    const int64_t b = idx % N, r = idx / N;
    const int64_t q0 = tstart[b], q1 = tstart[b + 1];
    if (q0 == q1) return;
    const int j = udom[b];
    const c64 tj = dc[3 * j + 1], gj = dc[3 * j + 2];
    const double nb[3] = {unrm[3 * b], unrm[3 * b + 1], unrm[3 * b + 2]};
    const double n0[3] = {-nb[0], -nb[1], -nb[2]};
    c64 acc[6] = {};
    for (int64_t k = q0; k < q1; ++k) {
        const int64_t p = tpair[k];
        const int32_t a = tgt[p];
        const c64 *cf = coef + 8 * p;
        const c64 *xa = x + (r * N + a) * 6;
        c64 u[3] = {xa[0], xa[1], xa[2]}, B[3];
        ns_bracket_t(n0, cf + 1, u, B);
        for (int q = 0; q < 3; ++q) {
            acc[q] -= B[q];
            acc[3 + q] -= cf[0] * u[q];
        }
        if (udom[a] == j) {
            c64 us[3] = {xa[3], xa[4], xa[5]}, TB[3];
            ns_bracket_t(nb, cf + 5, us, B);
            ns_T(nb, tj, B, TB);
            const c64 gs = gj * cf[4];
            for (int q = 0; q < 3; ++q) {
                acc[q] -= TB[q];
                acc[3 + q] += gs * us[q];
            }
        }
    }
    c64 *yb = y + (r * N + b) * 6;
    for (int q = 0; q < 6; ++q) yb[q] += acc[q];
}

}  // namespace

void build_near_singular(fmbem *h, const fmbem_mesh *mesh, cudaStream_t s) {
    const double rho = h->opt.near_singular_radius;
    const int L = h->opt.near_singular_levels;
    if (!(rho > 0)) return;
    if (h->ibc)
        throw fmbem_error{FMBEM_ERR_INVALID_ARGUMENT, "near_singular_radius > 0 needs the penetrable boundary"};
    const int64_t N = h->N, nv = mesh->n_vertices, nt = mesh->n_triangles;
    const double wmax = *std::max_element(h->h_w.begin(), h->h_w.end());
    const double leaf_w = h->lev[h->lmax].w;
    if (rho * std::sqrt(wmax) > leaf_w)
        throw fmbem_error{FMBEM_ERR_INVALID_ARGUMENT,
                          "near_singular_radius * sqrt(max node weight) = " + std::to_string(rho * std::sqrt(wmax)) +
                              " exceeds the leaf box width " + std::to_string(leaf_w) +
                              " (the Neighbor leaves would miss pairs): use a smaller radius or larger leaves"};
    const bool vertex = h->opt.node_mode == FMBEM_NODES_VERTEX;
    // patch pieces
    std::vector<int32_t> pcs(N + 1);
    if (vertex)
        for (int64_t v = 0; v <= N; ++v) pcs[v] = 2 * h->h_vt_start[v];
    else
        for (int64_t t = 0; t <= N; ++t) pcs[t] = (int32_t)t;
    const int64_t npc = pcs[N];
    double *dV = (double *)dev_alloc(h, sizeof(double) * 3 * nv);
    int32_t *dF = (int32_t *)dev_alloc(h, sizeof(int32_t) * 3 * nt);
    int32_t *dpcs = (int32_t *)dev_alloc(h, sizeof(int32_t) * (N + 1));
    double *dpc = (double *)dev_alloc(h, sizeof(double) * 9 * npc);
    CK(cudaMemcpyAsync(dV, mesh->vertices, sizeof(double) * 3 * nv, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dF, mesh->triangles, sizeof(int32_t) * 3 * nt, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dpcs, pcs.data(), sizeof(int32_t) * (N + 1), cudaMemcpyHostToDevice, s));
    const int TB = 128;
    if (vertex) {
        int32_t *dvs = (int32_t *)dev_alloc(h, sizeof(int32_t) * (nv + 1));
        int32_t *dvt = (int32_t *)dev_alloc(h, sizeof(int32_t) * 3 * nt);
        CK(cudaMemcpyAsync(dvs, h->h_vt_start.data(), sizeof(int32_t) * (nv + 1), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dvt, h->h_vt_tri.data(), sizeof(int32_t) * 3 * nt, cudaMemcpyHostToDevice, s));
        k_ns_pieces_vertex<<<(unsigned)((nv + TB - 1) / TB), TB, 0, s>>>(nv, dV, dF, dvs, dvt, dpc);
        CKL("k_ns_pieces_vertex");
        CK(cudaStreamSynchronize(s));
        dev_free(h, dvs);
        dev_free(h, dvt);
    } else {
        k_ns_pieces_centroid<<<(unsigned)((nt + TB - 1) / TB), TB, 0, s>>>(nt, dV, dF, dpc);
        CKL("k_ns_pieces_centroid");
    }
    // pairs: count, prefix sum, fill
    int32_t *dcnt = (int32_t *)dev_alloc(h, sizeof(int32_t) * N);
    k_ns_pairs<<<(unsigned)((N + TB - 1) / TB), TB, 0, s>>>(N, rho, h->box_leafpos, h->node_leaf, h->nbr_start, h->nbr_idx, h->box_nbeg,
                                                          h->box_nend, h->pos, h->w, h->perm, dcnt, nullptr, nullptr,
                                                          nullptr);
    CKL("k_ns_pairs");
    std::vector<int32_t> cnt(N);
    CK(cudaMemcpyAsync(cnt.data(), dcnt, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<int64_t> start(N + 1, 0);
    for (int64_t i = 0; i < N; ++i) start[i + 1] = start[i] + cnt[i];
    const int64_t np = start[N];
    h->ns_pairs = np;
    h->ns_start = (int64_t *)dev_alloc(h, sizeof(int64_t) * (N + 1));
    CK(cudaMemcpyAsync(h->ns_start, start.data(), sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice, s));
    if (np > 0) {
        h->ns_tgt = (int32_t *)dev_alloc(h, sizeof(int32_t) * np);
        h->ns_src = (int32_t *)dev_alloc(h, sizeof(int32_t) * np);
        h->ns_coef = (c64 *)dev_alloc(h, sizeof(c64) * 8 * np);
        k_ns_pairs<<<(unsigned)((N + TB - 1) / TB), TB, 0, s>>>(N, rho, h->box_leafpos, h->node_leaf, h->nbr_start, h->nbr_idx,
                                                              h->box_nbeg, h->box_nend, h->pos, h->w, h->perm, dcnt,
                                                              h->ns_start, h->ns_tgt, h->ns_src);
        CKL("k_ns_pairs");
        const int64_t threads = 32 * np;
        k_ns_coef<<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(np, L, h->ns_tgt, h->ns_src, dpcs, dpc, h->upos,
                                                                   h->uw, h->udom, (const c64 *)h->dcons, h->ns_coef);
        CKL("k_ns_coef");
        // by-source index for the transposed product (a counting sort of the pairs by source)
        std::vector<int32_t> srcs(np);
        CK(cudaMemcpyAsync(srcs.data(), h->ns_src, sizeof(int32_t) * np, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        std::vector<int64_t> ts(N + 1, 0), tp(np);
        for (int64_t p = 0; p < np; ++p) ts[srcs[p] + 1]++;
        for (int64_t i = 0; i < N; ++i) ts[i + 1] += ts[i];
        std::vector<int64_t> fill(ts.begin(), ts.end() - 1);
        for (int64_t p = 0; p < np; ++p) tp[fill[srcs[p]]++] = p;
        h->ns_tstart = (int64_t *)dev_alloc(h, sizeof(int64_t) * (N + 1));
        h->ns_tpair = (int64_t *)dev_alloc(h, sizeof(int64_t) * np);
        CK(cudaMemcpyAsync(h->ns_tstart, ts.data(), sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(h->ns_tpair, tp.data(), sizeof(int64_t) * np, cudaMemcpyHostToDevice, s));
    }
    CK(cudaStreamSynchronize(s));
    dev_free(h, dcnt);
    dev_free(h, dV);
    dev_free(h, dF);
    dev_free(h, dpcs);
    dev_free(h, dpc);
}

void apply_near_singular(fmbem *h, const c64 *x, c64 *y, int64_t nr, cudaStream_t s, bool transpose) {
    if (h->ns_pairs <= 0) return;
    const int64_t n = h->N * nr;
    const unsigned grid = (unsigned)((n + 127) / 128);
    if (transpose)
        k_ns_apply_t<<<grid, 128, 0, s>>>(h->N, nr, h->ns_tstart, h->ns_tpair, h->ns_tgt, h->ns_coef, h->unrm, h->udom,
                                          (const c64 *)h->dcons, x, y);
    else
        k_ns_apply<<<grid, 128, 0, s>>>(h->N, nr, h->ns_start, h->ns_src, h->ns_coef, h->unrm, h->udom,
                                        (const c64 *)h->dcons, x, y);
    CKL("k_ns_apply");
}
