// geometry.cu -- Nystrom nodes (Eq. 2.8), analytic self-patch integrals (Appendix B), the 6x6
// self blocks A_self of Eq. (3.2) with their LU factors, the block-diagonal preconditioner and the
// plane-wave right-hand sides (Eq. 2.12).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>

#include "fmbem_internal.cuh"

namespace {

__device__ __forceinline__ void sub3(const double *a, const double *b, double *o) {
    o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
__device__ __forceinline__ double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
__device__ __forceinline__ void cross3(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// Appendix B integrals over a planar polygon around O accumulated edge by edge in their boundary
// (divergence-theorem) form: for the edge a -> b (points relative to O, in the plane of unit
// normal n, traversed counter-clockwise about n) with outward in-plane normal nu = e x n/|e|,
// signed distance h = nu.a and tangential coordinate t = e/|e| . r,
//   int dA/rho       = sum h   int_e dt / sqrt(h^2+t^2)      (div rhohat = 1/rho)
//   int r/r dA       = sum nu  int_e sqrt(h^2+t^2) dt         (grad rho = rhohat)
//   CPV int r/r^3 dA = -sum nu int_e dt / sqrt(h^2+t^2)      (grad 1/rho = -rhohat/rho^2)
//   area             = sum h |e| / 2
struct PatchSums {
    double I1 = 0, S = 0, V1[3] = {0, 0, 0}, V3[3] = {0, 0, 0};
};
__device__ void patch_edge(const double *a, const double *b, const double *n, PatchSums &ps) {
    double e[3];
    sub3(b, a, e);
    double le = sqrt(dot3(e, e));
    if (le <= 0) return;
    double nu[3];
    cross3(e, n, nu);
    for (int q = 0; q < 3; ++q) nu[q] /= le;
    double h = dot3(nu, a);
    double ah = fabs(h);
    if (ah <= 1e-300) return;
    double ta = dot3(e, a) / le, tb = dot3(e, b) / le;
    double L = asinh(tb / ah) - asinh(ta / ah);
    double M = 0.5 * (tb * sqrt(h * h + tb * tb) - ta * sqrt(h * h + ta * ta)) + 0.5 * h * h * L;
    ps.I1 += h * L;
    ps.S += 0.5 * h * le;
    for (int q = 0; q < 3; ++q) {
        ps.V1[q] += nu[q] * M;
        ps.V3[q] -= nu[q] * L;
    }
}

__device__ void project_rel(const double *P, const double *O, const double *n, double *out) {
    double d[3];
    sub3(P, O, d);
    double a = dot3(d, n);
    for (int q = 0; q < 3; ++q) out[q] = d[q] - a * n[q];
}

// self blocks and LU for one node; ps are its patch integrals, n its outward normal.  With an
// impedance boundary (ibc) the scatterer rows are the local relation of Eq. (2.24),
// Psi - zeta (Phi - n (n.Phi)) = 0, zeta = i k0 mu_0 / Z.
__device__ void self_block(const PatchSums &ps, const double *n, c64 kb, c64 kj, c64 tj, c64 gj, bool ibc, c64 zeta,
                           c64 *M, c64 *LU, int8_t *piv) {
    const double inv4pi = 1.0 / (4.0 * FMBEM_PI), inv8pi = 1.0 / (8.0 * FMBEM_PI);
    for (int i = 0; i < 36; ++i) M[i] = {0, 0};
    for (int side = 0; side < 2; ++side) {
        c64 k = side == 0 ? kb : kj;
        double sgn = side == 0 ? -1.0 : 1.0;
        double nd[3] = {sgn * n[0], sgn * n[1], sgn * n[2]};
        // Eq. (B.2): int g dA ~ (I1 + i k S)/(4 pi);  Eq. (B.4): int grad'g dA ~ -k^2/(8pi) V1 - V3/(4pi)
        c64 Sg = c64{ps.I1 * inv4pi, 0.0} + (c64{0.0, ps.S * inv4pi} * k);
        c64 k2 = k * k;
        c64 Sdg[3];
        for (int q = 0; q < 3; ++q) Sdg[q] = (-inv8pi * ps.V1[q]) * k2 - c64{ps.V3[q] * inv4pi, 0.0};
        c64 nS = nd[0] * Sdg[0] + nd[1] * Sdg[1] + nd[2] * Sdg[2];
        // bracket B[q][p] = n_q Sdg_p - (n.Sdg) delta_qp - Sdg_q n_p (Eq. 2.12 with grad'g -> Sdg)
        c64 B[3][3];
        for (int q = 0; q < 3; ++q)
            for (int p = 0; p < 3; ++p) {
                c64 v = nd[q] * Sdg[p] - Sdg[q] * nd[p];
                if (p == q) v -= nS;
                B[q][p] = v;
            }
        // T of this side: identity for the background, I + t n n^T for the scatterer (Eq. 2.13)
        c64 T[3][3];
        for (int q = 0; q < 3; ++q)
            for (int p = 0; p < 3; ++p) {
                T[q][p] = (side == 1) ? (n[q] * n[p]) * tj : c64{0, 0};
                if (p == q) T[q][p] += c64{1.0, 0.0};
            }
        for (int q = 0; q < 3; ++q)
            for (int c = 0; c < 3; ++c) {
                c64 acc = 0.5 * T[q][c];
                for (int p = 0; p < 3; ++p) acc -= B[q][p] * T[p][c];
                M[(3 * side + q) * 6 + c] = acc;
            }
        // Psi columns: background uses n0 x curl E = -Psi (gamma_0 = 1), scatterer gamma_j Sg
        c64 dpsi = side == 0 ? -Sg : (gj * Sg);
        for (int q = 0; q < 3; ++q) M[(3 * side + q) * 6 + 3 + q] = dpsi;
    }
    if (ibc)
        for (int q = 0; q < 3; ++q)
            for (int c = 0; c < 6; ++c) {
                c64 v = {0, 0};
                if (c < 3) v = zeta * (n[q] * n[c] - (q == c ? 1.0 : 0.0));
                else if (c == 3 + q) v = {1.0, 0.0};
                M[(3 + q) * 6 + c] = v;
            }
    // LU with partial pivoting, row-major 6x6
    for (int i = 0; i < 36; ++i) LU[i] = M[i];
    for (int c = 0; c < 6; ++c) {
        int pv = c;
        double best = abs2(LU[c * 6 + c]);
        for (int r = c + 1; r < 6; ++r)
            if (abs2(LU[r * 6 + c]) > best) { best = abs2(LU[r * 6 + c]); pv = r; }
        piv[c] = (int8_t)pv;
        if (pv != c)
            for (int j = 0; j < 6; ++j) { c64 t = LU[c * 6 + j]; LU[c * 6 + j] = LU[pv * 6 + j]; LU[pv * 6 + j] = t; }
        c64 d = LU[c * 6 + c];
        for (int r = c + 1; r < 6; ++r) {
            c64 f = cdiv(LU[r * 6 + c], d);
            LU[r * 6 + c] = f;
            for (int j = c + 1; j < 6; ++j) LU[r * 6 + j] -= f * LU[c * 6 + j];
        }
    }
}

__device__ void domain_consts(const c64 *kd, const c64 *td, const c64 *gd, int j, c64 &kb, c64 &kj, c64 &tj, c64 &gj) {
    kb = kd[0]; kj = kd[j]; tj = td[j]; gj = gd[j];
}
__device__ c64 zeta_of(const c64 *zd, int j) { return zd ? zd[j] : c64{0, 0}; }

// vertex positions read as stored, or with one vertex displaced (the shape gradient)
struct PlainPos {
    const double *V;
    __device__ void operator()(int64_t i, double *o) const { o[0] = V[3 * i]; o[1] = V[3 * i + 1]; o[2] = V[3 * i + 2]; }
};
struct MovedPos {
    const double *V;
    int64_t moved;
    double d[3];
    __device__ void operator()(int64_t i, double *o) const {
        for (int q = 0; q < 3; ++q) o[q] = V[3 * i + q] + (i == moved ? d[q] : 0.0);
    }
};

// vertex node v: weight 1/3 of incident areas, area-weighted normal, dual-cell patch integrals
template <class Pos>
__device__ void vertex_geometry(int64_t v, const Pos &P, const int32_t *F, const int32_t *vt_start,
                                const int32_t *vt_tri, double *O, double *n, double &wsum, PatchSums &ps) {
    P(v, O);
    double nsum[3] = {0, 0, 0};
    wsum = 0;
    for (int q = vt_start[v]; q < vt_start[v + 1]; ++q) {
        int t = vt_tri[q];
        double A[3], B[3], C[3];
        P(F[3 * t], A); P(F[3 * t + 1], B); P(F[3 * t + 2], C);
        double ab[3], ac[3], cr[3];
        sub3(B, A, ab); sub3(C, A, ac); cross3(ab, ac, cr);
        for (int i = 0; i < 3; ++i) nsum[i] += cr[i];
        wsum += sqrt(dot3(cr, cr)) / 6.0;
    }
    double ln = sqrt(dot3(nsum, nsum));
    for (int i = 0; i < 3; ++i) n[i] = nsum[i] / ln;
    for (int q = vt_start[v]; q < vt_start[v + 1]; ++q) {
        int t = vt_tri[q];
        int c0 = F[3 * t] == v ? 0 : (F[3 * t + 1] == v ? 1 : 2);
        double A[3], B[3], C[3];
        P(F[3 * t + c0], A); P(F[3 * t + (c0 + 1) % 3], B); P(F[3 * t + (c0 + 2) % 3], C);
        double mab[3], g[3], mac[3];
        for (int i = 0; i < 3; ++i) {
            mab[i] = 0.5 * (A[i] + B[i]);
            mac[i] = 0.5 * (A[i] + C[i]);
            g[i] = (A[i] + B[i] + C[i]) / 3.0;
        }
        double pa[3], pg[3], pc[3];
        project_rel(mab, O, n, pa); project_rel(g, O, n, pg); project_rel(mac, O, n, pc);
        patch_edge(pa, pg, n, ps);
        patch_edge(pg, pc, n, ps);
    }
}

__global__ void k_vertex_nodes(int64_t nv, const double *V, const int32_t *F, const int32_t *vt_start,
                               const int32_t *vt_tri, const int32_t *vdom, const c64 *kd, const c64 *td, const c64 *gd,
                               const c64 *zd, double *pos, double *nrm, double *w, c64 *M, c64 *LU, int8_t *piv) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= nv) return;
    double O[3], n[3], wsum;
    PatchSums ps;
    vertex_geometry(v, PlainPos{V}, F, vt_start, vt_tri, O, n, wsum, ps);
    for (int i = 0; i < 3; ++i) { pos[3 * v + i] = O[i]; nrm[3 * v + i] = n[i]; }
    w[v] = wsum;
    c64 kb, kj, tj, gj;
    domain_consts(kd, td, gd, vdom[v], kb, kj, tj, gj);
    self_block(ps, n, kb, kj, tj, gj, zd != nullptr, zeta_of(zd, vdom[v]), M + 36 * v, LU + 36 * v, piv + 6 * v);
}

// Shape gradient, local part (vertex nodes): for vertex v and coordinate c, the central
// difference (step hv) of everything in G = L^T x + lambda^T b - lambda^T A x that depends on
// vertex v through the node data of the nodes u of its 1-ring S_v (v and the other vertices of
// the triangles at v): the node data themselves enter through the sensitivities sens[r][u] =
// dG/d(s_u, w_u, n_u) (pair terms, functional and right-hand side, from k_node_sens), and the self
// blocks M_u (Appendix B) directly: out[r][v][c] = sum_u [sens_u . d(s,w,n)_u - lambda_u^T dM_u x_u].
// One thread per vertex; err is set when a 1-ring has more than SG_RING nodes.
constexpr int SG_RING = 32;
__global__ void k_vertex_shape_grad(int64_t nv, int64_t nr, const double *V, const int32_t *F, const int32_t *vt_start,
                                    const int32_t *vt_tri, const int32_t *vdom, const c64 *kd, const c64 *td,
                                    const c64 *gd, const c64 *x, const c64 *lam, const c64 *sens, double hv, c64 *out,
                                    int *err) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= nv) return;
    int64_t ring[SG_RING];
    int nring = 0;
    for (int q = vt_start[v]; q < vt_start[v + 1]; ++q)
        for (int a = 0; a < 3; ++a) {
            const int64_t u = F[3 * vt_tri[q] + a];
            bool seen = false;
            for (int i = 0; i < nring; ++i) seen |= ring[i] == u;
            if (seen) continue;
            if (nring == SG_RING) { atomicExch(err, 1); return; }
            ring[nring++] = u;
        }
    for (int c = 0; c < 3; ++c) {
        for (int64_t r = 0; r < nr; ++r) out[(r * nv + v) * 3 + c] = {0, 0};
        for (int i = 0; i < nring; ++i) {
            const int64_t u = ring[i];
            double Op[3], Om[3], np_[3], nm[3], wp, wm;
            PatchSums pp, pm;
            MovedPos Pp{V, v, {0, 0, 0}}, Pm{V, v, {0, 0, 0}};
            Pp.d[c] = hv;
            Pm.d[c] = -hv;
            vertex_geometry(u, Pp, F, vt_start, vt_tri, Op, np_, wp, pp);
            vertex_geometry(u, Pm, F, vt_start, vt_tri, Om, nm, wm, pm);
            c64 kb, kj, tj, gj;
            domain_consts(kd, td, gd, vdom[u], kb, kj, tj, gj);
            c64 Mp[36], Mm[36], LU[36];
            int8_t piv[6];
            self_block(pp, np_, kb, kj, tj, gj, false, c64{0, 0}, Mp, LU, piv);
            self_block(pm, nm, kb, kj, tj, gj, false, c64{0, 0}, Mm, LU, piv);
            const double inv2h = 1.0 / (2.0 * hv);
            for (int64_t r = 0; r < nr; ++r) {
                const c64 *su = sens + (r * nv + u) * 7;
                const c64 *xu = x + (r * nv + u) * 6, *lu = lam + (r * nv + u) * 6;
                c64 acc = {0, 0};
                for (int q = 0; q < 3; ++q) acc += su[q] * ((Op[q] - Om[q]) * inv2h);
                acc += su[3] * ((wp - wm) * inv2h);
                for (int q = 0; q < 3; ++q) acc += su[4 + q] * ((np_[q] - nm[q]) * inv2h);
                for (int a = 0; a < 6; ++a) {
                    c64 row = {0, 0};
                    for (int b = 0; b < 6; ++b) row += (Mp[6 * a + b] - Mm[6 * a + b]) * xu[b];
                    acc -= lu[a] * row * inv2h;
                }
                out[(r * nv + v) * 3 + c] += acc;
            }
        }
    }
}

// centroid nodes: the triangle is its own patch
__global__ void k_centroid_nodes(int64_t nt, const double *V, const int32_t *F, const int32_t *tdom, const c64 *kd,
                                 const c64 *td, const c64 *gd, const c64 *zd, double *pos, double *nrm, double *w, c64 *M,
                                 c64 *LU, int8_t *piv) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const double *A = V + 3 * F[3 * t], *B = V + 3 * F[3 * t + 1], *C = V + 3 * F[3 * t + 2];
    double ab[3], ac[3], cr[3];
    sub3(B, A, ab); sub3(C, A, ac); cross3(ab, ac, cr);
    double l = sqrt(dot3(cr, cr));
    double n[3] = {cr[0] / l, cr[1] / l, cr[2] / l};
    double O[3];
    for (int i = 0; i < 3; ++i) O[i] = (A[i] + B[i] + C[i]) / 3.0;
    double pa[3], pb[3], pc[3];
    project_rel(A, O, n, pa); project_rel(B, O, n, pb); project_rel(C, O, n, pc);
    PatchSums ps;
    patch_edge(pa, pb, n, ps);
    patch_edge(pb, pc, n, ps);
    patch_edge(pc, pa, n, ps);
    for (int i = 0; i < 3; ++i) { pos[3 * t + i] = O[i]; nrm[3 * t + i] = n[i]; }
    w[t] = 0.5 * l;
    c64 kb, kj, tj, gj;
    domain_consts(kd, td, gd, tdom[t], kb, kj, tj, gj);
    self_block(ps, n, kb, kj, tj, gj, zd != nullptr, zeta_of(zd, tdom[t]), M + 36 * t, LU + 36 * t, piv + 6 * t);
}

// z = M^{-1} v per node (Eq. 3.1-3.2), vectors in user order [n_rhs][N][6]
__global__ void k_precond(int64_t N, int64_t n_rhs, const c64 *LU, const int8_t *piv, const c64 *v, c64 *z) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N * n_rhs) return;
    int64_t a = i % N;
    const c64 *L = LU + 36 * a;
    c64 b[6];
    for (int q = 0; q < 6; ++q) b[q] = v[6 * i + q];
    for (int c = 0; c < 6; ++c) {
        int pv = piv[6 * a + c];
        if (pv != c) { c64 t = b[c]; b[c] = b[pv]; b[pv] = t; }
        for (int r = c + 1; r < 6; ++r) b[r] -= L[r * 6 + c] * b[c];
    }
    for (int r = 5; r >= 0; --r) {
        c64 acc = b[r];
        for (int c = r + 1; c < 6; ++c) acc -= L[r * 6 + c] * b[c];
        b[r] = cdiv(acc, L[r * 6 + r]);
    }
    for (int q = 0; q < 6; ++q) z[6 * i + q] = b[q];
}

// z = M^-T v (the transposed preconditioner of the adjoint solve) from the LU factors PM = LU:
// M^T = U^T L^T P, so U^T y = v (forward), L^T w = y (backward, unit diagonal), z = P^T w (the
// row swaps undone in reverse order)
__global__ void k_precond_t(int64_t N, int64_t n_rhs, const c64 *LU, const int8_t *piv, const c64 *v, c64 *z) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N * n_rhs) return;
    const int64_t a = i % N;
    const c64 *L = LU + 36 * a;
    c64 b[6];
    for (int q = 0; q < 6; ++q) b[q] = v[6 * i + q];
    for (int r = 0; r < 6; ++r) {
        c64 acc = b[r];
        for (int c = 0; c < r; ++c) acc -= L[c * 6 + r] * b[c];
        b[r] = cdiv(acc, L[r * 6 + r]);
    }
    for (int r = 5; r >= 0; --r)
        for (int c = r + 1; c < 6; ++c) b[r] -= L[c * 6 + r] * b[c];
    for (int c = 5; c >= 0; --c) {
        const int pv = piv[6 * a + c];
        if (pv != c) { c64 t = b[c]; b[c] = b[pv]; b[pv] = t; }
    }
    for (int q = 0; q < 6; ++q) z[6 * i + q] = b[q];
}

// z = M^-T v with the single-precision explicit inverse (adjoint inner iterations)
__global__ void k_precond32_t(int64_t N, int64_t n_rhs, const c32 *Minv, const c32 *v, c64 *z) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N * n_rhs) return;
    const c32 *M = Minv + 36 * (i % N);
    c32 b[6];
    for (int q = 0; q < 6; ++q) b[q] = v[6 * i + q];
    for (int r = 0; r < 6; ++r) {
        c32 acc = {0.f, 0.f};
        for (int c = 0; c < 6; ++c) cfma(acc, M[6 * c + r], b[c]);
        z[6 * i + r] = c64{(double)acc.re, (double)acc.im};
    }
}

// explicit inverse of each node's 6x6 block M (Eq. 3.2) from its LU factors, column by column in
// double precision, stored in single precision for the inner iterations of the refined solve
__global__ void k_inverse32(int64_t N, const c64 *LU, const int8_t *piv, c32 *Minv) {
    const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= N) return;
    const c64 *L = LU + 36 * a;
    for (int j = 0; j < 6; ++j) {
        c64 b[6];
        for (int q = 0; q < 6; ++q) b[q] = c64{q == j ? 1.0 : 0.0, 0.0};
        for (int c = 0; c < 6; ++c) {
            const int pv = piv[6 * a + c];
            if (pv != c) { c64 t = b[c]; b[c] = b[pv]; b[pv] = t; }
            for (int r = c + 1; r < 6; ++r) b[r] -= L[r * 6 + c] * b[c];
        }
        for (int r = 5; r >= 0; --r) {
            c64 acc = b[r];
            for (int c = r + 1; c < 6; ++c) acc -= L[r * 6 + c] * b[c];
            b[r] = cdiv(acc, L[r * 6 + r]);
        }
        for (int r = 0; r < 6; ++r) Minv[36 * a + 6 * r + j] = c32{(float)b[r].re, (float)b[r].im};
    }
}

// z = M^-1 v with the single-precision explicit inverse; v single, z double precision
__global__ void k_precond32(int64_t N, int64_t n_rhs, const c32 *Minv, const c32 *v, c64 *z) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N * n_rhs) return;
    const c32 *M = Minv + 36 * (i % N);
    c32 b[6];
    for (int q = 0; q < 6; ++q) b[q] = v[6 * i + q];
    for (int r = 0; r < 6; ++r) {
        c32 acc = {0.f, 0.f};
        for (int c = 0; c < 6; ++c) cfma(acc, M[6 * r + c], b[c]);
        z[6 * i + r] = c64{(double)acc.re, (double)acc.im};
    }
}

// b = [e exp(i k_0 d.s); 0] per node (Eq. 2.12, Phi_inc); nodes in user order
__global__ void k_plane_wave(int64_t N, int64_t n_rhs, const double *pos_user, const double *dir, const c64 *pol, c64 k0,
                             c64 *b) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N * n_rhs) return;
    int64_t r = i / N, a = i % N;
    const double *d = dir + 3 * r;
    double ds = d[0] * pos_user[3 * a] + d[1] * pos_user[3 * a + 1] + d[2] * pos_user[3 * a + 2];
    c64 ph = cexpd(c64{0.0, 1.0} * (k0 * ds));
    for (int q = 0; q < 3; ++q) {
        b[6 * i + q] = pol[3 * r + q] * ph;
        b[6 * i + 3 + q] = {0, 0};
    }
}

}  // namespace

// ------------------------------------------------------------------------------------------
// host: mesh validation (closed, consistently oriented, domain ids) and node set-up
void build_geometry(fmbem *h, const fmbem_mesh *mesh, cudaStream_t s) {
    const int64_t nv = mesh->n_vertices, nt = mesh->n_triangles;
    const double *V = mesh->vertices;
    const int32_t *F = mesh->triangles, *TD = mesh->tri_domain;
    auto bad = [](const std::string &m) { throw fmbem_error{FMBEM_ERR_INVALID_MESH, m}; };
    if (nv < 3 || nt < 4) bad("mesh needs at least 3 vertices and 4 triangles");
    for (int64_t t = 0; t < nt; ++t) {
        for (int a = 0; a < 3; ++a)
            if (F[3 * t + a] < 0 || F[3 * t + a] >= nv) bad("triangle " + std::to_string(t) + ": vertex index out of range");
        if (F[3 * t] == F[3 * t + 1] || F[3 * t + 1] == F[3 * t + 2] || F[3 * t] == F[3 * t + 2])
            bad("triangle " + std::to_string(t) + " repeats a vertex");
        if (TD[t] < 1 || TD[t] > h->J) bad("triangle " + std::to_string(t) + ": domain id outside 1..n_scatterers");
        const double *A = V + 3 * F[3 * t], *B = V + 3 * F[3 * t + 1], *C = V + 3 * F[3 * t + 2];
        double ab[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]}, ac[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
        double cr[3] = {ab[1] * ac[2] - ab[2] * ac[1], ab[2] * ac[0] - ab[0] * ac[2], ab[0] * ac[1] - ab[1] * ac[0]};
        double a2 = cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2];
        double l2 = (ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2]) * (ac[0] * ac[0] + ac[1] * ac[1] + ac[2] * ac[2]);
        if (!(a2 > 1e-24 * l2) || !std::isfinite(a2)) bad("triangle " + std::to_string(t) + " is degenerate");
    }
    // every directed edge once, and its reverse once (closed, consistently oriented surface)
    std::unordered_map<uint64_t, int64_t> edges;
    edges.reserve((size_t)(3 * nt * 2));
    for (int64_t t = 0; t < nt; ++t)
        for (int a = 0; a < 3; ++a) {
            uint64_t u = (uint64_t)F[3 * t + a], v = (uint64_t)F[3 * t + (a + 1) % 3];
            auto r = edges.emplace(u * (uint64_t)nv + v, t);
            if (!r.second) bad("edge (" + std::to_string(u) + "," + std::to_string(v) + ") is used twice with the same orientation");
        }
    for (auto &kv : edges) {
        uint64_t u = kv.first / (uint64_t)nv, v = kv.first % (uint64_t)nv;
        auto it = edges.find(v * (uint64_t)nv + u);
        if (it == edges.end()) bad("edge (" + std::to_string(u) + "," + std::to_string(v) + ") has no opposite: surface not closed or not consistently oriented");
        if (TD[it->second] != TD[kv.second]) bad("an edge joins two scatterers (junctions are not supported)");
    }

    const bool vertex = h->opt.node_mode == FMBEM_NODES_VERTEX;
    const int64_t N = vertex ? nv : nt;
    h->N = N;
    std::vector<int32_t> ndom(N);
    std::vector<int32_t> vt_start, vt_tri;
    if (vertex) {
        std::vector<int32_t> cnt(nv + 1, 0);
        std::fill(ndom.begin(), ndom.end(), 0);
        for (int64_t t = 0; t < nt; ++t)
            for (int a = 0; a < 3; ++a) {
                int32_t v = F[3 * t + a];
                cnt[v + 1]++;
                if (ndom[v] == 0) ndom[v] = TD[t];
                else if (ndom[v] != TD[t]) bad("vertex " + std::to_string(v) + " touches two scatterers");
            }
        for (int64_t v = 0; v < nv; ++v)
            if (cnt[v + 1] == 0) bad("vertex " + std::to_string(v) + " is not used by any triangle");
        for (int64_t v = 0; v < nv; ++v) cnt[v + 1] += cnt[v];
        vt_start = cnt;
        vt_tri.resize(3 * nt);
        std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
        for (int64_t t = 0; t < nt; ++t)
            for (int a = 0; a < 3; ++a) vt_tri[fill[F[3 * t + a]]++] = (int32_t)t;
    } else {
        for (int64_t t = 0; t < nt; ++t) ndom[t] = TD[t];
    }

    // media tables (Eq. 2.13): k_d, t_d = (eps_0 - eps_d)/eps_d, gamma_d = mu_d/mu_0
    int J = h->J;
    std::vector<c64> kd(J + 1), td(J + 1), gd(J + 1);
    for (int d = 0; d <= J; ++d) {
        kd[d] = h->k[d];
        td[d] = d == 0 ? c64{0, 0} : cdiv(h->eps[0] - h->eps[d], h->eps[d]);
        gd[d] = h->gam[d];
    }

    // device inputs
    double *dV = (double *)dev_alloc(h, sizeof(double) * 3 * nv);
    int32_t *dF = (int32_t *)dev_alloc(h, sizeof(int32_t) * 3 * nt);
    int32_t *dDom = (int32_t *)dev_alloc(h, sizeof(int32_t) * N);
    c64 *dk = (c64 *)dev_alloc(h, sizeof(c64) * (J + 1));
    c64 *dt = (c64 *)dev_alloc(h, sizeof(c64) * (J + 1));
    c64 *dg = (c64 *)dev_alloc(h, sizeof(c64) * (J + 1));
    CK(cudaMemcpyAsync(dV, V, sizeof(double) * 3 * nv, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dF, F, sizeof(int32_t) * 3 * nt, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dDom, ndom.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dk, kd.data(), sizeof(c64) * (J + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dt, td.data(), sizeof(c64) * (J + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dg, gd.data(), sizeof(c64) * (J + 1), cudaMemcpyHostToDevice, s));

    double *upos = (double *)dev_alloc(h, sizeof(double) * 3 * N);
    double *unrm = (double *)dev_alloc(h, sizeof(double) * 3 * N);
    double *uw = (double *)dev_alloc(h, sizeof(double) * N);
    h->Mself = (c64 *)dev_alloc(h, sizeof(c64) * 36 * N);
    h->Mlu = (c64 *)dev_alloc(h, sizeof(c64) * 36 * N);
    h->piv = (int8_t *)dev_alloc(h, 6 * N);
    const int TB = 128;
    if (vertex) {
        int32_t *dvs = (int32_t *)dev_alloc(h, sizeof(int32_t) * (nv + 1));
        int32_t *dvt = (int32_t *)dev_alloc(h, sizeof(int32_t) * 3 * nt);
        CK(cudaMemcpyAsync(dvs, vt_start.data(), sizeof(int32_t) * (nv + 1), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dvt, vt_tri.data(), sizeof(int32_t) * 3 * nt, cudaMemcpyHostToDevice, s));
        k_vertex_nodes<<<(unsigned)((nv + TB - 1) / TB), TB, 0, s>>>(nv, dV, dF, dvs, dvt, dDom, dk, dt, dg, h->d_zeta, upos,
                                                                   unrm, uw, h->Mself, h->Mlu, h->piv);
        CKL("k_vertex_nodes");
        CK(cudaStreamSynchronize(s));
        dev_free(h, dvs);
        dev_free(h, dvt);
    } else {
        k_centroid_nodes<<<(unsigned)((nt + TB - 1) / TB), TB, 0, s>>>(nt, dV, dF, dDom, dk, dt, dg, h->d_zeta, upos, unrm,
                                                                     uw, h->Mself, h->Mlu, h->piv);
        CKL("k_centroid_nodes");
    }
    if (vertex) {  // kept for the shape gradient
        h->h_F.assign(F, F + 3 * nt);
        h->h_vt_start = vt_start;
        h->h_vt_tri = vt_tri;
    }
    // host copies of the user-order geometry; the sorted copies are made by the tree build
    h->h_pos.resize(3 * N);
    h->h_nrm.resize(3 * N);
    h->h_w.resize(N);
    CK(cudaMemcpyAsync(h->h_pos.data(), upos, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h->h_nrm.data(), unrm, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h->h_w.data(), uw, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // keep user-order device geometry for the tree build and the plane-wave kernel
    h->upos = upos;
    h->unrm = unrm;
    h->uw = uw;
    h->udom = dDom;
    dev_free(h, dV);
    dev_free(h, dF);
    dev_free(h, dk);
    dev_free(h, dt);
    dev_free(h, dg);
}

void run_vertex_shape_grad(fmbem *h, int64_t nr, const c64 *x, const c64 *lam, const c64 *sens, double hv, c64 *out,
                           cudaStream_t s) {
    const int64_t nv = h->N, nt = (int64_t)h->h_F.size() / 3;
    std::vector<c64> kd(h->J + 1), td(h->J + 1), gd(h->J + 1);
    for (int d = 0; d <= h->J; ++d) {
        kd[d] = h->k[d];
        td[d] = d == 0 ? c64{0, 0} : cdiv(h->eps[0] - h->eps[d], h->eps[d]);
        gd[d] = h->gam[d];
    }
    int32_t *dF = (int32_t *)dev_alloc(h, sizeof(int32_t) * 3 * nt);
    int32_t *dvs = (int32_t *)dev_alloc(h, sizeof(int32_t) * (nv + 1));
    int32_t *dvt = (int32_t *)dev_alloc(h, sizeof(int32_t) * 3 * nt);
    c64 *dk = (c64 *)dev_alloc(h, sizeof(c64) * 3 * (h->J + 1));
    int *derr = (int *)dev_alloc(h, sizeof(int));
    auto cleanup = [&] {
        for (void *p : {(void *)dF, (void *)dvs, (void *)dvt, (void *)dk, (void *)derr}) dev_free(h, p);
    };
    try {
        CK(cudaMemcpyAsync(dF, h->h_F.data(), sizeof(int32_t) * 3 * nt, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dvs, h->h_vt_start.data(), sizeof(int32_t) * (nv + 1), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dvt, h->h_vt_tri.data(), sizeof(int32_t) * 3 * nt, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dk, kd.data(), sizeof(c64) * (h->J + 1), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dk + (h->J + 1), td.data(), sizeof(c64) * (h->J + 1), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dk + 2 * (h->J + 1), gd.data(), sizeof(c64) * (h->J + 1), cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(derr, 0, sizeof(int), s));
        k_vertex_shape_grad<<<(unsigned)((nv + 63) / 64), 64, 0, s>>>(nv, nr, h->upos, dF, dvs, dvt, h->udom, dk,
                                                                   dk + (h->J + 1), dk + 2 * (h->J + 1), x, lam, sens,
                                                                   hv, out, derr);
        CKL("k_vertex_shape_grad");
        int e = 0;
        CK(cudaMemcpyAsync(&e, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (e) throw fmbem_error{FMBEM_ERR_INVALID_MESH, "a vertex 1-ring holds more than 32 vertices"};
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
}

void run_precond(fmbem *h, const c64 *v, c64 *z, int64_t n_rhs, cudaStream_t s) {
    int64_t n = h->N * n_rhs;
    k_precond<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(h->N, n_rhs, h->Mlu, h->piv, v, z);
    CKL("k_precond");
}

void run_precond32(fmbem *h, const c32 *v, c64 *z, int64_t n_rhs, cudaStream_t s, bool transpose) {
    if (h->Minv32 == nullptr) {
        h->Minv32 = (c32 *)dev_alloc(h, sizeof(c32) * 36 * h->N);
        k_inverse32<<<(unsigned)((h->N + 127) / 128), 128, 0, s>>>(h->N, h->Mlu, h->piv, h->Minv32);
        CKL("k_inverse32");
    }
    const int64_t n = h->N * n_rhs;
    if (transpose) k_precond32_t<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(h->N, n_rhs, h->Minv32, v, z);
    else k_precond32<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(h->N, n_rhs, h->Minv32, v, z);
    CKL("k_precond32");
}

void run_precond_t(fmbem *h, const c64 *v, c64 *z, int64_t n_rhs, cudaStream_t s) {
    const int64_t n = h->N * n_rhs;
    k_precond_t<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(h->N, n_rhs, h->Mlu, h->piv, v, z);
    CKL("k_precond_t");
}

void run_plane_wave(fmbem *h, int64_t n_rhs, const double *dir, const fmbem_c64 *pol, c64 *b, cudaStream_t s) {
    double *ddir = (double *)dev_alloc(h, sizeof(double) * 3 * n_rhs);
    c64 *dpol = (c64 *)dev_alloc(h, sizeof(c64) * 3 * n_rhs);
    CK(cudaMemcpyAsync(ddir, dir, sizeof(double) * 3 * n_rhs, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dpol, pol, sizeof(c64) * 3 * n_rhs, cudaMemcpyHostToDevice, s));
    int64_t n = h->N * n_rhs;
    k_plane_wave<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(h->N, n_rhs, h->upos, ddir, dpol, h->k[0], b);
    CKL("k_plane_wave");
    CK(cudaStreamSynchronize(s));
    dev_free(h, ddir);
    dev_free(h, dpol);
}
