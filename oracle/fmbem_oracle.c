/*
 * fmbem_oracle.c -- plain FP64 CPU oracle for the Nystrom EFIE boundary-element operator of
 * Wang, Zheng, Xiao, Lin & Chan, "Fast multipole boundary element method for three dimensional
 * electromagnetic scattering problem" (arXiv 1211.7177).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or includes this
 * file; only the tests, the smoke check and the benchmark's CPU-baseline leg use it.  It shares
 * no code with the CUDA path.
 *
 * What it computes (all in double precision, dense, O(N^2), no fast multipole approximation):
 *   - Nystrom nodes, weights and normals, one-point rule of Eq. (2.8): triangle centroids with
 *     triangle areas (the paper's "simplest case"), or mesh vertices with one third of the
 *     incident triangle areas and the area-weighted normal.
 *   - Media quantities of Eq. (2.13): k_d = k0 sqrt(eps_d mu_d) (root with Im k >= 0),
 *     T_j = I + (eps_0 - eps_j)/eps_j n n^T, gamma_j = mu_j / mu_0.
 *   - Self-patch integrals of Appendix B, Eqs. (B.2)-(B.9), on a planar polygon around each
 *     node (the triangle itself for centroid nodes; the barycentric dual cell projected on the
 *     node's tangent plane for vertex nodes), evaluated with the paper's polar decomposition
 *     into one triangle (O, P, Q) per polygon edge.
 *   - The matrix-vector product of the 6N system, Eqs. (2.9)-(2.12): for every node the
 *     background-domain equation (3 rows) and its scatterer's equation (3 rows), all source
 *     nodes of that domain summed directly with the one-point rule, plus the analytic self
 *     block.  The background domain uses the normal n0 = -n (outward from Omega_0) and the
 *     unknown n0 x curl E = -Psi (Psi is stored with the scatterer normal).
 *   - The transposed product A^T x of the same operator (complex bilinear transpose, no
 *     conjugation), gathered column by column from the transposed pair and self blocks.
 *   - Optionally (radius rho > 0; rho = 0 is the paper's operator), a near-singular correction:
 *     a source node beta within R < rho sqrt(w_beta) of the target contributes the integral of
 *     the pair kernel over its patch, with its density and normal held constant, instead of the
 *     one-point term of Eq. (2.8); the patch is the triangle (centroid nodes) or the unprojected
 *     barycentric dual cell (vertex nodes), each flat piece split L times into four by its edge
 *     midpoints and integrated with the centroid rule.
 *   - The block-diagonal right preconditioner M = A_self of Eq. (3.2) (6x6 per node) and its
 *     exact application by Gaussian elimination with partial pivoting.
 *   - Right-preconditioned restarted GMRES, Eq. (3.1), with modified Gram-Schmidt and Givens
 *     rotations; convergence is judged on the true residual ||b - A x|| / ||b||.
 *   - Plane-wave right-hand sides (incident field at the nodes in the background rows, zero in
 *     the scatterer rows, Eq. (2.12) Phi_inc) and the far-field amplitude of the scattered field
 *     from the representation formula of Eqs. (A.4)/(A.8).
 *   - The impedance-boundary-condition variant of Section 2.3: the 3N operator of Eq. (2.25)
 *     (background equation with n0 x curl E_0 replaced through Eq. (2.24)), its 3x3 self blocks,
 *     and the Psi that Eq. (2.24) implies for a given E_0.
 *
 * Layout of every vector: [n_rhs][N][6] complex128 (re, im interleaved), the 6 entries of a node
 * being (Phi_x, Phi_y, Phi_z, Psi_x, Psi_y, Psi_z) for unknowns and (background-domain x,y,z,
 * scatterer-domain x,y,z) for results.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

static const double PI = 3.14159265358979323846;

typedef struct {
    int64_t N;
    int mode;                /* 0 vertex nodes, 1 centroid nodes */
    int J;                   /* number of scatterers */
    double *s, *n, *w;       /* [N][3], [N][3], [N] */
    int32_t *dom;            /* [N], 1..J */
    double *I1, *S, *V1, *V3;/* self-patch integrals: [N], [N], [N][3], [N][3] */
    cplx *eps, *mu, *k, *gam;/* [J+1] */
    double k0;
    cplx *Sg;                /* [N][2]: self integral of g for (background, own scatterer) */
    cplx *Sdg;               /* [N][2][3]: self integral of grad' g */
    cplx *M;                 /* [N][6][6] preconditioner blocks, row-major */
    /* near-singular correction (off while ns_rho == 0): the flat pieces of each node's patch,
     * pieces pc_beg[a] .. pc_beg[a+1]-1, 9 doubles (three corners) each */
    double ns_rho;
    int ns_L;
    int64_t *pc_beg;
    double *pc_tri;
    char err[256];
} oracle_ctx;

/* ------------------------------------------------------------------------------------------ */
/* small vector helpers                                                                         */
static inline void sub3(const double *a, const double *b, double *o) { o[0]=a[0]-b[0]; o[1]=a[1]-b[1]; o[2]=a[2]-b[2]; }
static inline double dot3(const double *a, const double *b) { return a[0]*b[0]+a[1]*b[1]+a[2]*b[2]; }
static inline void cross3(const double *a, const double *b, double *o) {
    o[0]=a[1]*b[2]-a[2]*b[1]; o[1]=a[2]*b[0]-a[0]*b[2]; o[2]=a[0]*b[1]-a[1]*b[0];
}
static inline double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* k = k0 sqrt(eps mu), the root with non-negative imaginary part (decaying waves for the
 * exp(-i omega t) convention of Section 2.1). */
static cplx wavenumber(double k0, cplx eps, cplx mu) {
    cplx r = csqrt(eps * mu);
    if (cimag(r) < 0.0 || (cimag(r) == 0.0 && creal(r) < 0.0)) r = -r;
    return k0 * r;
}

/* ------------------------------------------------------------------------------------------ */
/* Appendix B: integrals over a planar polygon around O, split into one triangle (O,P,Q) per   */
/* edge; the polar angle phi is measured from the foot D of the perpendicular from O onto the  */
/* edge line (unit vector i = OD/|OD|, j = n x i), as in Eq. (B.1).                             */
/*   Eq. (B.3):  int dA/rho            = sum |OD| ln[tan(pi/4+phi_Q/2) / tan(pi/4+phi_P/2)]    */
/*   Eq. (B.5):  int r/r dA            = sum |OD|/2 [ ln(..) OD + (sec phi_Q - sec phi_P) n x OD]*/
/*   Eq. (B.9):  CPV int r/r^3 dA      = sum OD/|OD| ln[tan(pi/4-phi_Q/2) / tan(pi/4-phi_P/2)]  */
/* plus the polygon area.  p, q are the edge end points relative to O, already in the plane.  */
static void edge_triangle(const double *p, const double *q, const double *nrm,
                          double *I1, double *S, double *V1, double *V3) {
    double e[3]; sub3(q, p, e);
    double ee = dot3(e, e);
    if (ee <= 0.0) return;
    double tpar = -dot3(p, e) / ee;
    double D[3] = {p[0] + tpar * e[0], p[1] + tpar * e[1], p[2] + tpar * e[2]};
    double h = norm3(D);
    if (h <= 1e-300) return;
    double iv[3] = {D[0] / h, D[1] / h, D[2] / h};
    double jv[3]; cross3(nrm, iv, jv);
    double phiP = atan2(dot3(p, jv), dot3(p, iv));
    double phiQ = atan2(dot3(q, jv), dot3(q, iv));
    double lnP = log(tan(PI / 4 + phiP / 2)), lnQ = log(tan(PI / 4 + phiQ / 2));
    double L = lnQ - lnP;                                  /* Eq. (B.3) log ratio */
    *I1 += h * L;
    *S += 0.5 * h * h * (tan(phiQ) - tan(phiP));
    double dsec = 1.0 / cos(phiQ) - 1.0 / cos(phiP);
    for (int c = 0; c < 3; ++c) {
        V1[c] += 0.5 * h * (L * h * iv[c] + dsec * h * jv[c]);
        /* ln[tan(pi/4 - phi_Q/2)/tan(pi/4 - phi_P/2)] = -(lnQ - lnP) */
        V3[c] += iv[c] * (log(tan(PI / 4 - phiQ / 2)) - log(tan(PI / 4 - phiP / 2)));
    }
}

static void project_rel(const double *P, const double *O, const double *nrm, double *out) {
    double d[3]; sub3(P, O, d);
    double a = dot3(d, nrm);
    out[0] = d[0] - a * nrm[0]; out[1] = d[1] - a * nrm[1]; out[2] = d[2] - a * nrm[2];
}

/* ------------------------------------------------------------------------------------------ */
/* nodes (Eq. 2.8) and self-patch integrals                                                    */
static int build_nodes(oracle_ctx *c, int64_t nv, const double *V, int64_t nt, const int32_t *F,
                       const int32_t *td) {
    for (int64_t t = 0; t < nt; ++t) {
        for (int a = 0; a < 3; ++a)
            if (F[3 * t + a] < 0 || F[3 * t + a] >= nv) { snprintf(c->err, sizeof c->err, "triangle %lld: vertex index out of range", (long long)t); return -1; }
        if (td[t] < 1 || td[t] > c->J) { snprintf(c->err, sizeof c->err, "triangle %lld: domain id out of range", (long long)t); return -1; }
    }
    if (c->mode == 1) {
        c->N = nt;
    } else {
        c->N = nv;
    }
    int64_t N = c->N;
    c->s = calloc(3 * N, sizeof(double)); c->n = calloc(3 * N, sizeof(double));
    c->w = calloc(N, sizeof(double)); c->dom = calloc(N, sizeof(int32_t));
    c->I1 = calloc(N, sizeof(double)); c->S = calloc(N, sizeof(double));
    c->V1 = calloc(3 * N, sizeof(double)); c->V3 = calloc(3 * N, sizeof(double));
    if (c->mode == 1) {
        for (int64_t t = 0; t < nt; ++t) {
            const double *A = V + 3 * F[3 * t], *B = V + 3 * F[3 * t + 1], *C = V + 3 * F[3 * t + 2];
            double ab[3], ac[3], cr[3]; sub3(B, A, ab); sub3(C, A, ac); cross3(ab, ac, cr);
            double a2 = norm3(cr);
            if (a2 <= 0.0) { snprintf(c->err, sizeof c->err, "triangle %lld is degenerate", (long long)t); return -1; }
            for (int k = 0; k < 3; ++k) { c->s[3 * t + k] = (A[k] + B[k] + C[k]) / 3.0; c->n[3 * t + k] = cr[k] / a2; }
            c->w[t] = 0.5 * a2;
            c->dom[t] = td[t];
            /* self patch: the triangle itself, edges A->B->C->A relative to the centroid */
            double p[3], q[3], r[3], V1[3] = {0, 0, 0}, V3[3] = {0, 0, 0}, I1 = 0, S = 0;
            const double *O = c->s + 3 * t, *nn = c->n + 3 * t;
            project_rel(A, O, nn, p); project_rel(B, O, nn, q); project_rel(C, O, nn, r);
            edge_triangle(p, q, nn, &I1, &S, V1, V3);
            edge_triangle(q, r, nn, &I1, &S, V1, V3);
            edge_triangle(r, p, nn, &I1, &S, V1, V3);
            c->I1[t] = I1; c->S[t] = S;
            for (int k = 0; k < 3; ++k) { c->V1[3 * t + k] = V1[k]; c->V3[3 * t + k] = V3[k]; }
        }
        return 0;
    }
    /* vertex nodes: w = 1/3 sum of incident areas, n = normalised sum of (B-A)x(C-A) */
    for (int64_t i = 0; i < N; ++i) c->dom[i] = 0;
    for (int64_t t = 0; t < nt; ++t) {
        const double *A = V + 3 * F[3 * t], *B = V + 3 * F[3 * t + 1], *C = V + 3 * F[3 * t + 2];
        double ab[3], ac[3], cr[3]; sub3(B, A, ab); sub3(C, A, ac); cross3(ab, ac, cr);
        double a2 = norm3(cr);
        if (a2 <= 0.0) { snprintf(c->err, sizeof c->err, "triangle %lld is degenerate", (long long)t); return -1; }
        for (int a = 0; a < 3; ++a) {
            int32_t v = F[3 * t + a];
            c->w[v] += a2 / 6.0;
            for (int k = 0; k < 3; ++k) c->n[3 * v + k] += cr[k];
            if (c->dom[v] == 0) c->dom[v] = td[t];
            else if (c->dom[v] != td[t]) { snprintf(c->err, sizeof c->err, "vertex %d touches two scatterers", v); return -1; }
        }
    }
    for (int64_t i = 0; i < N; ++i) {
        if (c->dom[i] == 0) { snprintf(c->err, sizeof c->err, "vertex %lld is not used by any triangle", (long long)i); return -1; }
        double l = norm3(c->n + 3 * i);
        for (int k = 0; k < 3; ++k) { c->n[3 * i + k] /= l; c->s[3 * i + k] = V[3 * i + k]; }
    }
    /* self patch of a vertex: for each incident triangle (A = the vertex, B, C in the
     * triangle's counter-clockwise order) the dual-cell boundary runs mid(AB) -> centroid ->
     * mid(AC); all pieces are projected on the tangent plane of the vertex normal. */
    for (int64_t t = 0; t < nt; ++t) {
        for (int a = 0; a < 3; ++a) {
            int32_t v = F[3 * t + a];
            const double *A = V + 3 * F[3 * t + a], *B = V + 3 * F[3 * t + (a + 1) % 3], *C = V + 3 * F[3 * t + (a + 2) % 3];
            double mab[3], g[3], mac[3];
            for (int k = 0; k < 3; ++k) { mab[k] = 0.5 * (A[k] + B[k]); mac[k] = 0.5 * (A[k] + C[k]); g[k] = (A[k] + B[k] + C[k]) / 3.0; }
            const double *nn = c->n + 3 * v;
            double p[3], q[3], r[3];
            project_rel(mab, A, nn, p); project_rel(g, A, nn, q); project_rel(mac, A, nn, r);
            edge_triangle(p, q, nn, c->I1 + v, c->S + v, c->V1 + 3 * v, c->V3 + 3 * v);
            edge_triangle(q, r, nn, c->I1 + v, c->S + v, c->V1 + 3 * v, c->V3 + 3 * v);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* near-singular correction (reading of the option "near_singular_radius"; the paper itself uses
 * the one-point rule of Eq. (2.8) for every pair beta != alpha).  The patch of a node is the part
 * of the surface its one-point weight stands for: the triangle itself for centroid nodes; for a
 * vertex node the barycentric dual cell, i.e. in every incident triangle (A = the vertex, B, C)
 * the quadrilateral A -> mid(AB) -> centroid -> mid(AC), taken as the two flat pieces
 * (A, mid(AB), G) and (A, G, mid(AC)) on the triangle itself (not projected).  Their areas add up
 * to one third of every incident triangle, i.e. exactly to the node weight w.                */
static void build_patches(oracle_ctx *c, int64_t nv, const double *V, int64_t nt, const int32_t *F) {
    const int64_t N = c->N;
    c->pc_beg = calloc(N + 1, sizeof(int64_t));
    if (c->mode == 1) {
        c->pc_tri = malloc(sizeof(double) * 9 * nt);
        for (int64_t t = 0; t < nt; ++t) {
            c->pc_beg[t + 1] = t + 1;
            for (int a = 0; a < 3; ++a)
                for (int k = 0; k < 3; ++k) c->pc_tri[9 * t + 3 * a + k] = V[3 * F[3 * t + a] + k];
        }
        return;
    }
    (void)nv;
    for (int64_t t = 0; t < nt; ++t)
        for (int a = 0; a < 3; ++a) c->pc_beg[F[3 * t + a] + 1] += 2;
    for (int64_t i = 0; i < N; ++i) c->pc_beg[i + 1] += c->pc_beg[i];
    c->pc_tri = malloc(sizeof(double) * 9 * c->pc_beg[N]);
    int64_t *fill = calloc(N, sizeof(int64_t));
    for (int64_t t = 0; t < nt; ++t) {
        for (int a = 0; a < 3; ++a) {
            const int32_t v = F[3 * t + a];
            const double *A = V + 3 * F[3 * t + a], *B = V + 3 * F[3 * t + (a + 1) % 3], *C = V + 3 * F[3 * t + (a + 2) % 3];
            double mab[3], g[3], mac[3];
            for (int k = 0; k < 3; ++k) { mab[k] = 0.5 * (A[k] + B[k]); mac[k] = 0.5 * (A[k] + C[k]); g[k] = (A[k] + B[k] + C[k]) / 3.0; }
            double *p1 = c->pc_tri + 9 * (c->pc_beg[v] + fill[v]++);
            double *p2 = c->pc_tri + 9 * (c->pc_beg[v] + fill[v]++);
            for (int k = 0; k < 3; ++k) {
                p1[k] = A[k]; p1[3 + k] = mab[k]; p1[6 + k] = g[k];
                p2[k] = A[k]; p2[3 + k] = g[k]; p2[6 + k] = mac[k];
            }
        }
    }
    free(fill);
}

/* int g dA' and int grad' g dA' over the triangle (P0, P1, P2) seen from the point sa, with
 * g = exp(i k R)/(4 pi R), R = |s' - sa|, grad' g = g (i k - 1/R) (s' - sa)/R: the triangle is
 * split into four by its edge midpoints L times, and each of the 4^L pieces contributes its area
 * times the integrand at its centroid. */
static void piece_integral(const double *P0, const double *P1, const double *P2, int L, const double *sa, cplx k,
                           cplx *G, cplx *A) {
    if (L > 0) {
        double m01[3], m12[3], m20[3];
        for (int q = 0; q < 3; ++q) {
            m01[q] = 0.5 * (P0[q] + P1[q]);
            m12[q] = 0.5 * (P1[q] + P2[q]);
            m20[q] = 0.5 * (P2[q] + P0[q]);
        }
        piece_integral(P0, m01, m20, L - 1, sa, k, G, A);
        piece_integral(m01, P1, m12, L - 1, sa, k, G, A);
        piece_integral(m20, m12, P2, L - 1, sa, k, G, A);
        piece_integral(m12, m20, m01, L - 1, sa, k, G, A);
        return;
    }
    double e1[3], e2[3], cr[3], r[3];
    sub3(P1, P0, e1); sub3(P2, P0, e2); cross3(e1, e2, cr);
    const double area = 0.5 * norm3(cr);
    for (int q = 0; q < 3; ++q) r[q] = (P0[q] + P1[q] + P2[q]) / 3.0 - sa[q];
    const double R = norm3(r);
    const cplx g = cexp(I * k * R) / (4 * PI * R);
    const cplx cc = g * (I * k - 1.0 / R) / R;
    *G += area * g;
    for (int q = 0; q < 3; ++q) A[q] += area * cc * r[q];
}

/* the patch integrals of node b seen from sa, summed over its pieces */
static void patch_integral(const oracle_ctx *c, int64_t b, const double *sa, cplx k, int L, cplx *G, cplx *A) {
    *G = 0;
    A[0] = A[1] = A[2] = 0;
    for (int64_t p = c->pc_beg[b]; p < c->pc_beg[b + 1]; ++p) {
        const double *T = c->pc_tri + 9 * p;
        piece_integral(T, T + 3, T + 6, L, sa, k, G, A);
    }
}

/* does source b take its patch integral instead of the one-point rule for target distance R? */
static inline int near_singular(const oracle_ctx *c, int64_t b, double R) {
    return c->ns_rho > 0 && R < c->ns_rho * sqrt(c->w[b]);
}

void oracle_set_near_singular(oracle_ctx *c, double rho, int levels) {
    c->ns_rho = rho;
    c->ns_L = levels;
}

/* int g dA' (out[0..1]) and int grad' g dA' (out[2..7]) over node b's patch from the point pt,
 * wavenumber (kre, kim), L subdivision levels */
void oracle_patch_integral(const oracle_ctx *c, int64_t b, const double *pt, double kre, double kim, int L,
                           double *out) {
    cplx G, A[3];
    patch_integral(c, b, pt, kre + I * kim, L, &G, A);
    out[0] = creal(G); out[1] = cimag(G);
    for (int q = 0; q < 3; ++q) { out[2 + 2 * q] = creal(A[q]); out[3 + 2 * q] = cimag(A[q]); }
}

/* Self integrals of g and grad' g over the patch with the paper's Taylor truncations:
 * Eq. (B.2)  int g dA      ~ (I1 + i k S) / (4 pi)
 * Eq. (B.4)  int grad g dA ~ -k^2/(8 pi) int r/r dA - 1/(4 pi) CPV int r/r^3 dA             */
static void self_terms(oracle_ctx *c) {
    int64_t N = c->N;
    c->Sg = malloc(sizeof(cplx) * 2 * N);
    c->Sdg = malloc(sizeof(cplx) * 6 * N);
    for (int64_t a = 0; a < N; ++a) {
        for (int side = 0; side < 2; ++side) {
            cplx k = side == 0 ? c->k[0] : c->k[c->dom[a]];
            c->Sg[2 * a + side] = (c->I1[a] + I * k * c->S[a]) / (4 * PI);
            for (int q = 0; q < 3; ++q)
                c->Sdg[6 * a + 3 * side + q] = -(k * k) / (8 * PI) * c->V1[3 * a + q] - c->V3[3 * a + q] / (4 * PI);
        }
    }
}

/* [n a^T - (n.a) I - a n^T] . v  (complex bilinear), the bracket of Eq. (2.12) with a = grad'g */
static inline void bracket(const double *nn, const cplx *a, const cplx *v, cplx *out) {
    cplx av = a[0] * v[0] + a[1] * v[1] + a[2] * v[2];
    cplx na = nn[0] * a[0] + nn[1] * a[1] + nn[2] * a[2];
    cplx nv = nn[0] * v[0] + nn[1] * v[1] + nn[2] * v[2];
    for (int q = 0; q < 3; ++q) out[q] = nn[q] * av - na * v[q] - a[q] * nv;
}

/* T_d v for the node's normal (Eq. 2.13); d = 0 is the identity */
static inline void apply_T(const oracle_ctx *c, int d, const double *nn, const cplx *v, cplx *o) {
    if (d == 0) { o[0] = v[0]; o[1] = v[1]; o[2] = v[2]; return; }
    cplx t = (c->eps[0] - c->eps[d]) / c->eps[d];
    cplx nv = nn[0] * v[0] + nn[1] * v[1] + nn[2] * v[2];
    for (int q = 0; q < 3; ++q) o[q] = v[q] + t * nn[q] * nv;
}

/* 6x6 preconditioner block of node a: the self part of both equations, Eq. (3.2) A_self */
static void build_precond(oracle_ctx *c) {
    int64_t N = c->N;
    c->M = calloc(36 * N, sizeof(cplx));
    for (int64_t a = 0; a < N; ++a) {
        cplx *M = c->M + 36 * a;
        int j = c->dom[a];
        for (int col = 0; col < 3; ++col) {
            cplx e[3] = {0, 0, 0}; e[col] = 1.0;
            for (int side = 0; side < 2; ++side) {
                int d = side == 0 ? 0 : j;
                double nd[3]; for (int q = 0; q < 3; ++q) nd[q] = (side == 0 ? -1.0 : 1.0) * c->n[3 * a + q];
                cplx Te[3], B[3];
                apply_T(c, d, c->n + 3 * a, e, Te);
                bracket(nd, c->Sdg + 6 * a + 3 * side, Te, B);
                for (int q = 0; q < 3; ++q) M[(3 * side + q) * 6 + col] = 0.5 * Te[q] - B[q];
            }
        }
        for (int q = 0; q < 3; ++q) {
            M[q * 6 + 3 + q] = -c->gam[0] * c->Sg[2 * a];                 /* background: Psi0 = -Psi */
            M[(3 + q) * 6 + 3 + q] = c->gam[j] * c->Sg[2 * a + 1];
        }
    }
}

/* ------------------------------------------------------------------------------------------ */
oracle_ctx *oracle_create(int mode, int64_t nv, const double *V, int64_t nt, const int32_t *F, const int32_t *td,
                          int J, const double *eps, const double *mu, double k0, char *errbuf, int errlen) {
    oracle_ctx *c = calloc(1, sizeof(oracle_ctx));
    c->mode = mode; c->J = J; c->k0 = k0;
    c->eps = malloc(sizeof(cplx) * (J + 1)); c->mu = malloc(sizeof(cplx) * (J + 1));
    c->k = malloc(sizeof(cplx) * (J + 1)); c->gam = malloc(sizeof(cplx) * (J + 1));
    for (int d = 0; d <= J; ++d) {
        c->eps[d] = eps[2 * d] + I * eps[2 * d + 1];
        c->mu[d] = mu[2 * d] + I * mu[2 * d + 1];
        c->k[d] = wavenumber(k0, c->eps[d], c->mu[d]);
        c->gam[d] = d == 0 ? 1.0 : c->mu[d] / c->mu[0];
    }
    if (build_nodes(c, nv, V, nt, F, td) != 0) {
        if (errbuf) snprintf(errbuf, errlen, "%s", c->err);
        return NULL;  /* leaks on the error path; test infrastructure */
    }
    build_patches(c, nv, V, nt, F);
    self_terms(c);
    build_precond(c);
    return c;
}

void oracle_destroy(oracle_ctx *c) {
    if (!c) return;
    free(c->s); free(c->n); free(c->w); free(c->dom); free(c->I1); free(c->S); free(c->V1); free(c->V3);
    free(c->eps); free(c->mu); free(c->k); free(c->gam); free(c->Sg); free(c->Sdg); free(c->M);
    free(c->pc_beg); free(c->pc_tri);
    free(c);
}

int64_t oracle_num_nodes(const oracle_ctx *c) { return c->N; }

void oracle_geometry(const oracle_ctx *c, double *s, double *n, double *w, int32_t *dom,
                     double *I1, double *S, double *V1, double *V3) {
    int64_t N = c->N;
    if (s) memcpy(s, c->s, 3 * N * sizeof(double));
    if (n) memcpy(n, c->n, 3 * N * sizeof(double));
    if (w) memcpy(w, c->w, N * sizeof(double));
    if (dom) memcpy(dom, c->dom, N * sizeof(int32_t));
    if (I1) memcpy(I1, c->I1, N * sizeof(double));
    if (S) memcpy(S, c->S, N * sizeof(double));
    if (V1) memcpy(V1, c->V1, 3 * N * sizeof(double));
    if (V3) memcpy(V3, c->V3, 3 * N * sizeof(double));
}

void oracle_wavenumbers(const oracle_ctx *c, double *k) {
    for (int d = 0; d <= c->J; ++d) { k[2 * d] = creal(c->k[d]); k[2 * d + 1] = cimag(c->k[d]); }
}

void oracle_precond_blocks(const oracle_ctx *c, double *M) { memcpy(M, c->M, 36 * c->N * sizeof(cplx)); }

/* Eq. (2.12)/(2.22)-(2.23) without the multipole split: result rows of node a for all RHS.
 * x: [n_rhs][N][6], out: [n_rhs][6] for this node. */
static void node_rows(const oracle_ctx *c, int64_t a, int64_t n_rhs, const cplx *x, cplx *out) {
    const int64_t N = c->N;
    const int j = c->dom[a];
    const double *sa = c->s + 3 * a;
    const cplx k0 = c->k[0], kj = c->k[j], gj = c->gam[j];
    for (int64_t r = 0; r < n_rhs * 6; ++r) out[r] = 0;
    for (int64_t b = 0; b < N; ++b) {
        if (b == a) continue;
        double rv[3]; sub3(c->s + 3 * b, sa, rv);            /* r = s_beta - s_alpha */
        double R = norm3(rv);
        const double wb = c->w[b];
        const double *nb = c->n + 3 * b;
        double n0[3] = {-nb[0], -nb[1], -nb[2]};
        if (near_singular(c, b, R)) {
            /* the patch integrals of g and grad' g replace w_b g and w_b grad' g (the density of
             * node b and its normal held constant over the patch, so the bracket of Eq. (2.12)
             * takes the integrated gradient) */
            cplx G0, A0[3], Gj = 0, Aj[3] = {0, 0, 0};
            patch_integral(c, b, sa, k0, c->ns_L, &G0, A0);
            const int same_ns = c->dom[b] == j;
            if (same_ns) patch_integral(c, b, sa, kj, c->ns_L, &Gj, Aj);
            for (int64_t r = 0; r < n_rhs; ++r) {
                const cplx *xb = x + (r * N + b) * 6;
                cplx B[3];
                bracket(n0, A0, xb, B);
                for (int q = 0; q < 3; ++q) out[6 * r + q] += -B[q] + G0 * (-xb[3 + q]);
                if (same_ns) {
                    cplx Tv[3];
                    apply_T(c, j, nb, xb, Tv);
                    bracket(nb, Aj, Tv, B);
                    for (int q = 0; q < 3; ++q) out[6 * r + 3 + q] += -B[q] + gj * Gj * xb[3 + q];
                }
            }
            continue;
        }
        /* background domain: every node is a source */
        cplx g0 = cexp(I * k0 * R) / (4 * PI * R);
        cplx c0 = g0 * (I * k0 - 1.0 / R) / R;                /* grad' g = c0 r */
        cplx a0[3] = {c0 * rv[0], c0 * rv[1], c0 * rv[2]};
        int same = c->dom[b] == j;
        cplx gj_ = 0, aj[3] = {0, 0, 0};
        if (same) {
            gj_ = cexp(I * kj * R) / (4 * PI * R);
            cplx cj = gj_ * (I * kj - 1.0 / R) / R;
            aj[0] = cj * rv[0]; aj[1] = cj * rv[1]; aj[2] = cj * rv[2];
        }
        for (int64_t r = 0; r < n_rhs; ++r) {
            const cplx *xb = x + (r * N + b) * 6;
            cplx B[3];
            bracket(n0, a0, xb, B);
            for (int q = 0; q < 3; ++q) out[6 * r + q] += -wb * B[q] + wb * g0 * (-xb[3 + q]);
            if (same) {
                cplx Tv[3];
                apply_T(c, j, nb, xb, Tv);
                bracket(nb, aj, Tv, B);
                for (int q = 0; q < 3; ++q) out[6 * r + 3 + q] += -wb * B[q] + gj * wb * gj_ * xb[3 + q];
            }
        }
    }
    /* self block (delta_{alpha beta} terms and the analytic patch integrals) */
    const cplx *M = c->M + 36 * a;
    for (int64_t r = 0; r < n_rhs; ++r) {
        const cplx *xa = x + (r * N + a) * 6;
        for (int q = 0; q < 6; ++q) {
            cplx acc = 0;
            for (int p = 0; p < 6; ++p) acc += M[q * 6 + p] * xa[p];
            out[6 * r + q] += acc;
        }
    }
}

/* The transpose A^T (complex bilinear, no conjugation) applied to x: the result at column node b
 * gathers, over every row node a != b, the transposed 6x6 block of node_rows' pair term, and the
 * transposed self block.  With the bracket matrix Bk(n, a) v = n (a.v) - (n.a) v - a (n.v) of
 * Eq. (2.12), Bk(n, a)^T u = a (n.u) - (n.a) u - n (a.u), and T_j is symmetric.  x: [n_rhs][N][6],
 * out: [n_rhs][6] for node b. */
static inline void bracket_t(const double *nn, const cplx *a, const cplx *u, cplx *out) {
    cplx nu = nn[0] * u[0] + nn[1] * u[1] + nn[2] * u[2];
    cplx na = nn[0] * a[0] + nn[1] * a[1] + nn[2] * a[2];
    cplx au = a[0] * u[0] + a[1] * u[1] + a[2] * u[2];
    for (int q = 0; q < 3; ++q) out[q] = a[q] * nu - na * u[q] - nn[q] * au;
}
static void node_cols(const oracle_ctx *c, int64_t b, int64_t n_rhs, const cplx *x, cplx *out) {
    const int64_t N = c->N;
    const int j = c->dom[b];
    const double *sb = c->s + 3 * b;
    const double wb = c->w[b];
    const double *nb = c->n + 3 * b;
    const double n0[3] = {-nb[0], -nb[1], -nb[2]};
    const cplx k0 = c->k[0], kj = c->k[j], gj = c->gam[j];
    for (int64_t r = 0; r < n_rhs * 6; ++r) out[r] = 0;
    for (int64_t a = 0; a < N; ++a) {
        if (a == b) continue;
        double rv[3]; sub3(sb, c->s + 3 * a, rv);            /* r = s_beta - s_alpha, as in node_rows */
        double R = norm3(rv);
        if (near_singular(c, b, R)) {
            /* transposed patch-integral blocks of node_rows' near-singular branch */
            cplx G0, A0[3], Gj = 0, Aj[3] = {0, 0, 0};
            patch_integral(c, b, c->s + 3 * a, k0, c->ns_L, &G0, A0);
            const int same_ns = c->dom[a] == j;
            if (same_ns) patch_integral(c, b, c->s + 3 * a, kj, c->ns_L, &Gj, Aj);
            for (int64_t r = 0; r < n_rhs; ++r) {
                const cplx *xa = x + (r * N + a) * 6;
                cplx B[3];
                bracket_t(n0, A0, xa, B);
                for (int q = 0; q < 3; ++q) {
                    out[6 * r + q] += -B[q];
                    out[6 * r + 3 + q] += -G0 * xa[q];
                }
                if (same_ns) {
                    cplx TB[3];
                    bracket_t(nb, Aj, xa + 3, B);
                    apply_T(c, j, nb, B, TB);
                    for (int q = 0; q < 3; ++q) {
                        out[6 * r + q] += -TB[q];
                        out[6 * r + 3 + q] += gj * Gj * xa[3 + q];
                    }
                }
            }
            continue;
        }
        cplx g0 = cexp(I * k0 * R) / (4 * PI * R);
        cplx c0 = g0 * (I * k0 - 1.0 / R) / R;
        cplx a0[3] = {c0 * rv[0], c0 * rv[1], c0 * rv[2]};
        int same = c->dom[a] == j;
        cplx gj_ = 0, aj[3] = {0, 0, 0};
        if (same) {
            gj_ = cexp(I * kj * R) / (4 * PI * R);
            cplx cj = gj_ * (I * kj - 1.0 / R) / R;
            aj[0] = cj * rv[0]; aj[1] = cj * rv[1]; aj[2] = cj * rv[2];
        }
        for (int64_t r = 0; r < n_rhs; ++r) {
            const cplx *xa = x + (r * N + a) * 6;
            cplx B[3];
            /* background rows of node a: blocks -w_b Bk(n0_b, a0) (Phi) and -w_b g0 I (Psi) */
            bracket_t(n0, a0, xa, B);
            for (int q = 0; q < 3; ++q) {
                out[6 * r + q] += -wb * B[q];
                out[6 * r + 3 + q] += -wb * g0 * xa[q];
            }
            if (same) {
                /* scatterer rows: blocks -w_b Bk(n_b, aj) T_j(b) (Phi) and gamma_j w_b gj I (Psi) */
                cplx TB[3];
                bracket_t(nb, aj, xa + 3, B);
                apply_T(c, j, nb, B, TB);
                for (int q = 0; q < 3; ++q) {
                    out[6 * r + q] += -wb * TB[q];
                    out[6 * r + 3 + q] += gj * wb * gj_ * xa[3 + q];
                }
            }
        }
    }
    const cplx *M = c->M + 36 * b;
    for (int64_t r = 0; r < n_rhs; ++r) {
        const cplx *xb = x + (r * N + b) * 6;
        for (int p = 0; p < 6; ++p) {
            cplx acc = 0;
            for (int q = 0; q < 6; ++q) acc += M[q * 6 + p] * xb[q];
            out[6 * r + p] += acc;
        }
    }
}

/* y = A^T x, x and y [n_rhs][N][6] complex */
void oracle_matvec_transpose(const oracle_ctx *c, int64_t n_rhs, const double *x_, double *y_) {
    const cplx *x = (const cplx *)x_;
    cplx *y = (cplx *)y_;
    const int64_t N = c->N;
#pragma omp parallel
    {
        cplx *buf = malloc(sizeof(cplx) * 6 * n_rhs);
#pragma omp for schedule(dynamic, 8)
        for (int64_t b = 0; b < N; ++b) {
            node_cols(c, b, n_rhs, x, buf);
            for (int64_t r = 0; r < n_rhs; ++r)
                for (int q = 0; q < 6; ++q) y[(r * N + b) * 6 + q] = buf[6 * r + q];
        }
        free(buf);
    }
}

/* entries of A^T x for a subset of nodes: y [n_rhs][n_rows][6] */
void oracle_matvec_transpose_rows(const oracle_ctx *c, int64_t n_rhs, int64_t n_rows, const int64_t *rows,
                                  const double *x_, double *y_) {
    const cplx *x = (const cplx *)x_;
    cplx *y = (cplx *)y_;
#pragma omp parallel
    {
        cplx *buf = malloc(sizeof(cplx) * 6 * n_rhs);
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < n_rows; ++i) {
            node_cols(c, rows[i], n_rhs, x, buf);
            for (int64_t r = 0; r < n_rhs; ++r)
                for (int q = 0; q < 6; ++q) y[(r * n_rows + i) * 6 + q] = buf[6 * r + q];
        }
        free(buf);
    }
}

/* y = A x, x and y [n_rhs][N][6] complex */
void oracle_matvec(const oracle_ctx *c, int64_t n_rhs, const double *x_, double *y_) {
    const cplx *x = (const cplx *)x_;
    cplx *y = (cplx *)y_;
    const int64_t N = c->N;
#pragma omp parallel
    {
        cplx *buf = malloc(sizeof(cplx) * 6 * n_rhs);
#pragma omp for schedule(dynamic, 8)
        for (int64_t a = 0; a < N; ++a) {
            node_rows(c, a, n_rhs, x, buf);
            for (int64_t r = 0; r < n_rhs; ++r)
                for (int q = 0; q < 6; ++q) y[(r * N + a) * 6 + q] = buf[6 * r + q];
        }
        free(buf);
    }
}

/* rows of A x for a subset of nodes: y [n_rhs][n_rows][6] */
void oracle_matvec_rows(const oracle_ctx *c, int64_t n_rhs, int64_t n_rows, const int64_t *rows,
                        const double *x_, double *y_) {
    const cplx *x = (const cplx *)x_;
    cplx *y = (cplx *)y_;
#pragma omp parallel
    {
        cplx *buf = malloc(sizeof(cplx) * 6 * n_rhs);
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < n_rows; ++i) {
            node_rows(c, rows[i], n_rhs, x, buf);
            for (int64_t r = 0; r < n_rhs; ++r)
                for (int q = 0; q < 6; ++q) y[(r * n_rows + i) * 6 + q] = buf[6 * r + q];
        }
        free(buf);
    }
}

/* solve the 6x6 system M z = v by Gaussian elimination with partial pivoting */
static void solve6(const cplx *M_, const cplx *v, cplx *z) {
    cplx A[6][7];
    for (int i = 0; i < 6; ++i) { for (int j = 0; j < 6; ++j) A[i][j] = M_[i * 6 + j]; A[i][6] = v[i]; }
    for (int col = 0; col < 6; ++col) {
        int piv = col; double best = cabs(A[col][col]);
        for (int i = col + 1; i < 6; ++i) if (cabs(A[i][col]) > best) { best = cabs(A[i][col]); piv = i; }
        if (piv != col) for (int j = 0; j < 7; ++j) { cplx t = A[col][j]; A[col][j] = A[piv][j]; A[piv][j] = t; }
        for (int i = col + 1; i < 6; ++i) {
            cplx f = A[i][col] / A[col][col];
            for (int j = col; j < 7; ++j) A[i][j] -= f * A[col][j];
        }
    }
    for (int i = 5; i >= 0; --i) {
        cplx acc = A[i][6];
        for (int j = i + 1; j < 6; ++j) acc -= A[i][j] * z[j];
        z[i] = acc / A[i][i];
    }
}

/* z = M^-1 v, Eq. (3.1)-(3.2) block-diagonal preconditioner */
void oracle_precond_apply(const oracle_ctx *c, int64_t n_rhs, const double *v_, double *z_) {
    const cplx *v = (const cplx *)v_;
    cplx *z = (cplx *)z_;
    const int64_t N = c->N;
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < N; ++a)
        for (int64_t r = 0; r < n_rhs; ++r) solve6(c->M + 36 * a, v + (r * N + a) * 6, z + (r * N + a) * 6);
}

/* plane waves E_inc = e exp(i k_0 d.s) in the background rows, zero in the scatterer rows */
void oracle_plane_wave_rhs(const oracle_ctx *c, int64_t n_rhs, const double *dirs, const double *pols_, double *b_) {
    const cplx *pols = (const cplx *)pols_;
    cplx *b = (cplx *)b_;
    const int64_t N = c->N;
    for (int64_t r = 0; r < n_rhs; ++r)
        for (int64_t a = 0; a < N; ++a) {
            cplx ph = cexp(I * c->k[0] * dot3(dirs + 3 * r, c->s + 3 * a));
            for (int q = 0; q < 3; ++q) { b[(r * N + a) * 6 + q] = pols[3 * r + q] * ph; b[(r * N + a) * 6 + 3 + q] = 0; }
        }
}

/* ------------------------------------------------------------------------------------------ */
/* right-preconditioned restarted GMRES, Eq. (3.1), one right-hand side                        */
static double vnorm(const cplx *v, int64_t n) {
    double s = 0;
    for (int64_t i = 0; i < n; ++i) s += creal(v[i]) * creal(v[i]) + cimag(v[i]) * cimag(v[i]);
    return sqrt(s);
}

static cplx vdot(const cplx *a, const cplx *b, int64_t n) {   /* sum conj(a) b */
    cplx s = 0;
    for (int64_t i = 0; i < n; ++i) s += conj(a[i]) * b[i];
    return s;
}

int oracle_gmres(const oracle_ctx *c, const double *b_, double *x_, double tol, int restart, int max_iter,
                 int use_precond, int *iters_out, double *relres_out) {
    const int64_t n = 6 * c->N;
    const cplx *b = (const cplx *)b_;
    cplx *x = (cplx *)x_;
    const int m = restart;
    cplx *Vb = malloc(sizeof(cplx) * n * (m + 1));
    cplx *z = malloc(sizeof(cplx) * n), *w = malloc(sizeof(cplx) * n), *r = malloc(sizeof(cplx) * n);
    cplx *H = calloc((m + 1) * m, sizeof(cplx));
    cplx *cs = malloc(sizeof(cplx) * m), *sn = malloc(sizeof(cplx) * m), *g = malloc(sizeof(cplx) * (m + 1));
    cplx *yv = malloc(sizeof(cplx) * m);
    double bn = vnorm(b, n);
    int it = 0, status = 1;
    double rel = 1.0;
    if (bn == 0.0) { memset(x, 0, sizeof(cplx) * n); *iters_out = 0; *relres_out = 0; status = 0; goto done; }
    for (;;) {
        oracle_matvec(c, 1, (const double *)x, (double *)r);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
        double beta = vnorm(r, n);
        rel = beta / bn;
        if (rel <= tol) { status = 0; break; }
        if (it >= max_iter) break;
        for (int64_t i = 0; i < n; ++i) Vb[i] = r[i] / beta;
        for (int i = 0; i <= m; ++i) g[i] = 0;
        g[0] = beta;
        int jdone = 0;
        for (int j = 0; j < m && it < max_iter; ++j) {
            if (use_precond) oracle_precond_apply(c, 1, (const double *)(Vb + j * n), (double *)z);
            else memcpy(z, Vb + j * n, sizeof(cplx) * n);
            oracle_matvec(c, 1, (const double *)z, (double *)w);
            ++it;
            for (int i = 0; i <= j; ++i) {                      /* modified Gram-Schmidt */
                cplx h = vdot(Vb + i * n, w, n);
                H[i * m + j] = h;
                for (int64_t q = 0; q < n; ++q) w[q] -= h * Vb[i * n + q];
            }
            double hn = vnorm(w, n);
            H[(j + 1) * m + j] = hn;
            if (hn > 0) for (int64_t q = 0; q < n; ++q) Vb[(j + 1) * n + q] = w[q] / hn;
            for (int i = 0; i < j; ++i) {                       /* previous Givens rotations */
                cplx t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
                H[(i + 1) * m + j] = -conj(sn[i]) * H[i * m + j] + conj(cs[i]) * H[(i + 1) * m + j];
                H[i * m + j] = t;
            }
            /* new rotation Q = [cs sn; -conj(sn) conj(cs)], cs = conj(a)/d, sn = conj(b)/d,
             * maps (a, b) = (H[j][j], H[j+1][j]) to (d, 0) with d = sqrt(|a|^2 + |b|^2) */
            cplx hjj = H[j * m + j], hj1 = H[(j + 1) * m + j];
            double den = sqrt(creal(hjj) * creal(hjj) + cimag(hjj) * cimag(hjj) + creal(hj1) * creal(hj1) + cimag(hj1) * cimag(hj1));
            if (den == 0) { cs[j] = 1; sn[j] = 0; }
            else { cs[j] = conj(hjj) / den; sn[j] = conj(hj1) / den; }
            H[j * m + j] = cs[j] * hjj + sn[j] * hj1;
            H[(j + 1) * m + j] = 0;
            g[j + 1] = -conj(sn[j]) * g[j];
            g[j] = cs[j] * g[j];
            jdone = j + 1;
            if (cabs(g[j + 1]) / bn <= tol || hn == 0) break;
        }
        for (int i = jdone - 1; i >= 0; --i) {
            cplx acc = g[i];
            for (int q = i + 1; q < jdone; ++q) acc -= H[i * m + q] * yv[q];
            yv[i] = acc / H[i * m + i];
        }
        memset(w, 0, sizeof(cplx) * n);
        for (int i = 0; i < jdone; ++i) for (int64_t q = 0; q < n; ++q) w[q] += yv[i] * Vb[i * n + q];
        if (use_precond) oracle_precond_apply(c, 1, (const double *)w, (double *)z);
        else memcpy(z, w, sizeof(cplx) * n);
        for (int64_t q = 0; q < n; ++q) x[q] += z[q];
    }
    *iters_out = it;
    *relres_out = rel;
done:
    free(Vb); free(z); free(w); free(r); free(H); free(cs); free(sn); free(g); free(yv);
    return status;
}

/* far-field amplitude F(rhat) of the scattered field, E_sca ~ exp(i k0 r)/r F, from the
 * representation formula of Eqs. (A.4)/(A.8) with the background normal n0 = -n and
 * n0 x curl E = -Psi.  x: one solution [N][6]; rhat [nd][3]; F [nd][3] complex. */
void oracle_far_field(const oracle_ctx *c, const double *x_, int64_t nd, const double *rhat, double *F_) {
    const cplx *x = (const cplx *)x_;
    cplx *F = (cplx *)F_;
    const cplx k = c->k[0];
#pragma omp parallel for schedule(static)
    for (int64_t d = 0; d < nd; ++d) {
        const double *u = rhat + 3 * d;
        cplx acc[3] = {0, 0, 0};
        for (int64_t b = 0; b < c->N; ++b) {
            const double *nb = c->n + 3 * b;
            double n0[3] = {-nb[0], -nb[1], -nb[2]};
            const cplx *Phi = x + 6 * b, *Psi = x + 6 * b + 3;
            cplx ph = c->w[b] * cexp(-I * k * dot3(u, c->s + 3 * b));
            cplx uP = u[0] * Phi[0] + u[1] * Phi[1] + u[2] * Phi[2];
            double nu = dot3(n0, u);
            cplx nP = n0[0] * Phi[0] + n0[1] * Phi[1] + n0[2] * Phi[2];
            for (int q = 0; q < 3; ++q)
                acc[q] += ph * ((-I * k) * (n0[q] * uP - nu * Phi[q] - u[q] * nP) + Psi[q]);
        }
        for (int q = 0; q < 3; ++q) F[3 * d + q] = acc[q] / (4 * PI);
    }
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* total field at exterior points r (not on the surface) from the representation formula of
 * Eqs. (A.4)/(A.8) for the background domain:
 *   E(r) = E_inc(r) + sum_b w_b { [n0 (grad'g . Phi) - (n0 . grad'g) Phi - grad'g (n0 . Phi)]
 *                                 - g (n0 x curl E) },  n0 = -n_b, n0 x curl E = -Psi_b,
 * with g = g_0(s_b, r) and grad' taken at the source s_b.  E_inc = e exp(i k0 d.r). */
void oracle_near_field(const oracle_ctx *c, const double *x_, int64_t np_, const double *pts,
                       const double *dir, const double *pol_, double *E_) {
    const cplx *x = (const cplx *)x_;
    const cplx *pol = (const cplx *)pol_;
    cplx *E = (cplx *)E_;
    const cplx k = c->k[0];
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < np_; ++p) {
        const double *r = pts + 3 * p;
        cplx ph = cexp(I * k * dot3(dir, r));
        cplx acc[3] = {pol[0] * ph, pol[1] * ph, pol[2] * ph};
        for (int64_t b = 0; b < c->N; ++b) {
            double rv[3]; sub3(c->s + 3 * b, r, rv);
            double R = norm3(rv);
            const double *nb = c->n + 3 * b;
            double n0[3] = {-nb[0], -nb[1], -nb[2]};
            cplx g = cexp(I * k * R) / (4 * PI * R);
            cplx cc = g * (I * k - 1.0 / R) / R;
            cplx a[3] = {cc * rv[0], cc * rv[1], cc * rv[2]};
            cplx B[3];
            bracket(n0, a, x + 6 * b, B);
            for (int q = 0; q < 3; ++q) acc[q] += c->w[b] * (B[q] + g * x[6 * b + 3 + q]);
        }
        for (int q = 0; q < 3; ++q) E[3 * p + q] = acc[q];
    }
}

/* Total magnetic field at exterior points, H = curl E / (i omega mu_0) with omega = k0 (c = 1)
 * and mu_0 the background's relative permeability, from the curl of the representation formula
 * used by oracle_near_field.  With a = grad_s g = g'(R) rhat (rhat = (s_b - r)/R) and the Hessian
 * K = d^2 g / ds ds = g''(R) rhat rhat^T + g'(R)/R (I - rhat rhat^T),
 * g' = g (i k - 1/R), g'' = g ((i k - 1/R)^2 + 1/R^2), the curl over r of the bracket
 * n0 (a.Phi) - (n0.a) Phi - a (n0.Phi) is (K n0) x Phi + n0 x (K Phi) (curl_r a = 0, d a / d r = -K),
 * and that of g Psi is -a x Psi.  The incident wave e exp(i k d.r) contributes
 * (k / (omega mu_0)) d x e exp(i k d.r). */
void oracle_near_field_h(const oracle_ctx *c, const double *x_, int64_t np_, const double *pts,
                         const double *dir, const double *pol_, double *H_) {
    const cplx *x = (const cplx *)x_;
    const cplx *pol = (const cplx *)pol_;
    cplx *H = (cplx *)H_;
    const cplx k = c->k[0], mu0 = c->mu[0];
    const cplx iwm = I * c->k0 * mu0;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < np_; ++p) {
        const double *r = pts + 3 * p;
        const cplx ph = cexp(I * k * dot3(dir, r));
        cplx curl[3];
        {
            const cplx de[3] = {dir[1] * pol[2] - dir[2] * pol[1], dir[2] * pol[0] - dir[0] * pol[2],
                                dir[0] * pol[1] - dir[1] * pol[0]};
            for (int q = 0; q < 3; ++q) curl[q] = I * k * de[q] * ph;  /* curl of the incident wave */
        }
        for (int64_t b = 0; b < c->N; ++b) {
            double rv[3]; sub3(c->s + 3 * b, r, rv);
            const double R = norm3(rv);
            const double rh[3] = {rv[0] / R, rv[1] / R, rv[2] / R};
            const double *nb = c->n + 3 * b;
            const double n0[3] = {-nb[0], -nb[1], -nb[2]};
            const cplx g = cexp(I * k * R) / (4 * PI * R);
            const cplx g1 = g * (I * k - 1.0 / R);
            const cplx g2 = g * ((I * k - 1.0 / R) * (I * k - 1.0 / R) + 1.0 / (R * R));
            const cplx *Phi = x + 6 * b, *Psi = x + 6 * b + 3;
            /* K v = g'' rhat (rhat.v) + g'/R (v - rhat (rhat.v)) */
            const double rn = dot3(rh, n0);
            const cplx rP = rh[0] * Phi[0] + rh[1] * Phi[1] + rh[2] * Phi[2];
            cplx Kn[3], KP[3], a[3];
            for (int q = 0; q < 3; ++q) {
                Kn[q] = g2 * rh[q] * rn + g1 / R * (n0[q] - rh[q] * rn);
                KP[q] = g2 * rh[q] * rP + g1 / R * (Phi[q] - rh[q] * rP);
                a[q] = g1 * rh[q];
            }
            const cplx t[3] = {Kn[1] * Phi[2] - Kn[2] * Phi[1] + n0[1] * KP[2] - n0[2] * KP[1] - (a[1] * Psi[2] - a[2] * Psi[1]),
                               Kn[2] * Phi[0] - Kn[0] * Phi[2] + n0[2] * KP[0] - n0[0] * KP[2] - (a[2] * Psi[0] - a[0] * Psi[2]),
                               Kn[0] * Phi[1] - Kn[1] * Phi[0] + n0[0] * KP[1] - n0[1] * KP[0] - (a[0] * Psi[1] - a[1] * Psi[0])};
            for (int q = 0; q < 3; ++q) curl[q] += c->w[b] * t[q];
        }
        for (int q = 0; q < 3; ++q) H[3 * p + q] = curl[q] / iwm;
    }
}

/* Appendix B integrals over an arbitrary planar polygon (vertices relative to O, counter-
 * clockwise about n, already in the plane): out = {I1, S, V1x, V1y, V1z, V3x, V3y, V3z}. */
void oracle_polygon_integrals(int nv, const double *pts, const double *nrm, double *out) {
    double I1 = 0, S = 0, V1[3] = {0, 0, 0}, V3[3] = {0, 0, 0};
    for (int e = 0; e < nv; ++e) edge_triangle(pts + 3 * e, pts + 3 * ((e + 1) % nv), nrm, &I1, &S, V1, V3);
    out[0] = I1; out[1] = S;
    for (int q = 0; q < 3; ++q) { out[2 + q] = V1[q]; out[5 + q] = V3[q]; }
}

/* ------------------------------------------------------------------------------------------ */
/* Impedance boundary condition, Section 2.3.
 * On a good conductor Eq. (2.24), n x E = Z n x (n x H), with n the scatterer's outward normal
 * and Z = sqrt(mu_j / eps_j) the surface impedance relative to the vacuum impedance (principal
 * root, Re Z >= 0), ties the tangential exterior fields together.  With curl E = i k0 mu_0 H (H
 * in units of the vacuum impedance) it gives
 *   n0 x curl E_0 = zeta n0 x (n0 x E_0),   zeta = i k0 mu_0 / Z,
 * and the background equation (2.5) becomes Eq. (2.25), in E_0 alone (3 unknowns per node).
 * Moved into the form of Eq. (2.12) (operator on the left, E_inc on the right) and discretised
 * with the one-point rule of Eq. (2.8):
 *   1/2 E(s_a) - sum_b w_b [n0 grad'g0 - (n0.grad'g0) I - grad'g0 n0] . E(s_b)
 *              + sum_b w_b zeta_b g0 n0 x (n0 x E(s_b))  =  E_inc(s_a),
 * n0 = -n_b, g0 = g_0(s_b, s_a); the b = a term from the background self-patch integrals of
 * Appendix B.  Vectors are [n_rhs][N][3] complex. */
static cplx ibc_zeta(const oracle_ctx *c, int j) { return I * c->k0 * c->mu[0] / csqrt(c->mu[j] / c->eps[j]); }

/* n0 x (n0 x v) = n0 (n0.v) - v for a unit normal (the same for n and -n) */
static inline void nxnx(const double *nn, const cplx *v, cplx *o) {
    cplx nv = nn[0] * v[0] + nn[1] * v[1] + nn[2] * v[2];
    for (int q = 0; q < 3; ++q) o[q] = nn[q] * nv - v[q];
}

static void ibc_node_rows(const oracle_ctx *c, int64_t a, int64_t n_rhs, const cplx *x, cplx *out) {
    const int64_t N = c->N;
    const double *sa = c->s + 3 * a;
    const cplx k0 = c->k[0];
    for (int64_t r = 0; r < n_rhs * 3; ++r) out[r] = 0;
    for (int64_t b = 0; b < N; ++b) {
        if (b == a) continue;
        double rv[3]; sub3(c->s + 3 * b, sa, rv);
        double R = norm3(rv);
        const double wb = c->w[b];
        const double *nb = c->n + 3 * b;
        double n0[3] = {-nb[0], -nb[1], -nb[2]};
        cplx g0 = cexp(I * k0 * R) / (4 * PI * R);
        cplx c0 = g0 * (I * k0 - 1.0 / R) / R;
        cplx a0[3] = {c0 * rv[0], c0 * rv[1], c0 * rv[2]};
        cplx zg = ibc_zeta(c, c->dom[b]) * g0;
        for (int64_t r = 0; r < n_rhs; ++r) {
            const cplx *xb = x + (r * N + b) * 3;
            cplx B[3], T[3];
            bracket(n0, a0, xb, B);
            nxnx(n0, xb, T);
            for (int q = 0; q < 3; ++q) out[3 * r + q] += -wb * B[q] + wb * zg * T[q];
        }
    }
    const double *na = c->n + 3 * a;
    double n0a[3] = {-na[0], -na[1], -na[2]};
    cplx zs = ibc_zeta(c, c->dom[a]) * c->Sg[2 * a];
    for (int64_t r = 0; r < n_rhs; ++r) {
        const cplx *xa = x + (r * N + a) * 3;
        cplx B[3], T[3];
        bracket(n0a, c->Sdg + 6 * a, xa, B);
        nxnx(n0a, xa, T);
        for (int q = 0; q < 3; ++q) out[3 * r + q] += 0.5 * xa[q] - B[q] + zs * T[q];
    }
}

/* y = A_IBC x (Eq. 2.25), x and y [n_rhs][N][3] */
void oracle_ibc_matvec(const oracle_ctx *c, int64_t n_rhs, const double *x_, double *y_) {
    const cplx *x = (const cplx *)x_;
    cplx *y = (cplx *)y_;
    const int64_t N = c->N;
#pragma omp parallel
    {
        cplx *buf = malloc(sizeof(cplx) * 3 * n_rhs);
#pragma omp for schedule(dynamic, 8)
        for (int64_t a = 0; a < N; ++a) {
            ibc_node_rows(c, a, n_rhs, x, buf);
            for (int64_t r = 0; r < n_rhs; ++r)
                for (int q = 0; q < 3; ++q) y[(r * N + a) * 3 + q] = buf[3 * r + q];
        }
        free(buf);
    }
}

/* 3x3 self block of Eq. (2.25) per node, row-major [N][3][3]: the preconditioner block of
 * Eq. (3.2) for the impedance system */
void oracle_ibc_precond_blocks(const oracle_ctx *c, double *M_) {
    cplx *M = (cplx *)M_;
    for (int64_t a = 0; a < c->N; ++a)
        for (int col = 0; col < 3; ++col) {
            cplx e[3] = {0, 0, 0};
            e[col] = 1.0;
            cplx y[3];
            const double *na = c->n + 3 * a;
            double n0a[3] = {-na[0], -na[1], -na[2]};
            cplx B[3], T[3];
            bracket(n0a, c->Sdg + 6 * a, e, B);
            nxnx(n0a, e, T);
            cplx zs = ibc_zeta(c, c->dom[a]) * c->Sg[2 * a];
            for (int q = 0; q < 3; ++q) y[q] = 0.5 * e[q] - B[q] + zs * T[q];
            for (int q = 0; q < 3; ++q) M[9 * a + 3 * q + col] = y[q];
        }
}

/* The unknown Psi = n x curl E_0 of Eq. (2.12) (scatterer normal) implied by Eq. (2.24):
 * Psi = -(n0 x curl E_0) = -zeta n0 x (n0 x E_0) = zeta (E_0 - n (n.E_0)).  E, Psi [n_rhs][N][3]. */
void oracle_ibc_psi(const oracle_ctx *c, int64_t n_rhs, const double *E_, double *Psi_) {
    const cplx *E = (const cplx *)E_;
    cplx *Psi = (cplx *)Psi_;
    for (int64_t r = 0; r < n_rhs; ++r)
        for (int64_t a = 0; a < c->N; ++a) {
            const cplx *e = E + (r * c->N + a) * 3;
            cplx T[3];
            nxnx(c->n + 3 * a, e, T);
            cplx z = ibc_zeta(c, c->dom[a]);
            for (int q = 0; q < 3; ++q) Psi[(r * c->N + a) * 3 + q] = -z * T[q];
        }
}

/* zeta_j = i k0 mu_0 / Z_j of every scatterer, [J+1] complex (entry 0 unused, set to 0) */
void oracle_ibc_zeta(const oracle_ctx *c, double *z_) {
    cplx *z = (cplx *)z_;
    z[0] = 0;
    for (int j = 1; j <= c->J; ++j) z[j] = ibc_zeta(c, j);
}

/* ------------------------------------------------------------------------------------------ */
/* Fields inside the scatterers from the representation formula of domain j (Appendix A, the
 * relation behind Eq. 2.5 at a point r inside Omega_j rather than on its boundary):
 *   E_j(r) = sum_{b in j} w_b { [n_b (grad'g_j . v_b) - (n_b . grad'g_j) v_b - grad'g_j (n_b . v_b)]
 *                               - g_j (n_b x curl E_j)(s_b) },
 * n_b the scatterer's outward normal (outward from Omega_j), v_b = E_j(s_b) = T_j Phi_b (Eq. 2.6),
 * n x curl E_j = gamma_j Psi_b (Eq. 2.7), g_j = g_j(s_b, r); no incident field inside.  The
 * magnetic field H_j = curl E_j / (i k0 mu_j) is the curl of the same sum: (K n) x v + n x (K v)
 * for the bracket (K the Hessian of g_j in the source point) and +grad'g_j x (gamma_j Psi) for the
 * single layer.  At a point outside Omega_j the same sum is the extinction (null-field) integral,
 * zero for exact data.  x one solution [N][6]; pts [np][3]; pdom [np] scatterer ids; E, H [np][3]
 * (H may be NULL). */
void oracle_interior_field(const oracle_ctx *c, const double *x_, int64_t np_, const double *pts, const int32_t *pdom,
                           double *E_, double *H_) {
    const cplx *x = (const cplx *)x_;
    cplx *E = (cplx *)E_;
    cplx *H = (cplx *)H_;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < np_; ++p) {
        const double *r = pts + 3 * p;
        const int j = pdom[p];
        const cplx k = c->k[j], gam = c->gam[j];
        cplx acc[3] = {0, 0, 0}, curl[3] = {0, 0, 0};
        for (int64_t b = 0; b < c->N; ++b) {
            if (c->dom[b] != j) continue;
            double rv[3]; sub3(c->s + 3 * b, r, rv);
            const double R = norm3(rv);
            const double rh[3] = {rv[0] / R, rv[1] / R, rv[2] / R};
            const double *nb = c->n + 3 * b;
            const cplx g = cexp(I * k * R) / (4 * PI * R);
            const cplx g1 = g * (I * k - 1.0 / R);
            const cplx g2 = g * ((I * k - 1.0 / R) * (I * k - 1.0 / R) + 1.0 / (R * R));
            cplx v[3], q[3];
            apply_T(c, j, nb, x + 6 * b, v);
            for (int i = 0; i < 3; ++i) q[i] = gam * x[6 * b + 3 + i];
            cplx a[3] = {g1 * rh[0], g1 * rh[1], g1 * rh[2]};
            cplx B[3];
            bracket(nb, a, v, B);
            for (int i = 0; i < 3; ++i) acc[i] += c->w[b] * (B[i] - g * q[i]);
            if (H) {
                const double rn = dot3(rh, nb);
                const cplx rv_ = rh[0] * v[0] + rh[1] * v[1] + rh[2] * v[2];
                cplx Kn[3], Kv[3];
                for (int i = 0; i < 3; ++i) {
                    Kn[i] = g2 * rh[i] * rn + g1 / R * (nb[i] - rh[i] * rn);
                    Kv[i] = g2 * rh[i] * rv_ + g1 / R * (v[i] - rh[i] * rv_);
                }
                const cplx t[3] = {Kn[1] * v[2] - Kn[2] * v[1] + nb[1] * Kv[2] - nb[2] * Kv[1] + (a[1] * q[2] - a[2] * q[1]),
                                   Kn[2] * v[0] - Kn[0] * v[2] + nb[2] * Kv[0] - nb[0] * Kv[2] + (a[2] * q[0] - a[0] * q[2]),
                                   Kn[0] * v[1] - Kn[1] * v[0] + nb[0] * Kv[1] - nb[1] * Kv[0] + (a[0] * q[1] - a[1] * q[0])};
                for (int i = 0; i < 3; ++i) curl[i] += c->w[b] * t[i];
            }
        }
        for (int i = 0; i < 3; ++i) E[3 * p + i] = acc[i];
        if (H) {
            const cplx iwm = I * c->k0 * c->mu[j];
            for (int i = 0; i < 3; ++i) H[3 * p + i] = curl[i] / iwm;
        }
    }
}
