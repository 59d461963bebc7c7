// tables.cu -- multipole bases of the nodes and translation matrices, Eqs. (2.14)-(2.21).
//
// Scaled coefficients.  With lambda = |k_d| w_l on level l (box width w_l) the library stores
//   multipole  Ct_n^m = C_n^m / lambda^(n+1),   local  Dt_n^m = D_n^m lambda^n,
// so that neither underflows nor overflows in single precision when |k| w << 1 (the expansions
// themselves are those of Eq. 2.17, truncated at n = p-1).
//
// P2M (Eqs. 2.18-2.19) for a source with monopole strength Q and dipole moment m at s:
//   Ct_n^m += (i k / lambda^(n+1)) [ Q R_n^{-m}(s - c) + m . grad R_n^{-m}(s - c) ]
// L2P (first term of Eq. 2.23):  phi(r) = sum Dt_n^m R_n^m(r - c) / lambda^n.
//
// Translation matrices are obtained by projecting the translated basis function on the sphere
// |x| = rho around the new centre: for the column of input basis function F_c(x + t),
//   T[r][c] = (1 / rad_{n_r}(k rho)) int F_c(rho xhat + t) conj(Y_r(xhat)) dOmega,
// rad = j_n for regular output bases (S|R of Eq. 2.21 and R|R), h_n for singular output bases
// (S|S of Eq. 2.20).  The integral uses Gauss-Legendre nodes in cos(theta) and the trapezoid rule
// in phi, exact for spherical-harmonic degree well above p, so the aliasing error is set by the
// decay of F_c's harmonic content on the sphere (rho/|t| <= 1/2 for S|R with rho = w_l,
// |t|/rho < 1/2 for S|S with rho = 2 w_l).
#include <algorithm>
#include <cmath>

#include "fmbem_internal.cuh"
#include "special.cuh"

namespace {

constexpr int PMAX = 20;  // largest supported truncation number

inline unsigned nblk(int64_t n, int tb) { return (unsigned)((n + tb - 1) / tb); }

}  // namespace

// Gauss-Legendre nodes and weights on [-1,1] (Newton iteration on P_n)
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = cos(FMBEM_PI * (i + 0.75) / (n + 0.5)), dp = 0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1, p1 = 0;
            for (int j = 1; j <= n; ++j) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
            }
            dp = n * (z * p0 - p1) / (z * z - 1.0);
            double dz = p0 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

namespace {

__global__ void k_to32(const c64 *a, c32 *b, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = to<float>(a[i]);
}

// per node and side: P2M basis (scaled, with the i k prefactor) and L2P basis
// (the scale lambda = |k_d| w_l of the node's leaf level: |k_d| w_0 / 2^l, as the level tables')
__global__ void k_node_bases(int64_t N, int p, const double *pos, const int32_t *dom, const int32_t *node_leaf,
                             const int32_t *box_leafpos, const int32_t *leaf_level, const double *box_ctr,
                             const c64 *kd, const double *kw0 /* [J+1] |k_d| w_0 */, c64 *Bp2m, c64 *Bl2p,
                             c64 *Bl2pg) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int side = blockIdx.y;
    if (i >= N) return;
    int d = side == 0 ? 0 : dom[i];
    c64 k = kd[d];
    double la = ldexp(kw0[d], -leaf_level[box_leafpos[node_leaf[i]]]);
    const double *c = box_ctr + 3 * node_leaf[i];
    double r[3] = {pos[3 * i] - c[0], pos[3 * i + 1] - c[1], pos[3 * i + 2] - c[2]};
    c64 R[(PMAX + 1) * (PMAX + 1)], rad[PMAX + 2];
    double Pb[(PMAX + 2) * (PMAX + 3) / 2];
    wave_functions<false>(p, k, r, R, rad, Pb);  // degrees 0..p (one more for the gradient)
    const int p2 = p * p;
    c64 ik = c64{-k.im, k.re};
    c64 *bp = Bp2m + ((int64_t)side * N + i) * 4 * p2;
    c64 *bl = Bl2p + ((int64_t)side * N + i) * p2;
    c64 *bg = Bl2pg + ((int64_t)side * N + i) * 3 * p2;  // gradient of the L2P basis (adjoint product)
    double lpow = 1.0;  // lambda^n
    for (int n = 0; n < p; ++n) {
        double sm = 1.0 / (lpow * la);  // 1/lambda^(n+1)
        for (int m = -n; m <= n; ++m) {
            int q = n * n + n + m;
            c64 g[3];
            grad_regular(p, k, R, n, -m, g);
            bp[0 * p2 + q] = (ik * R[n * n + n - m]) * sm;
            bp[1 * p2 + q] = (ik * g[0]) * sm;
            bp[2 * p2 + q] = (ik * g[1]) * sm;
            bp[3 * p2 + q] = (ik * g[2]) * sm;
            bl[q] = R[q] * (1.0 / lpow);
            grad_regular(p, k, R, n, m, g);
            for (int a = 0; a < 3; ++a) bg[a * p2 + q] = g[a] * (1.0 / lpow);
        }
        lpow *= la;
    }
}

// evaluate the input basis functions of a batch of translations at the quadrature points:
// F[m][q][c] = F_c(rho xhat_q + t_m), c = 0..p2-1; F_c = S_c (singular) or R_c (regular)
template <bool SINGULAR>
__global__ void k_eval_cols(int nmat, int Q, int p, c64 k, double rho, const double *xq /* [Q][3] unit */,
                            const double *tvec /* [nmat][3] */, c64 *F) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nmat * Q) return;
    int m = (int)(idx / Q), q = (int)(idx % Q);
    double r[3];
    for (int a = 0; a < 3; ++a) r[a] = rho * xq[3 * q + a] + tvec[3 * m + a];
    c64 V[PMAX * PMAX], rad[PMAX + 1];
    double Pb[(PMAX + 1) * (PMAX + 2) / 2];
    wave_functions<SINGULAR>(p - 1, k, r, V, rad, Pb);
    c64 *out = F + idx * (int64_t)(p * p);
    for (int c = 0; c < p * p; ++c) out[c] = V[c];
}

// spherical harmonics at rotated quadrature points: F[m][q][c] = Y_c(M_m xhat_q), M_m a 3x3
// rotation (row-major); projected on Y_r this gives the degree-preserving rotation matrices
__global__ void k_eval_rot(int nmat, int Q, int p, const double *xq, const double *Mrot, c64 *F) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nmat * Q) return;
    int m = (int)(idx / Q), q = (int)(idx % Q);
    const double *M = Mrot + 9 * m, *x = xq + 3 * q;
    double v[3];
    for (int a = 0; a < 3; ++a) v[a] = M[3 * a] * x[0] + M[3 * a + 1] * x[1] + M[3 * a + 2] * x[2];
    double nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double ct = v[2] / nv;
    double phi = (v[0] == 0.0 && v[1] == 0.0) ? 0.0 : atan2(v[1], v[0]);
    double Pb[(PMAX + 1) * (PMAX + 2) / 2];
    legendre_bar(p - 1, ct, Pb);
    c64 *out = F + idx * (int64_t)(p * p);
    for (int n = 0; n < p; ++n)
        for (int mm = -n; mm <= n; ++mm) {
            int am = mm < 0 ? -mm : mm;
            double sp, cp;
            sincos(mm * phi, &sp, &cp);
            out[n * n + n + mm] = c64{cp, sp} * (((am & 1) ? -1.0 : 1.0) * Pb[n * (n + 1) / 2 + am]);
        }
}

// projection weights Yc[q][r] = W_q conj(Y_r(xhat_q)) / rad_{n_r}(k rho), rad = j_n (radial 0),
// h_n (radial 1) or 1 (radial 2)
__global__ void k_proj_weights(int Q, int p, const double *xq, const double *wq, c64 k, double rho, int radial,
                               c64 *Yc) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    double Pb[(PMAX + 1) * (PMAX + 2) / 2];
    double r[3] = {xq[3 * q], xq[3 * q + 1], xq[3 * q + 2]};
    double ct = r[2];
    double phi = (r[0] == 0.0 && r[1] == 0.0) ? 0.0 : atan2(r[1], r[0]);
    legendre_bar(p - 1, ct, Pb);
    c64 radv[PMAX + 1];
    c64 z = k * rho;
    if (radial == 1) sph_h1(p - 1, z, radv);
    else if (radial == 0) sph_j(p - 1, z, radv);
    else
        for (int n = 0; n < p; ++n) radv[n] = {1.0, 0.0};
    for (int n = 0; n < p; ++n)
        for (int m = -n; m <= n; ++m) {
            int am = m < 0 ? -m : m;
            double sgn = (am & 1) ? -1.0 : 1.0;
            double sp, cp;
            sincos(m * phi, &sp, &cp);
            c64 Ynm = c64{cp, sp} * (sgn * Pb[n * (n + 1) / 2 + am]);
            c64 v = cdiv(conjg(Ynm) * wq[q], radv[n]);
            Yc[(int64_t)q * p * p + n * n + n + m] = v;
        }
}

// T[m][r][c] = sum_q Yc[q][r] F[m][q][c]  (complex FP64 GEMM per matrix, 16x16 tiles),
// then scaled: out[m][c][r] = sr[r] * T * sc[c], stored input-major for the apply kernels
__global__ void k_project(int nmat, int Q, int p2, const c64 *Yc, const c64 *F, const double *sr, const double *sc,
                          c64 *out64, c32 *out32, const int64_t *dst /* [nmat] destination matrix index */) {
    __shared__ c64 As[16][17], Bs[16][17];
    int m = blockIdx.z;
    int r0 = blockIdx.y * 16, c0 = blockIdx.x * 16;
    int tr = threadIdx.y, tc = threadIdx.x;
    const c64 *Fm = F + (int64_t)m * Q * p2;
    c64 acc = {0, 0};
    for (int q0 = 0; q0 < Q; q0 += 16) {
        int q = q0 + tc;
        As[tr][tc] = (q < Q && r0 + tr < p2) ? Yc[(int64_t)q * p2 + r0 + tr] : c64{0, 0};
        int q2 = q0 + tr;
        Bs[tr][tc] = (q2 < Q && c0 + tc < p2) ? Fm[(int64_t)q2 * p2 + c0 + tc] : c64{0, 0};
        __syncthreads();
        for (int u = 0; u < 16; ++u) cfma(acc, As[tr][u], Bs[u][tc]);
        __syncthreads();
    }
    int r = r0 + tr, c = c0 + tc;
    if (r < p2 && c < p2) {
        c64 v = acc * (sr[r] * sc[c]);
        int64_t o = dst[m] * (int64_t)p2 * p2 + (int64_t)c * p2 + r;
        out64[o] = v;
        out32[o] = to<float>(v);
    }
}

}  // namespace

// ---- truncation number from a tolerance (option fmm_tol; reading of Eq. 2.17 and "FMM tolerance")
// For every level l and domain d, the relative RMS error of the truncated addition theorem
// (Eq. 2.14 summed over m: g = (i k / 4 pi) sum_n (2n + 1) j_n(k rho) h_n(k r) P_n(cos gamma)) is
// sampled over source points s in a box of width w_l centred at the origin and target points t in
// boxes of the far-field offsets (2,0,0), (2,1,0), (2,1,1), (2,2,1), (3,0,0), (3,2,1) w_l: the
// multipole expansion about the source centre (rho = s, r = t) and the local expansion about the
// target centre (rho = t - c_t, r = s - c_t) each truncated after degree p - 1, their errors added
// per sample; err[(l * (J+1) + d) * (TRUNC_PMAX + 1) + p] = sqrt(sum err^2 / sum |g|^2).
constexpr int TRUNC_PMAX = 20;
__device__ inline uint64_t trunc_hash(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
__device__ inline double trunc_u01(uint64_t a, uint64_t b) { return (trunc_hash(a * 1000003ull + b) >> 11) * 0x1.0p-53; }

__device__ inline void gegenbauer_partials(c64 k, double rho, double r, double cg, c64 *part) {
    c64 jn[TRUNC_PMAX + 1], hn[TRUNC_PMAX + 1];
    sph_j(TRUNC_PMAX, k * rho, jn);
    sph_h1(TRUNC_PMAX, k * r, hn);
    double P0 = 1.0, P1 = cg;  // Legendre P_n(cos gamma) by the three-term recurrence
    c64 acc = {0, 0};
    const c64 pre = (1.0 / (4.0 * FMBEM_PI)) * (c64{0.0, 1.0} * k);
    part[0] = acc;
    for (int n = 0; n < TRUNC_PMAX; ++n) {
        const double Pn = n == 0 ? P0 : (n == 1 ? P1 : 0.0);
        double Pcur = Pn;
        if (n >= 2) {
            Pcur = ((2.0 * n - 1.0) * cg * P1 - (n - 1.0) * P0) / n;
            P0 = P1;
            P1 = Pcur;
        }
        acc += (2.0 * n + 1.0) * Pcur * (jn[n] * hn[n]);
        part[n + 1] = pre * acc;  // sum over degrees 0..n: truncation number n + 1
    }
}

__global__ void k_trunc_error(int nlev, int lev0, const double *wl, int nd, const c64 *kd, int nsamp, double *err) {
    const int li = blockIdx.x, d = blockIdx.y;
    const double w = wl[li];
    const c64 k = kd[d];
    __shared__ double se[TRUNC_PMAX + 1], sg;
    for (int q = threadIdx.x; q <= TRUNC_PMAX; q += blockDim.x) se[q] = 0.0;
    if (threadIdx.x == 0) sg = 0.0;
    __syncthreads();
    const int offs[6][3] = {{2, 0, 0}, {2, 1, 0}, {2, 1, 1}, {2, 2, 1}, {3, 0, 0}, {3, 2, 1}};
    double le[TRUNC_PMAX + 1];
    for (int q = 0; q <= TRUNC_PMAX; ++q) le[q] = 0.0;
    double lg = 0.0;
    for (int i = threadIdx.x; i < nsamp; i += blockDim.x) {
        const uint64_t key = ((uint64_t)(lev0 + li) * 64 + d) * 1000000ull + i;
        const int o = i % 6;
        double sp[3], tp[3], ct[3];
        for (int c = 0; c < 3; ++c) {
            sp[c] = (trunc_u01(key, c) - 0.5) * w;
            ct[c] = offs[o][c] * w;
            tp[c] = ct[c] + (trunc_u01(key, 3 + c) - 0.5) * w;
        }
        const double R = sqrt((tp[0] - sp[0]) * (tp[0] - sp[0]) + (tp[1] - sp[1]) * (tp[1] - sp[1]) +
                              (tp[2] - sp[2]) * (tp[2] - sp[2]));
        const c64 g = (1.0 / (4.0 * FMBEM_PI * R)) * cexpd(c64{-k.im * R, k.re * R});
        // multipole about the source centre (the origin)
        const double rs = sqrt(sp[0] * sp[0] + sp[1] * sp[1] + sp[2] * sp[2]);
        const double rt = sqrt(tp[0] * tp[0] + tp[1] * tp[1] + tp[2] * tp[2]);
        const double cm = (sp[0] * tp[0] + sp[1] * tp[1] + sp[2] * tp[2]) / fmax(rs * rt, 1e-300);
        // local about the target centre
        double a[3], b[3];
        for (int c = 0; c < 3; ++c) { a[c] = tp[c] - ct[c]; b[c] = sp[c] - ct[c]; }
        const double ra = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        const double rb = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
        const double cl = (a[0] * b[0] + a[1] * b[1] + a[2] * b[2]) / fmax(ra * rb, 1e-300);
        c64 pm[TRUNC_PMAX + 1], pl[TRUNC_PMAX + 1];
        gegenbauer_partials(k, rs, rt, cm, pm);
        gegenbauer_partials(k, ra, rb, cl, pl);
        for (int q = 0; q <= TRUNC_PMAX; ++q) {
            const double e = sqrt(abs2(g - pm[q])) + sqrt(abs2(g - pl[q]));
            le[q] += e * e;
        }
        lg += abs2(g);
    }
    for (int q = 0; q <= TRUNC_PMAX; ++q) atomicAdd(&se[q], le[q]);
    atomicAdd(&sg, lg);
    __syncthreads();
    for (int q = threadIdx.x; q <= TRUNC_PMAX; q += blockDim.x)
        err[((int64_t)li * nd + d) * (TRUNC_PMAX + 1) + q] = sqrt(se[q] / fmax(sg, 1e-300));
}

void choose_truncation(fmbem *h, cudaStream_t s) {
    const double tol = h->opt.fmm_tol;
    const int lmax = h->lmax, nlev = lmax - 1, nd = h->Jf + 1;  // levels 2..lmax
    std::vector<double> wl(nlev);
    for (int l = 2; l <= lmax; ++l) wl[l - 2] = h->lev[l].w;
    double *dw = (double *)dev_alloc(h, sizeof(double) * nlev);
    c64 *dk = (c64 *)dev_alloc(h, sizeof(c64) * nd);
    double *de = (double *)dev_alloc(h, sizeof(double) * nlev * nd * (TRUNC_PMAX + 1));
    CK(cudaMemcpyAsync(dw, wl.data(), sizeof(double) * nlev, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dk, h->k.data(), sizeof(c64) * nd, cudaMemcpyHostToDevice, s));
    k_trunc_error<<<dim3((unsigned)nlev, (unsigned)nd), 128, 0, s>>>(nlev, 2, dw, nd, dk, 6 * 512, de);
    CKL("k_trunc_error");
    std::vector<double> e((size_t)nlev * nd * (TRUNC_PMAX + 1));
    CK(cudaMemcpyAsync(e.data(), de, sizeof(double) * e.size(), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    dev_free(h, dw);
    dev_free(h, dk);
    dev_free(h, de);
    h->p_level.assign(lmax + 1, 0);
    h->trunc_err.assign(lmax + 1, 0.0);
    int p = 2;
    for (int l = 2; l <= lmax; ++l) {
        int pl = 2;
        for (int d = 0; d < nd; ++d) {
            const double *el = &e[((size_t)(l - 2) * nd + d) * (TRUNC_PMAX + 1)];
            int q = 2;
            while (q < TRUNC_PMAX && !(el[q] <= tol)) ++q;
            pl = std::max(pl, q);
        }
        h->p_level[l] = pl;
        p = std::max(p, pl);
    }
    for (int l = 2; l <= lmax; ++l) {
        double worst = 0.0;
        for (int d = 0; d < nd; ++d) worst = std::max(worst, e[((size_t)(l - 2) * nd + d) * (TRUNC_PMAX + 1) + p]);
        h->trunc_err[l] = worst;
    }
    h->p = p;
    h->p2 = p * p;
}

void build_tables(fmbem *h, cudaStream_t s) {
    const int p = h->p, p2 = p * p, J = h->J, lmax = h->lmax;
    const int64_t N = h->N;
    if (p < 2 || p > PMAX) throw fmbem_error{FMBEM_ERR_INVALID_ARGUMENT, "p must be in 2..20"};
    // scales lambda = |k_d| w_l
    h->lam.assign((size_t)(J + 1) * (lmax + 1), 0.0);
    for (int d = 0; d <= J; ++d)
        for (int l = 0; l <= lmax; ++l) h->lam[d * (lmax + 1) + l] = cabsd(h->k[d]) * h->lev[l].w;

    // ---- node bases
    c64 *dk = (c64 *)dev_alloc(h, sizeof(c64) * (J + 1));
    double *dl = (double *)dev_alloc(h, sizeof(double) * (J + 1));
    std::vector<double> lleaf(J + 1);
    for (int d = 0; d <= J; ++d) lleaf[d] = cabsd(h->k[d]) * h->lev[0].w;
    CK(cudaMemcpyAsync(dk, h->k.data(), sizeof(c64) * (J + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dl, lleaf.data(), sizeof(double) * (J + 1), cudaMemcpyHostToDevice, s));
    h->B_p2m64 = (c64 *)dev_alloc(h, sizeof(c64) * 2 * N * 4 * p2);
    h->B_l2p64 = (c64 *)dev_alloc(h, sizeof(c64) * 2 * N * p2);
    h->B_l2pg64 = (c64 *)dev_alloc(h, sizeof(c64) * 2 * N * 3 * p2);
    {
        dim3 grid(nblk(N, 64), 2);
        k_node_bases<<<grid, 64, 0, s>>>(N, p, h->pos, h->dom, h->node_leaf, h->box_leafpos, h->leaf_level, h->box_ctr,
                                          dk, dl, h->B_p2m64, h->B_l2p64,
                                          h->B_l2pg64);
        CKL("k_node_bases");
    }
    h->B_p2m32 = (c32 *)dev_alloc(h, sizeof(c32) * 2 * N * 4 * p2);
    h->B_l2p32 = (c32 *)dev_alloc(h, sizeof(c32) * 2 * N * p2);
    h->B_l2pg32 = (c32 *)dev_alloc(h, sizeof(c32) * 2 * N * 3 * p2);
    k_to32<<<nblk(2 * N * 4 * p2, 256), 256, 0, s>>>(h->B_p2m64, h->B_p2m32, 2 * N * 4 * p2);
    k_to32<<<nblk(2 * N * p2, 256), 256, 0, s>>>(h->B_l2p64, h->B_l2p32, 2 * N * p2);
    k_to32<<<nblk(2 * N * 3 * p2, 256), 256, 0, s>>>(h->B_l2pg64, h->B_l2pg32, 2 * N * 3 * p2);
    CKL("k_to32");

    // ---- translation matrices
    const int Lt = p / 2 + 22, Lp = p + 44, Q = Lt * Lp;
    std::vector<double> gx, gw;
    gauss_legendre(Lt, gx, gw);
    std::vector<double> xq(3 * Q), wq(Q);
    for (int i = 0; i < Lt; ++i)
        for (int j = 0; j < Lp; ++j) {
            double ct = gx[i], st = sqrt(std::max(0.0, 1 - ct * ct)), ph = 2 * FMBEM_PI * j / Lp;
            int q = i * Lp + j;
            xq[3 * q] = st * cos(ph);
            xq[3 * q + 1] = st * sin(ph);
            xq[3 * q + 2] = ct;
            wq[q] = gw[i] * 2 * FMBEM_PI / Lp;
        }
    double *dxq = (double *)dev_alloc(h, sizeof(double) * 3 * Q);
    double *dwq = (double *)dev_alloc(h, sizeof(double) * Q);
    CK(cudaMemcpyAsync(dxq, xq.data(), sizeof(double) * 3 * Q, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dwq, wq.data(), sizeof(double) * Q, cudaMemcpyHostToDevice, s));

    const int64_t n_m2l = (int64_t)(J + 1) * (lmax + 1) * 316, n_oct = (int64_t)(J + 1) * (lmax + 1) * 8;
    h->T_m2l64 = (c64 *)dev_alloc(h, sizeof(c64) * n_m2l * p2 * p2);
    h->T_m2l32 = (c32 *)dev_alloc(h, sizeof(c32) * n_m2l * p2 * p2);
    h->T_mm64 = (c64 *)dev_alloc(h, sizeof(c64) * n_oct * p2 * p2);
    h->T_mm32 = (c32 *)dev_alloc(h, sizeof(c32) * n_oct * p2 * p2);
    h->T_ll64 = (c64 *)dev_alloc(h, sizeof(c64) * n_oct * p2 * p2);
    h->T_ll32 = (c32 *)dev_alloc(h, sizeof(c32) * n_oct * p2 * p2);
    CK(cudaMemsetAsync(h->T_m2l64, 0, sizeof(c64) * n_m2l * p2 * p2, s));
    CK(cudaMemsetAsync(h->T_m2l32, 0, sizeof(c32) * n_m2l * p2 * p2, s));
    CK(cudaMemsetAsync(h->T_mm64, 0, sizeof(c64) * n_oct * p2 * p2, s));
    CK(cudaMemsetAsync(h->T_mm32, 0, sizeof(c32) * n_oct * p2 * p2, s));
    CK(cudaMemsetAsync(h->T_ll64, 0, sizeof(c64) * n_oct * p2 * p2, s));
    CK(cudaMemsetAsync(h->T_ll32, 0, sizeof(c32) * n_oct * p2 * p2, s));

    const int BATCH = 316;
    c64 *F = (c64 *)dev_alloc(h, sizeof(c64) * (int64_t)BATCH * Q * p2);
    c64 *Yc = (c64 *)dev_alloc(h, sizeof(c64) * (int64_t)Q * p2);
    double *dt = (double *)dev_alloc(h, sizeof(double) * 3 * BATCH);
    int64_t *ddst = (int64_t *)dev_alloc(h, sizeof(int64_t) * BATCH);
    double *dsr = (double *)dev_alloc(h, sizeof(double) * p2);
    double *dsc = (double *)dev_alloc(h, sizeof(double) * p2);
    std::vector<double> sr(p2), sc(p2);

    // one batch of translations sharing (k, rho, output basis): evaluate, project, scale, store
    auto run_batch = [&](bool sing_in, bool sing_out, c64 k, double rho, const std::vector<double> &tv,
                         const std::vector<int64_t> &dst, c64 *o64, c32 *o32) {
        int nm = (int)dst.size();
        CK(cudaMemcpyAsync(dt, tv.data(), sizeof(double) * 3 * nm, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ddst, dst.data(), sizeof(int64_t) * nm, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dsr, sr.data(), sizeof(double) * p2, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dsc, sc.data(), sizeof(double) * p2, cudaMemcpyHostToDevice, s));
        k_proj_weights<<<nblk(Q, 64), 64, 0, s>>>(Q, p, dxq, dwq, k, rho, sing_out ? 1 : 0, Yc);
        CKL("k_proj_weights");
        if (sing_in) k_eval_cols<true><<<nblk((int64_t)nm * Q, 64), 64, 0, s>>>(nm, Q, p, k, rho, dxq, dt, F);
        else k_eval_cols<false><<<nblk((int64_t)nm * Q, 64), 64, 0, s>>>(nm, Q, p, k, rho, dxq, dt, F);
        CKL("k_eval_cols");
        dim3 grid((p2 + 15) / 16, (p2 + 15) / 16, nm), tb(16, 16);
        k_project<<<grid, tb, 0, s>>>(nm, Q, p2, Yc, F, dsr, dsc, o64, o32, ddst);
        CKL("k_project");
        CK(cudaStreamSynchronize(s));  // the staging buffers are reused by the next batch
    };
    auto nof = [](int q) { int n = 0; while ((n + 1) * (n + 1) <= q) ++n; return n; };

    for (int d = 0; d <= J; ++d) {
        const c64 k = h->k[d];
        for (int l = 2; l <= lmax; ++l) {
            const double w = h->lev[l].w, la = h->lam[d * (lmax + 1) + l];
            // S|R (M2L), t = c_target - c_source = -(offset) w, rho = w
            std::vector<double> tv;
            std::vector<int64_t> dst;
            for (int dx = -3; dx <= 3; ++dx)
                for (int dy = -3; dy <= 3; ++dy)
                    for (int dz = -3; dz <= 3; ++dz) {
                        if (abs(dx) <= 1 && abs(dy) <= 1 && abs(dz) <= 1) continue;
                        tv.push_back(-dx * w); tv.push_back(-dy * w); tv.push_back(-dz * w);
                        dst.push_back(m2l_matrix(d, l, m2l_offset_code(dx, dy, dz), lmax));
                    }
            for (int q = 0; q < p2; ++q) {
                int n = nof(q);
                sr[q] = pow(la, n);          // output local: times lambda^n
                sc[q] = pow(la, n + 1);      // input multipole: C = Ct lambda^(n+1)
            }
            run_batch(true, false, k, w, tv, dst, h->T_m2l64, h->T_m2l32);
            if (l >= 3) {
                const double lp = h->lam[d * (lmax + 1) + l - 1];
                // S|S (M2M): child octant o at level l, t = c_parent - c_child = (0.5 - o) w, rho = 2 w
                std::vector<double> tm, tl;
                std::vector<int64_t> dm;
                for (int o = 0; o < 8; ++o) {
                    int ox = (o >> 2) & 1, oy = (o >> 1) & 1, oz = o & 1;  // Morton bit order x,y,z
                    tm.push_back((0.5 - ox) * w); tm.push_back((0.5 - oy) * w); tm.push_back((0.5 - oz) * w);
                    tl.push_back((ox - 0.5) * w); tl.push_back((oy - 0.5) * w); tl.push_back((oz - 0.5) * w);
                    dm.push_back(oct_matrix(d, l, o, lmax));
                }
                for (int q = 0; q < p2; ++q) {
                    int n = nof(q);
                    sr[q] = 1.0 / pow(lp, n + 1);  // output parent multipole
                    sc[q] = pow(la, n + 1);        // input child multipole
                }
                run_batch(true, true, k, 2 * w, tm, dm, h->T_mm64, h->T_mm32);
                // R|R (L2L): t = c_child - c_parent, rho = w
                for (int q = 0; q < p2; ++q) {
                    int n = nof(q);
                    sr[q] = pow(la, n);            // output child local
                    sc[q] = 1.0 / pow(lp, n);      // input parent local
                }
                run_batch(false, false, k, w, tl, dm, h->T_ll64, h->T_ll32);
            }
        }
    }

    // ---- rotation form of S|R: T_o = B_o Z_{|t_o|} A_o, with A_o rotating the multipole
    // expansion into the frame whose z axis is t_o = c_target - c_source, Z the coaxial S|R
    // translation along z by |t_o| (block-diagonal in m) and B_o rotating the local expansion back.
    // A_o[r = (n,m')][c = (n,m)] = int Y_c(Q^T xhat) conj(Y_r(xhat)), B_o = same with Q, Q t_o = |t_o| z.
    if (h->m2l_rotation) {
        std::vector<int> sq;  // distinct squared offset lengths
        for (int dx = -3; dx <= 3; ++dx)
            for (int dy = -3; dy <= 3; ++dy)
                for (int dz = -3; dz <= 3; ++dz) {
                    if (abs(dx) <= 1 && abs(dy) <= 1 && abs(dz) <= 1) continue;
                    int v = dx * dx + dy * dy + dz * dz;
                    if (std::find(sq.begin(), sq.end(), v) == sq.end()) sq.push_back(v);
                }
        std::sort(sq.begin(), sq.end());
        h->n_tlen = (int)sq.size();
        std::vector<int8_t> tidx(316);
        // per offset: Rz (the azimuthal rotation), Ry (the polar one) and their transposes
        std::vector<double> Mz(9 * 316), MzT(9 * 316), My(9 * 316), MyT(9 * 316);
        std::vector<int64_t> dst(316);
        for (int dx = -3; dx <= 3; ++dx)
            for (int dy = -3; dy <= 3; ++dy)
                for (int dz = -3; dz <= 3; ++dz) {
                    if (abs(dx) <= 1 && abs(dy) <= 1 && abs(dz) <= 1) continue;
                    int o = m2l_offset_code(dx, dy, dz);
                    int v = dx * dx + dy * dy + dz * dz;
                    tidx[o] = (int8_t)(std::find(sq.begin(), sq.end(), v) - sq.begin());
                    // direction of t = -(dx, dy, dz)
                    double tx = -dx, ty = -dy, tz = -dz, tn = sqrt((double)v);
                    double ct = tz / tn, st = sqrt(std::max(0.0, 1 - ct * ct));
                    double ph = (tx == 0 && ty == 0) ? 0.0 : atan2(ty, tx), cp = cos(ph), sp = sin(ph);
                    // Q = R_y(-theta) R_z(-phi) maps t/|t| to z
                    double Rz[9] = {cp, sp, 0, -sp, cp, 0, 0, 0, 1};
                    double Ry[9] = {ct, 0, -st, 0, 1, 0, st, 0, ct};
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) {
                            Mz[9 * o + 3 * a + b] = Rz[3 * a + b];
                            MzT[9 * o + 3 * a + b] = Rz[3 * b + a];
                            My[9 * o + 3 * a + b] = Ry[3 * a + b];
                            MyT[9 * o + 3 * a + b] = Ry[3 * b + a];
                        }
                    dst[o] = o;
                }
        h->rot_tidx = (int8_t *)dev_alloc(h, 316);
        CK(cudaMemcpyAsync(h->rot_tidx, tidx.data(), 316, cudaMemcpyHostToDevice, s));
        // Q = Ry Rz maps t/|t| to z.  With T(M)[c][r] = <Y_r, Y_c o M>, T(M1 M2) = T(M1) T(M2), so the
        // forward factor T(Q^T) = T(Rz^T) T(Ry^T) and the back factor T(Q) = T(Ry) T(Rz); the z
        // factors are diagonal (phases e^{i m phi}) and the y factors real (see pack_rot_factors)
        const std::vector<double> *mats[4] = {&MzT, &MyT, &My, &Mz};
        c64 *Tf[4];
        c32 *Tf32 = (c32 *)dev_alloc(h, sizeof(c32) * 316 * p2 * p2);  // unused single-precision copy
        for (int f = 0; f < 4; ++f) Tf[f] = (c64 *)dev_alloc(h, sizeof(c64) * 316 * p2 * p2);
        double *dM = (double *)dev_alloc(h, sizeof(double) * 9 * 316);
        for (int q = 0; q < p2; ++q) { sr[q] = 1.0; sc[q] = 1.0; }
        CK(cudaMemcpyAsync(dsr, sr.data(), sizeof(double) * p2, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dsc, sc.data(), sizeof(double) * p2, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ddst, dst.data(), sizeof(int64_t) * 316, cudaMemcpyHostToDevice, s));
        k_proj_weights<<<nblk(Q, 64), 64, 0, s>>>(Q, p, dxq, dwq, c64{0, 0}, 1.0, 2, Yc);
        CKL("k_proj_weights");
        for (int pass = 0; pass < 4; ++pass) {
            CK(cudaMemcpyAsync(dM, mats[pass]->data(), sizeof(double) * 9 * 316, cudaMemcpyHostToDevice, s));
            k_eval_rot<<<nblk((int64_t)316 * Q, 64), 64, 0, s>>>(316, Q, p, dxq, dM, F);
            CKL("k_eval_rot");
            dim3 grid((p2 + 15) / 16, (p2 + 15) / 16, 316), tb(16, 16);
            k_project<<<grid, tb, 0, s>>>(316, Q, p2, Yc, F, dsr, dsc, Tf[pass], Tf32, ddst);
            CKL("k_project");
            CK(cudaStreamSynchronize(s));
        }
        dev_free(h, dM);
        pack_rot_factors(h, Tf[0], Tf[1], Tf[2], Tf[3], s);
        for (int f = 0; f < 4; ++f) dev_free(h, Tf[f]);
        dev_free(h, Tf32);
        // coaxial S|R per (domain, level, distinct length), scaled like the dense S|R
        const int64_t nz = (int64_t)(J + 1) * (lmax + 1) * h->n_tlen;
        h->R_Z64 = (c64 *)dev_alloc(h, sizeof(c64) * nz * p2 * p2);
        h->R_Z32 = (c32 *)dev_alloc(h, sizeof(c32) * nz * p2 * p2);
        CK(cudaMemsetAsync(h->R_Z64, 0, sizeof(c64) * nz * p2 * p2, s));
        CK(cudaMemsetAsync(h->R_Z32, 0, sizeof(c32) * nz * p2 * p2, s));
        for (int d = 0; d <= J; ++d)
            for (int l = 2; l <= lmax; ++l) {
                const double w = h->lev[l].w, la = h->lam[d * (lmax + 1) + l];
                std::vector<double> tv;
                std::vector<int64_t> dz;
                for (int i = 0; i < h->n_tlen; ++i) {
                    tv.push_back(0.0); tv.push_back(0.0); tv.push_back(sqrt((double)sq[i]) * w);
                    dz.push_back(((int64_t)d * (lmax + 1) + l) * h->n_tlen + i);
                }
                for (int q = 0; q < p2; ++q) {
                    int n = nof(q);
                    sr[q] = pow(la, n);
                    sc[q] = pow(la, n + 1);
                }
                run_batch(true, false, h->k[d], w, tv, dz, h->R_Z64, h->R_Z32);
            }
        pack_rot_tables(h, s);
        // coaxial S|S (M2M, child to parent) and R|R (L2L, parent to child) along z by the half
        // diagonal sqrt(3) w / 2 of a child box, scaled like the dense S|S and R|R
        const int64_t nzl = (int64_t)(J + 1) * (lmax + 1);
        h->R_Zmm64 = (c64 *)dev_alloc(h, sizeof(c64) * nzl * p2 * p2);
        h->R_Zmm32 = (c32 *)dev_alloc(h, sizeof(c32) * nzl * p2 * p2);
        h->R_Zll64 = (c64 *)dev_alloc(h, sizeof(c64) * nzl * p2 * p2);
        h->R_Zll32 = (c32 *)dev_alloc(h, sizeof(c32) * nzl * p2 * p2);
        CK(cudaMemsetAsync(h->R_Zmm64, 0, sizeof(c64) * nzl * p2 * p2, s));
        CK(cudaMemsetAsync(h->R_Zmm32, 0, sizeof(c32) * nzl * p2 * p2, s));
        CK(cudaMemsetAsync(h->R_Zll64, 0, sizeof(c64) * nzl * p2 * p2, s));
        CK(cudaMemsetAsync(h->R_Zll32, 0, sizeof(c32) * nzl * p2 * p2, s));
        for (int d = 0; d <= J; ++d)
            for (int l = 3; l <= lmax; ++l) {
                const double w = h->lev[l].w, la = h->lam[d * (lmax + 1) + l], lp = h->lam[d * (lmax + 1) + l - 1];
                const std::vector<double> tv = {0.0, 0.0, 0.5 * sqrt(3.0) * w};
                const std::vector<int64_t> dz = {(int64_t)d * (lmax + 1) + l};
                for (int q = 0; q < p2; ++q) {
                    int n = nof(q);
                    sr[q] = 1.0 / pow(lp, n + 1);  // output parent multipole
                    sc[q] = pow(la, n + 1);        // input child multipole
                }
                run_batch(true, true, h->k[d], 2 * w, tv, dz, h->R_Zmm64, h->R_Zmm32);
                for (int q = 0; q < p2; ++q) {
                    int n = nof(q);
                    sr[q] = pow(la, n);            // output child local
                    sc[q] = 1.0 / pow(lp, n);      // input parent local
                }
                run_batch(false, false, h->k[d], w, tv, dz, h->R_Zll64, h->R_Zll32);
            }
        pack_rot_tables_mm(h, s);
    }
    dev_free(h, F);
    dev_free(h, Yc);
    dev_free(h, dt);
    dev_free(h, ddst);
    dev_free(h, dsr);
    dev_free(h, dsc);
    dev_free(h, dxq);
    dev_free(h, dwq);
    dev_free(h, dk);
    dev_free(h, dl);
    // tensor-core images of the S|R and R|R matrices for the batched TF32 path
    if (m2l_tc_supported(h) && !h->opt.fp32_only) build_tc_tables(h, s);
    // bf16 S|R images for the offset-stationary few-column tensor-core M2L (BF16x3)
    if (m2l_ofs_supported(h) && !h->opt.fp32_only) build_ofs_tables(h, s);
    if (h->opt.fp32_only) {  // single-precision tables only: the FP64 bases and matrices go
        CK(cudaStreamSynchronize(s));
        for (c64 **q : {&h->T_m2l64, &h->T_mm64, &h->T_ll64, &h->B_p2m64, &h->B_l2p64, &h->B_l2pg64}) {
            dev_free(h, *q);
            *q = nullptr;
        }
    }
}
