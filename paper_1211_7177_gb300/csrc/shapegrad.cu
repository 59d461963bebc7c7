// shapegrad.cu -- gradient of a linear functional of the solution with respect to the mesh
// vertex positions (vertex nodes), by the adjoint method of the discrete system of Eq. (2.9).
//
// For A(V) x = b(V), a functional f = L(V)^T x and the adjoint A^T lambda = L,
//   df/dtheta = d/dtheta [ L^T x + lambda^T b - lambda^T A x ]   at fixed x and lambda
// for every vertex coordinate theta.  The vertex positions enter through the node data (position
// s_u, weight w_u, normal n_u) of the nodes of the vertex's 1-ring and through their self blocks
// (Appendix B).  Here the sensitivities of G = L^T x + lambda^T b - lambda^T A x to the node data
// of every node are summed over all partners (the pair blocks of Eq. 2.12 depend on s_a, s_b,
// w_b and n_b), by closed-form pair derivatives (FP64 for pairs closer than 8 mean edge lengths,
// FP32 beyond), O(N^2) pair evaluations in all;
// k_vertex_shape_grad (geometry.cu) then chains them with the node data of each vertex's 1-ring
// and adds the self blocks' change.
#include <algorithm>

#include "fmbem_internal.cuh"

namespace {

struct DomainC {  // per domain, as in the matvec: k, t = (eps_0 - eps_d)/eps_d, gamma
    c64 k, t, gamma;
};

__device__ __forceinline__ double dot3d(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
template <typename T>
__device__ __forceinline__ T dot3(const T *a, const T *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
template <typename T>
__device__ __forceinline__ cx<T> cexp_t(cx<T> z);
template <>
__device__ __forceinline__ c64 cexp_t<double>(c64 z) { return cexpd(z); }
template <>
__device__ __forceinline__ c32 cexp_t<float>(c32 z) {
    float sn, cs;
    sincosf(z.im, &sn, &cs);
    const float e = expf(z.re);
    return c32{e * cs, e * sn};
}

// lambda_a . (pair block of Eq. 2.12 for target a, source b) x_b with r = s_b - s_a (val): the
// background side always (normal -n_b, Psi^(0) = -Psi), the scatterer side when a and b share
// scatterer j; and its derivatives with respect to r (gr) and, if gn != nullptr, to the source
// normal n_b (as a free vector, unnormalised), in closed form: with
// g = e^{ikR}/(4 pi R) and c = g (ik - 1/R)/R, grad_r g = c r and grad_r c = c2 r with
// c2 = g (-k^2/R^2 - 3ik/R^3 + 3/R^4); the brackets are linear in r and n (the scatterer side's
// density v = Phi + t n (n.Phi) depends on n too).  One exponential per domain instead of the
// central differences' 2 per derivative.
template <typename T>
__device__ void pair_grad(const T *r, T wb, const T *nb, bool same, cx<T> k0, cx<T> kj, cx<T> tj, cx<T> gj,
                          const cx<T> *la, const cx<T> *xb, cx<T> *val, cx<T> *gr, cx<T> *gn) {
    using C = cx<T>;
    const T R2 = dot3<T>(r, r), R = sqrt(R2);
    const T iR = (T)1 / R;
    const C *Phi = xb, *Psi = xb + 3;
    const T nr = dot3<T>(nb, r);
    C v0 = {0, 0}, g3[3] = {{0, 0}, {0, 0}, {0, 0}}, n3[3] = {{0, 0}, {0, 0}, {0, 0}};
    {
        const C ik = {-k0.im, k0.re};
        const C g = cexp_t<T>(ik * R) * (iR / (T)(4.0 * FMBEM_PI));
        const C c = g * (ik - C{iR, 0}) * iR;
        const C c2 = g * ((ik * ik) * (iR * iR) - ik * ((T)3 * iR * iR * iR) + C{(T)3 * iR * iR * iR * iR, 0});
        const C rP = r[0] * Phi[0] + r[1] * Phi[1] + r[2] * Phi[2];
        const C nP = nb[0] * Phi[0] + nb[1] * Phi[1] + nb[2] * Phi[2];
        const C lP = la[0] * Phi[0] + la[1] * Phi[1] + la[2] * Phi[2];
        const C lPs = la[0] * Psi[0] + la[1] * Psi[1] + la[2] * Psi[2];
        const C ln = la[0] * nb[0] + la[1] * nb[1] + la[2] * nb[2];
        const C lr = la[0] * r[0] + la[1] * r[1] + la[2] * r[2];
        // lambda . beta with beta_q = -n_q (r.Phi) + (n.r) Phi_q + r_q (n.Phi)
        const C lb = -(ln * rP) + nr * lP + lr * nP;
        v0 = -wb * (c * lb + g * lPs);
        for (int j = 0; j < 3; ++j) {
            g3[j] = -wb * (c2 * lb * r[j] + c * (-(ln * Phi[j]) + nb[j] * lP + la[j] * nP) + c * lPs * r[j]);
            n3[j] = -wb * (c * (-(la[j] * rP) + r[j] * lP + lr * Phi[j]));
        }
    }
    if (same) {
        const C ik = {-kj.im, kj.re};
        const C g = cexp_t<T>(ik * R) * (iR / (T)(4.0 * FMBEM_PI));
        const C c = g * (ik - C{iR, 0}) * iR;
        const C c2 = g * ((ik * ik) * (iR * iR) - ik * ((T)3 * iR * iR * iR) + C{(T)3 * iR * iR * iR * iR, 0});
        const C *l = la + 3;
        const C nP0 = nb[0] * Phi[0] + nb[1] * Phi[1] + nb[2] * Phi[2];
        const C tn = tj * nP0;
        C v[3];
        for (int q = 0; q < 3; ++q) v[q] = Phi[q] + nb[q] * tn;  // T_j Phi (Eq. 2.13)
        const C rv = r[0] * v[0] + r[1] * v[1] + r[2] * v[2];
        const C nv = nb[0] * v[0] + nb[1] * v[1] + nb[2] * v[2];
        const C lv = l[0] * v[0] + l[1] * v[1] + l[2] * v[2];
        const C ln = l[0] * nb[0] + l[1] * nb[1] + l[2] * nb[2];
        const C lr = l[0] * r[0] + l[1] * r[1] + l[2] * r[2];
        const C lPs = l[0] * Psi[0] + l[1] * Psi[1] + l[2] * Psi[2];
        const T nn = dot3<T>(nb, nb);
        // lambda' . beta' with beta'_q = n_q (r.v) - (n.r) v_q - r_q (n.v)
        const C lb = ln * rv - nr * lv - lr * nv;
        v0 += -wb * (c * lb) + (gj * g) * wb * lPs;
        for (int j = 0; j < 3; ++j) {
            g3[j] += -wb * (c2 * lb * r[j] + c * (ln * v[j] - nb[j] * lv - l[j] * nv)) + (gj * c) * wb * lPs * r[j];
            const C drv = tj * (r[j] * nP0 + nr * Phi[j]);                // d(r.v)/dn_j
            const C dnv = v[j] + tj * (nb[j] * nP0 + nn * Phi[j]);         // d(n.v)/dn_j
            const C dlv = tj * (l[j] * nP0 + ln * Phi[j]);                 // d(lambda'.v)/dn_j
            const C dlb = l[j] * rv + ln * drv - r[j] * lv - nr * dlv - lr * dnv;
            n3[j] += -wb * (c * dlb);
        }
    }
    *val = v0;
    for (int j = 0; j < 3; ++j) {
        gr[j] = g3[j];
        if (gn) gn[j] = n3[j];
    }
}

// partial sensitivities of G's pair part over one slice of partners (closed-form pair derivatives,
// pair_grad): part[slice][r][u][7] = dG/d(s_u (3), w_u, n_u (3)); grid (node tiles, slices, rhs).
// Pairs farther apart than far_r take the derivatives in single precision (their terms are smooth
// and small against the near pairs', where the kernel's 1/R^3 growth makes double precision
// count); each tile's single-precision sums are added to the double accumulators.
constexpr int SG_NT = 128, SG_NS = 32;
__global__ void __launch_bounds__(SG_NT) k_node_sens(int64_t N, int64_t nr, const double *pos, const double *nrm,
                                                   const double *w, const int32_t *dom, const DomainC *dc,
                                                   const c64 *x, const c64 *lam, int64_t slice_len, double far_r,
                                                   c64 *part) {
    __shared__ double sp[SG_NS][3], sn[SG_NS][3], sw[SG_NS];
    __shared__ int sd[SG_NS];
    __shared__ c64 sx[SG_NS][6], sl[SG_NS][6];
    __shared__ c32 sx32[SG_NS][6], sl32[SG_NS][6];
    const int64_t u = blockIdx.x * (int64_t)SG_NT + threadIdx.x, slice = blockIdx.y, r = blockIdx.z;
    const bool valid = u < N;
    double su[3] = {0, 0, 0}, nu[3] = {0, 0, 1}, wu = 1;
    int du = 0;
    c64 xu[6], lu[6];
    c32 xu32[6], lu32[6];
    for (int q = 0; q < 6; ++q) { xu[q] = {0, 0}; lu[q] = {0, 0}; }
    if (valid) {
        for (int q = 0; q < 3; ++q) { su[q] = pos[3 * u + q]; nu[q] = nrm[3 * u + q]; }
        wu = w[u];
        du = dom[u];
        for (int q = 0; q < 6; ++q) { xu[q] = x[(r * N + u) * 6 + q]; lu[q] = lam[(r * N + u) * 6 + q]; }
    }
    for (int q = 0; q < 6; ++q) { xu32[q] = to<float>(xu[q]); lu32[q] = to<float>(lu[q]); }
    const c64 k0 = dc[0].k, kj = dc[du].k, tj = dc[du].t, gj = dc[du].gamma;
    const c32 k0f = to<float>(k0), kjf = to<float>(kj), tjf = to<float>(tj), gjf = to<float>(gj);
    const float nuf[3] = {(float)nu[0], (float)nu[1], (float)nu[2]}, wuf = (float)wu;
    const double far2 = far_r * far_r;
    const int64_t b0s = slice * slice_len, b1s = min(N, b0s + slice_len);
    c64 acc[7];
    for (int q = 0; q < 7; ++q) acc[q] = {0, 0};
    for (int64_t b0 = b0s; b0 < b1s; b0 += SG_NS) {
        const int nb = (int)min((int64_t)SG_NS, b1s - b0);
        __syncthreads();
        for (int e = threadIdx.x; e < nb; e += blockDim.x) {
            const int64_t m = b0 + e;
            for (int q = 0; q < 3; ++q) { sp[e][q] = pos[3 * m + q]; sn[e][q] = nrm[3 * m + q]; }
            sw[e] = w[m];
            sd[e] = dom[m];
            for (int q = 0; q < 6; ++q) {
                sx[e][q] = x[(r * N + m) * 6 + q];
                sl[e][q] = lam[(r * N + m) * 6 + q];
                sx32[e][q] = to<float>(sx[e][q]);
                sl32[e][q] = to<float>(sl[e][q]);
            }
        }
        __syncthreads();
        if (!valid) continue;
        c32 accf[7];
        for (int q = 0; q < 7; ++q) accf[q] = {0, 0};
        for (int e = 0; e < nb; ++e) {
            if (b0 + e == u) continue;
            const bool same = sd[e] == du;
            const double rt[3] = {sp[e][0] - su[0], sp[e][1] - su[1], sp[e][2] - su[2]};
            if (dot3d(rt, rt) > far2) {
                const float rf[3] = {(float)rt[0], (float)rt[1], (float)rt[2]};
                const float rs[3] = {-rf[0], -rf[1], -rf[2]};
                const float snf[3] = {(float)sn[e][0], (float)sn[e][1], (float)sn[e][2]};
                c32 val, gr[3], gn[3];
                pair_grad<float>(rf, (float)sw[e], snf, same, k0f, kjf, tjf, gjf, lu32, sx32[e], &val, gr, nullptr);
                for (int c = 0; c < 3; ++c) accf[c] += gr[c];
                pair_grad<float>(rs, wuf, nuf, same, k0f, kjf, tjf, gjf, sl32[e], xu32, &val, gr, gn);
                for (int c = 0; c < 3; ++c) {
                    accf[c] -= gr[c];
                    accf[4 + c] -= gn[c];
                }
                accf[3] -= val * (1.0f / wuf);
                continue;
            }
            c64 val, gr[3], gn[3];
            // u as the target: r = s_m - s_u, dG/ds_u = +dt/dr (G holds -t)
            pair_grad<double>(rt, sw[e], sn[e], same, k0, kj, tj, gj, lu, sx[e], &val, gr, nullptr);
            for (int c = 0; c < 3; ++c) acc[c] += gr[c];
            // u as the source: r = s_u - s_m, dG/ds_u = -dsigma/dr, dG/dn_u, dG/dw_u = -sigma / w_u
            const double rs[3] = {-rt[0], -rt[1], -rt[2]};
            pair_grad<double>(rs, wu, nu, same, k0, kj, tj, gj, sl[e], xu, &val, gr, gn);
            for (int c = 0; c < 3; ++c) {
                acc[c] -= gr[c];
                acc[4 + c] -= gn[c];
            }
            acc[3] -= val * (1.0 / wu);
        }
        for (int q = 0; q < 7; ++q) acc[q] += c64{(double)accf[q].re, (double)accf[q].im};
    }
    if (valid)
        for (int q = 0; q < 7; ++q) part[((slice * nr + r) * N + u) * 7 + q] = acc[q];
}

// far-field functional value L_u(s, w, n) . x_u (the coefficients of fmbem_far_field_functional)
__device__ c64 ff_functional(const double *s, double w, const double *n, c64 k0, const double *u, const c64 *c,
                             const c64 *xu) {
    const c64 mik = {k0.im, -k0.re};  // -i k0
    const double n0[3] = {-n[0], -n[1], -n[2]};
    const c64 f = cexpd(mik * dot3d(u, s)) * (w / (4.0 * FMBEM_PI));
    const c64 cn = c[0] * n0[0] + c[1] * n0[1] + c[2] * n0[2], cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
    const double nu = dot3d(n0, u);
    c64 val = {0, 0};
    for (int q = 0; q < 3; ++q) val += f * (mik * (cn * u[q] - nu * c[q] - cu * n0[q]) * xu[q] + c[q] * xu[3 + q]);
    return val;
}

// sens[r][u] = sum over slices + the local terms of G: the functional L_u . x_u and the right-
// hand side lambda_u . e exp(i k0 d.s_u) (background rows, Eq. 2.12); thread per (node, rhs)
__global__ void k_node_sens_reduce(int64_t N, int64_t nr, int n_slices, const c64 *part, const double *pos,
                                   const double *nrm, const double *w, c64 k0, const double *dir, const c64 *pol,
                                   const double *rhat, const c64 *coef, const c64 *x, const c64 *lam, double hs,
                                   double hn, c64 *sens) {
    const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, r = blockIdx.y;
    if (u >= N) return;
    c64 acc[7];
    for (int q = 0; q < 7; ++q) acc[q] = {0, 0};
    for (int sl = 0; sl < n_slices; ++sl)
        for (int q = 0; q < 7; ++q) acc[q] += part[(((int64_t)sl * nr + r) * N + u) * 7 + q];
    const double s[3] = {pos[3 * u], pos[3 * u + 1], pos[3 * u + 2]}, n[3] = {nrm[3 * u], nrm[3 * u + 1], nrm[3 * u + 2]};
    const double wu = w[u];
    const c64 *xu = x + (r * N + u) * 6, *lu = lam + (r * N + u) * 6;
    {  // right-hand side
        const double *d = dir + 3 * r;
        const c64 *e = pol + 3 * r;
        const c64 ik = {-k0.im, k0.re};
        const c64 ph = cexpd(ik * dot3d(d, s));
        const c64 le = lu[0] * e[0] + lu[1] * e[1] + lu[2] * e[2];
        for (int c = 0; c < 3; ++c) acc[c] += ik * le * ph * d[c];
    }
    if (rhat != nullptr) {  // far-field functional
        const double *ud = rhat + 3 * r;
        const c64 *cf = coef + 3 * r;
        const double i2s = 1.0 / (2.0 * hs), i2n = 1.0 / (2.0 * hn);
        for (int c = 0; c < 3; ++c) {
            double sp_[3] = {s[0], s[1], s[2]}, sm[3] = {s[0], s[1], s[2]};
            sp_[c] += hs;
            sm[c] -= hs;
            acc[c] += (ff_functional(sp_, wu, n, k0, ud, cf, xu) - ff_functional(sm, wu, n, k0, ud, cf, xu)) * i2s;
            double np_[3] = {n[0], n[1], n[2]}, nm[3] = {n[0], n[1], n[2]};
            np_[c] += hn;
            nm[c] -= hn;
            acc[4 + c] += (ff_functional(s, wu, np_, k0, ud, cf, xu) - ff_functional(s, wu, nm, k0, ud, cf, xu)) * i2n;
        }
        acc[3] += ff_functional(s, wu, n, k0, ud, cf, xu) * (1.0 / wu);
    }
    for (int q = 0; q < 7; ++q) sens[(r * N + u) * 7 + q] = acc[q];
}

// node u's part of sum_p cE_p . E_sca(r_p) + cH_p . H_sca(r_p) with its own data (s, w, n): the
// representation formula of fmbem_near_field (background normal -n, Psi^(0) = -Psi) and its curl
__device__ c64 nf_val(const double *t, const double *s, double w, const double *n, const c64 *xu, c64 k0, c64 iwmu,
                      const c64 *cE, const c64 *cH) {
    const double rv[3] = {s[0] - t[0], s[1] - t[1], s[2] - t[2]};
    const double R = sqrt(dot3d(rv, rv)), iR = 1.0 / R;
    const c64 ik = {-k0.im, k0.re};
    const c64 g = cexpd(ik * R) * (iR / (4.0 * FMBEM_PI));
    const c64 g1 = g * (ik - c64{iR, 0});
    const c64 c = g1 * iR;
    const double n0[3] = {-n[0], -n[1], -n[2]};
    const c64 *Phi = xu, *Psi = xu + 3;
    const c64 rP = rv[0] * Phi[0] + rv[1] * Phi[1] + rv[2] * Phi[2];
    const c64 nP = n0[0] * Phi[0] + n0[1] * Phi[1] + n0[2] * Phi[2];
    const double nr = dot3d(n0, rv);
    c64 val = {0, 0};
    for (int q = 0; q < 3; ++q) val += cE[q] * (w * (c * (n0[q] * rP - nr * Phi[q] - rv[q] * nP) + g * Psi[q]));
    if (cH != nullptr) {
        const double rh[3] = {rv[0] * iR, rv[1] * iR, rv[2] * iR};
        const c64 q1 = ik - c64{iR, 0};
        const c64 g2 = g * (q1 * q1 + c64{iR * iR, 0});
        const double rn = dot3d(rh, n0);
        const c64 rhP = rP * iR;
        c64 Kn[3], KP[3], av[3];
        for (int q = 0; q < 3; ++q) {
            Kn[q] = g2 * (rh[q] * rn) + c * (n0[q] - rh[q] * rn);
            KP[q] = g2 * rhP * rh[q] + c * (Phi[q] - rhP * rh[q]);
            av[q] = g1 * rh[q];
        }
        const c64 cur[3] = {Kn[1] * Phi[2] - Kn[2] * Phi[1] + n0[1] * KP[2] - n0[2] * KP[1] - (av[1] * Psi[2] - av[2] * Psi[1]),
                            Kn[2] * Phi[0] - Kn[0] * Phi[2] + n0[2] * KP[0] - n0[0] * KP[2] - (av[2] * Psi[0] - av[0] * Psi[2]),
                            Kn[0] * Phi[1] - Kn[1] * Phi[0] + n0[0] * KP[1] - n0[1] * KP[0] - (av[0] * Psi[1] - av[1] * Psi[0])};
        for (int q = 0; q < 3; ++q) val += cH[q] * cdiv(cur[q] * w, iwmu);
    }
    return val;
}

// adds to sens[r][u] the derivatives of node u's part of the near-field functional of right-hand
// side r with respect to its position, weight and normal; thread per (node, rhs), the points
// staged in shared memory SG_NS at a time
__global__ void __launch_bounds__(SG_NT) k_node_sens_near(int64_t N, int64_t nr, const double *pos,
                                                        const double *nrm, const double *w, const c64 *x,
                                                        int64_t n_pts, const double *pts, const c64 *cE,
                                                        const c64 *cH, c64 k0, c64 iwmu, double hs,
                                                        int64_t pslice_len, c64 *part) {
    __shared__ double spt[SG_NS][3];
    __shared__ c64 sce[SG_NS][3], sch[SG_NS][3];
    const int64_t u = blockIdx.x * (int64_t)SG_NT + threadIdx.x, r = blockIdx.y, slice = blockIdx.z;
    const int64_t pb = slice * pslice_len, pe = min(n_pts, pb + pslice_len);
    const bool valid = u < N;
    double s[3] = {0, 0, 0}, n[3] = {0, 0, 1}, wu = 1;
    c64 xu[6];
    for (int q = 0; q < 6; ++q) xu[q] = {0, 0};
    if (valid) {
        for (int q = 0; q < 3; ++q) { s[q] = pos[3 * u + q]; n[q] = nrm[3 * u + q]; }
        wu = w[u];
        for (int q = 0; q < 6; ++q) xu[q] = x[(r * N + u) * 6 + q];
    }
    c64 acc[7];
    for (int q = 0; q < 7; ++q) acc[q] = {0, 0};
    const double i2s = 1.0 / (2.0 * hs);
    for (int64_t p0 = pb; p0 < pe; p0 += SG_NS) {
        const int np = (int)min((int64_t)SG_NS, pe - p0);
        __syncthreads();
        for (int e = threadIdx.x; e < np; e += blockDim.x) {
            for (int q = 0; q < 3; ++q) {
                spt[e][q] = pts[3 * (p0 + e) + q];
                sce[e][q] = cE[(r * n_pts + p0 + e) * 3 + q];
                sch[e][q] = cH ? cH[(r * n_pts + p0 + e) * 3 + q] : c64{0, 0};
            }
        }
        __syncthreads();
        if (!valid) continue;
        for (int e = 0; e < np; ++e) {
            const c64 *ch = cH ? sch[e] : nullptr;
            // the functional is affine in the normal (the representation formula's kernel and its
            // curl are linear in n), val(n) = val(0) + sum_c n_c dval/dn_c: the normal derivatives
            // exactly from the unit normals, and the value from them
            const double zero[3] = {0, 0, 0};
            const c64 v0 = nf_val(spt[e], s, wu, zero, xu, k0, iwmu, sce[e], ch);
            c64 val = v0;
            for (int c = 0; c < 3; ++c) {
                double ec[3] = {0, 0, 0};
                ec[c] = 1;
                const c64 dn = nf_val(spt[e], s, wu, ec, xu, k0, iwmu, sce[e], ch) - v0;
                acc[4 + c] += dn;
                val += dn * n[c];
                double sp_[3] = {s[0], s[1], s[2]}, sm[3] = {s[0], s[1], s[2]};
                sp_[c] += hs;
                sm[c] -= hs;
                acc[c] += (nf_val(spt[e], sp_, wu, n, xu, k0, iwmu, sce[e], ch) -
                           nf_val(spt[e], sm, wu, n, xu, k0, iwmu, sce[e], ch)) * i2s;
            }
            acc[3] += val * (1.0 / wu);
        }
    }
    if (valid)
        for (int q = 0; q < 7; ++q) part[((slice * nr + r) * N + u) * 7 + q] = acc[q];
}

// sens[r][u] += sum over the point slices of k_node_sens_near's partial sums, fixed order
__global__ void k_node_sens_near_reduce(int64_t N, int64_t nr, int n_slices, const c64 *part, c64 *sens) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // (r, u, q)
    if (e >= nr * N * 7) return;
    c64 a = sens[e];
    for (int sl = 0; sl < n_slices; ++sl) a += part[sl * nr * N * 7 + e];
    sens[e] = a;
}

}  // namespace

void run_shape_gradient(fmbem *h, const c64 *x, const c64 *lam, int64_t nr, const double *dir_host,
                        const c64 *pol_host, const double *rhat_host, const c64 *coef_host, int64_t n_pts,
                        const double *pts_host, const c64 *cE_host, const c64 *cH_host, c64 *out_host,
                        cudaStream_t s) {
    if (h->opt.node_mode != FMBEM_NODES_VERTEX)
        throw fmbem_error{FMBEM_ERR_INVALID_ARGUMENT, "the shape gradient needs vertex nodes"};
    if (h->ibc) throw fmbem_error{FMBEM_ERR_INVALID_ARGUMENT, "the shape gradient is for penetrable scatterers"};
    const int64_t N = h->N;
    // finite-difference steps: positions 1e-6 of the mean edge length, normals 1e-6
    double ledge = 0;
    const int64_t nt = (int64_t)h->h_F.size() / 3;
    for (int64_t t = 0; t < nt; ++t)
        for (int a = 0; a < 3; ++a) {
            const double *A = &h->h_pos[3 * h->h_F[3 * t + a]], *B = &h->h_pos[3 * h->h_F[3 * t + (a + 1) % 3]];
            ledge += std::sqrt((A[0] - B[0]) * (A[0] - B[0]) + (A[1] - B[1]) * (A[1] - B[1]) + (A[2] - B[2]) * (A[2] - B[2]));
        }
    ledge /= (double)(3 * nt);
    const double hs = 1e-6 * ledge, hn = 1e-6;
    const int64_t ntile = (N + SG_NT - 1) / SG_NT;
    // partner slices (and point slices of the force's near-field functional): enough blocks for
    // about 16 per SM, so that the last wave is a small part of the launch
    const int n_slices = (int)std::max<int64_t>(1, std::min<int64_t>(64, (16 * 152 + ntile * nr - 1) / (ntile * nr)));
    const int64_t slice_len = (N + n_slices - 1) / n_slices;
    std::vector<c64> dch(3 * (h->J + 1));
    for (int d = 0; d <= h->J; ++d) {
        dch[3 * d] = h->k[d];
        dch[3 * d + 1] = d == 0 ? c64{0, 0} : cdiv(h->eps[0] - h->eps[d], h->eps[d]);
        dch[3 * d + 2] = h->gam[d];
    }
    DomainC *ddc = (DomainC *)dev_alloc(h, sizeof(c64) * dch.size());
    c64 *part = (c64 *)dev_alloc(h, sizeof(c64) * 7 * N * nr * n_slices);
    c64 *sens = (c64 *)dev_alloc(h, sizeof(c64) * 7 * N * nr);
    double *dd = (double *)dev_alloc(h, sizeof(double) * 3 * nr), *dr = (double *)dev_alloc(h, sizeof(double) * 3 * nr);
    c64 *dp = (c64 *)dev_alloc(h, sizeof(c64) * 3 * nr), *dcf = (c64 *)dev_alloc(h, sizeof(c64) * 3 * nr);
    c64 *dout = (c64 *)dev_alloc(h, sizeof(c64) * 3 * N * nr);
    const bool nearf = pts_host != nullptr;
    double *dpt = nearf ? (double *)dev_alloc(h, sizeof(double) * 3 * n_pts) : nullptr;
    c64 *dcE = nearf ? (c64 *)dev_alloc(h, sizeof(c64) * 3 * n_pts * nr) : nullptr;
    c64 *dcH = nearf && cH_host ? (c64 *)dev_alloc(h, sizeof(c64) * 3 * n_pts * nr) : nullptr;
    auto cleanup = [&] {
        for (void *p : {(void *)ddc, (void *)part, (void *)sens, (void *)dd, (void *)dr, (void *)dp, (void *)dcf,
                        (void *)dout, (void *)dpt, (void *)dcE, (void *)dcH})
            if (p) dev_free(h, p);
    };
    try {
        CK(cudaMemcpyAsync(ddc, dch.data(), sizeof(c64) * dch.size(), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dd, dir_host, sizeof(double) * 3 * nr, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dp, pol_host, sizeof(c64) * 3 * nr, cudaMemcpyHostToDevice, s));
        if (rhat_host) {
            CK(cudaMemcpyAsync(dr, rhat_host, sizeof(double) * 3 * nr, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(dcf, coef_host, sizeof(c64) * 3 * nr, cudaMemcpyHostToDevice, s));
        }
        if (nearf) {
            CK(cudaMemcpyAsync(dpt, pts_host, sizeof(double) * 3 * n_pts, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(dcE, cE_host, sizeof(c64) * 3 * n_pts * nr, cudaMemcpyHostToDevice, s));
            if (dcH) CK(cudaMemcpyAsync(dcH, cH_host, sizeof(c64) * 3 * n_pts * nr, cudaMemcpyHostToDevice, s));
        }
        k_node_sens<<<dim3((unsigned)ntile, (unsigned)n_slices, (unsigned)nr), SG_NT, 0, s>>>(
            N, nr, h->upos, h->unrm, h->uw, h->udom, ddc, x, lam, slice_len, 8.0 * ledge, part);
        CKL("k_node_sens");
        k_node_sens_reduce<<<dim3((unsigned)((N + 127) / 128), (unsigned)nr), 128, 0, s>>>(
            N, nr, n_slices, part, h->upos, h->unrm, h->uw, h->k[0], dd, dp, rhat_host ? dr : nullptr, dcf, x, lam, hs,
            hn, sens);
        CKL("k_node_sens_reduce");
        if (nearf) {
            const c64 iwmu = c64{0, h->k0} * h->mu[0];  // i omega mu_0 with omega = k0 (c = 1)
            // point slices into the partner-slice buffer (free again after k_node_sens_reduce)
            const int64_t pslice_len = (n_pts + n_slices - 1) / n_slices;
            k_node_sens_near<<<dim3((unsigned)ntile, (unsigned)nr, (unsigned)n_slices), SG_NT, 0, s>>>(
                N, nr, h->upos, h->unrm, h->uw, x, n_pts, dpt, dcE, dcH, h->k[0], iwmu, hs, pslice_len, part);
            CKL("k_node_sens_near");
            k_node_sens_near_reduce<<<(unsigned)((nr * N * 7 + 255) / 256), 256, 0, s>>>(N, nr, n_slices, part, sens);
            CKL("k_node_sens_near_reduce");
        }
        run_vertex_shape_grad(h, nr, x, lam, sens, hs, dout, s);
        CK(cudaMemcpyAsync(out_host, dout, sizeof(c64) * 3 * N * nr, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
}
