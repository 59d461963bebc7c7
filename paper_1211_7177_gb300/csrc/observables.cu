// observables.cu -- quantities of a solution: the total field at exterior points and the far-field
// amplitude of the scattered field (Section 4; representation formula of Appendix A, near and in
// the far zone), and the absorbed power (Eq. 4.2).
//
// Far field: with n0 = -n (the outward normal of the background) and Psi0 = -Psi,
//   F(u) = 1/(4 pi) sum_b w_b exp(-i k0 u.s_b) { (-i k0) [n0 (u.Phi_b) - (n0.u) Phi_b - u (n0.Phi_b)]
//                                                 - Psi0_b },
// so that the scattered field behaves as E_sca ~ exp(i k0 r)/r F(u) in direction u.
// Absorption: the inward flux of the time-averaged Poynting vector through the surface, Eq. (4.2),
// with n x curl E = Psi, reduces to C_abs = -(1/k0) sum_b w_b Im(Phi_b . conj(Psi_b)).
#include <string>
#include <vector>

#include "fmbem_internal.cuh"
#include "special.cuh"

namespace {

constexpr int OB_TB = 256;

// F[r][dir][3]; grid (direction, right-hand side), nodes in user order
__global__ void __launch_bounds__(OB_TB) k_far_field(int64_t N, const double *pos, const double *nrm, const double *w,
                                                   const c64 *x, const double *rhat, c64 k0, int64_t n_dir, c64 *F) {
    __shared__ double red[6][OB_TB];
    const int64_t dir = blockIdx.x, r = blockIdx.y;
    const double u[3] = {rhat[3 * dir], rhat[3 * dir + 1], rhat[3 * dir + 2]};
    const c64 mik = c64{k0.im, -k0.re};  // -i k0
    c64 acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int64_t b = threadIdx.x; b < N; b += blockDim.x) {
        const double n0[3] = {-nrm[3 * b], -nrm[3 * b + 1], -nrm[3 * b + 2]};
        const c64 *Phi = x + (r * N + b) * 6, *Psi = Phi + 3;
        const double us = u[0] * pos[3 * b] + u[1] * pos[3 * b + 1] + u[2] * pos[3 * b + 2];
        const c64 ph = cexpd(mik * us) * w[b];
        const c64 uP = u[0] * Phi[0] + u[1] * Phi[1] + u[2] * Phi[2];
        const c64 nP = n0[0] * Phi[0] + n0[1] * Phi[1] + n0[2] * Phi[2];
        const double nu = n0[0] * u[0] + n0[1] * u[1] + n0[2] * u[2];
        for (int q = 0; q < 3; ++q) {
            const c64 br = n0[q] * uP - nu * Phi[q] - u[q] * nP;
            acc[q] += ph * (mik * br + Psi[q]);
        }
    }
    for (int q = 0; q < 3; ++q) {
        red[2 * q][threadIdx.x] = acc[q].re;
        red[2 * q + 1][threadIdx.x] = acc[q].im;
    }
    __syncthreads();
    for (int off = OB_TB / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off)
            for (int e = 0; e < 6; ++e) red[e][threadIdx.x] += red[e][threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x < 3) {
        const double s = 1.0 / (4.0 * FMBEM_PI);
        F[(r * n_dir + dir) * 3 + threadIdx.x] = c64{red[2 * threadIdx.x][0] * s, red[2 * threadIdx.x + 1][0] * s};
    }
}

// Coefficients of the linear functional x -> c_r . F(u_r) of each right-hand side's solution:
// out[r][b] = (d/dPhi_b, d/dPsi_b) of 1/(4 pi) w_b e_b { -i k0 [(c.n0)(u.Phi_b) - (n0.u)(c.Phi_b)
// - (c.u)(n0.Phi_b)] + c.Psi_b }, e_b = exp(-i k0 u.s_b), so that c . F(u) = sum_b out[r][b] . x_b
// (no conjugation).  One thread per (node, right-hand side), nodes in user order.
__global__ void k_far_field_functional(int64_t N, int64_t nr, const double *pos, const double *nrm, const double *w,
                                       const double *rhat, const c64 *coef, c64 k0, c64 *out) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, r = blockIdx.y;
    if (b >= N) return;
    const double u[3] = {rhat[3 * r], rhat[3 * r + 1], rhat[3 * r + 2]};
    const c64 c[3] = {coef[3 * r], coef[3 * r + 1], coef[3 * r + 2]};
    const double n0[3] = {-nrm[3 * b], -nrm[3 * b + 1], -nrm[3 * b + 2]};
    const c64 mik = c64{k0.im, -k0.re};  // -i k0
    const double us = u[0] * pos[3 * b] + u[1] * pos[3 * b + 1] + u[2] * pos[3 * b + 2];
    const c64 f = cexpd(mik * us) * (w[b] / (4.0 * FMBEM_PI));
    const c64 cn = c[0] * n0[0] + c[1] * n0[1] + c[2] * n0[2], cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
    const double nu = n0[0] * u[0] + n0[1] * u[1] + n0[2] * u[2];
    c64 *o = out + (r * N + b) * 6;
    for (int q = 0; q < 3; ++q) {
        o[q] = f * mik * (cn * u[q] - nu * c[q] - cu * n0[q]);
        o[3 + q] = f * c[q];
    }
}

// out[r] = sum_b w_b Im(Phi_b . conj(Psi_b)); one block per right-hand side
__global__ void __launch_bounds__(OB_TB) k_absorption(int64_t N, const double *w, const c64 *x, double *out) {
    __shared__ double red[OB_TB];
    const int64_t r = blockIdx.x;
    double acc = 0;
    for (int64_t b = threadIdx.x; b < N; b += blockDim.x) {
        const c64 *xb = x + (r * N + b) * 6;
        double im = 0;
        for (int q = 0; q < 3; ++q) im += xb[3 + q].re * xb[q].im - xb[3 + q].im * xb[q].re;  // Im(Phi conj(Psi))
        acc += w[b] * im;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int off = OB_TB / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[r] = red[0];
}

// Total fields at exterior points, direct summation over the nodes (see fmbem_near_field): one
// thread per point, a block per (tile of OB_NT points, right-hand side), the nodes staged in
// shared memory OB_NS at a time.  With the magnetic field, curl E is summed beside E (the curl
// of the bracket is (K n0) x Phi + n0 x (K Phi) with K the Hessian of g in the source point, the
// curl of g Psi is -grad_s g x Psi) and H = curl E / (i k0 mu_0).  No incident plane wave when
// dir is null.
constexpr int OB_NT = 128, OB_NS = 64;
template <bool WITH_H>
__global__ void __launch_bounds__(OB_NT) k_near_field(int64_t N, const double *pos, const double *nrm, const double *w,
                                                    const c64 *x, int64_t n_pts, const double *pts, c64 k0,
                                                    c64 iwmu, const double *dir, const c64 *pol, c64 *E, c64 *H) {
    __shared__ double sp[OB_NS][3], sn[OB_NS][3], sw[OB_NS];
    __shared__ c64 sx[OB_NS][6];
    const int64_t pt = blockIdx.x * (int64_t)OB_NT + threadIdx.x, r = blockIdx.y;
    const bool valid = pt < n_pts;
    const double t[3] = {valid ? pts[3 * pt] : 0.0, valid ? pts[3 * pt + 1] : 0.0, valid ? pts[3 * pt + 2] : 0.0};
    const c64 ik = {-k0.im, k0.re};
    c64 acc[3] = {{0, 0}, {0, 0}, {0, 0}}, cur[3] = {{0, 0}, {0, 0}, {0, 0}};
    if (dir != nullptr && pol != nullptr) {  // incident plane wave e exp(i k0 d.r), curl i k0 d x e exp(..)
        const double *d = dir + 3 * r;
        const c64 *e = pol + 3 * r;
        const c64 ph = cexpd(ik * (d[0] * t[0] + d[1] * t[1] + d[2] * t[2]));
        for (int q = 0; q < 3; ++q) acc[q] = e[q] * ph;
        if (WITH_H) {
            const c64 de[3] = {d[1] * e[2] - d[2] * e[1], d[2] * e[0] - d[0] * e[2], d[0] * e[1] - d[1] * e[0]};
            for (int q = 0; q < 3; ++q) cur[q] = ik * de[q] * ph;
        }
    }
    for (int64_t b0 = 0; b0 < N; b0 += OB_NS) {
        const int nb = (int)min((int64_t)OB_NS, N - b0);
        __syncthreads();
        for (int e = threadIdx.x; e < nb; e += blockDim.x) {
            const int64_t b = b0 + e;
            for (int q = 0; q < 3; ++q) { sp[e][q] = pos[3 * b + q]; sn[e][q] = -nrm[3 * b + q]; }
            sw[e] = w[b];
        }
        for (int e = threadIdx.x; e < 6 * nb; e += blockDim.x) sx[e / 6][e % 6] = x[(r * N + b0) * 6 + e];
        __syncthreads();
        if (!valid) continue;
        for (int e = 0; e < nb; ++e) {
            const double rv[3] = {sp[e][0] - t[0], sp[e][1] - t[1], sp[e][2] - t[2]};
            const double R = sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
            const c64 g = cexpd(ik * R) * (1.0 / (4.0 * FMBEM_PI * R));
            const c64 g1 = g * (ik - c64{1.0 / R, 0});  // dg/dR
            const c64 c = g1 * (1.0 / R);                // grad_s g = c (s - r)
            const double *n0 = sn[e];
            const c64 *Phi = sx[e], *Psi = sx[e] + 3;
            const c64 rP = rv[0] * Phi[0] + rv[1] * Phi[1] + rv[2] * Phi[2];
            const c64 nP = n0[0] * Phi[0] + n0[1] * Phi[1] + n0[2] * Phi[2];
            const double nr = n0[0] * rv[0] + n0[1] * rv[1] + n0[2] * rv[2];
            for (int q = 0; q < 3; ++q) {
                // n0 (a.Phi) - (n0.a) Phi - a (n0.Phi) with a = c rv, plus g Psi
                const c64 br = c * (n0[q] * rP - nr * Phi[q] - rv[q] * nP);
                acc[q] += sw[e] * (br + g * Psi[q]);
            }
            if (WITH_H) {
                // K v = g'' rh (rh.v) + g'/R (v - rh (rh.v)), rh = rv / R
                const double iR = 1.0 / R, rh[3] = {rv[0] * iR, rv[1] * iR, rv[2] * iR};
                const c64 q1 = ik - c64{iR, 0};
                const c64 g2 = g * (q1 * q1 + c64{iR * iR, 0});
                const double rn = rh[0] * n0[0] + rh[1] * n0[1] + rh[2] * n0[2];
                const c64 rhP = rP * iR;
                c64 Kn[3], KP[3], av[3];
                for (int q = 0; q < 3; ++q) {
                    Kn[q] = g2 * (rh[q] * rn) + c * (n0[q] - rh[q] * rn);
                    KP[q] = g2 * rhP * rh[q] + c * (Phi[q] - rhP * rh[q]);
                    av[q] = g1 * rh[q];
                }
                cur[0] += sw[e] * (Kn[1] * Phi[2] - Kn[2] * Phi[1] + n0[1] * KP[2] - n0[2] * KP[1] - (av[1] * Psi[2] - av[2] * Psi[1]));
                cur[1] += sw[e] * (Kn[2] * Phi[0] - Kn[0] * Phi[2] + n0[2] * KP[0] - n0[0] * KP[2] - (av[2] * Psi[0] - av[0] * Psi[2]));
                cur[2] += sw[e] * (Kn[0] * Phi[1] - Kn[1] * Phi[0] + n0[0] * KP[1] - n0[1] * KP[0] - (av[0] * Psi[1] - av[1] * Psi[0]));
            }
        }
    }
    if (valid) {
        for (int q = 0; q < 3; ++q) E[(r * n_pts + pt) * 3 + q] = acc[q];
        if (WITH_H)
            for (int q = 0; q < 3; ++q) H[(r * n_pts + pt) * 3 + q] = cdiv(cur[q], iwmu);
    }
}

// Fields inside the scatterers (see fmbem_interior_field): the representation formula of the
// point's own scatterer domain j, summed over that scatterer's nodes,
//   E = sum_b w_b { [n (a.v) - (n.a) v - a (n.v)] - g_j q },   v = T_j Phi_b (Eq. 2.6),
//   q = gamma_j Psi_b (Eq. 2.7), n the scatterer's outward normal, a = grad_s g_j;
// curl E sums (K n) x v + n x (K v) + a x q (K the Hessian of g_j in the source point), and
// H = curl E / (i k0 mu_j).  Thread and staging layout as k_near_field: the nodes are staged with
// v and q already formed, and each thread skips the nodes of the other scatterers.
// dcon[4 d .. 4 d + 3] = (k_d, t_d, gamma_d, i k0 mu_d).
template <bool WITH_H>
__global__ void __launch_bounds__(OB_NT) k_interior_field(int64_t N, const double *pos, const double *nrm,
                                                        const double *w, const int32_t *ndom, const c64 *x,
                                                        int64_t n_pts, const double *pts, const int32_t *pdom,
                                                        const c64 *dcon, c64 *E, c64 *H) {
    __shared__ double sp[OB_NS][3], sn[OB_NS][3], sw[OB_NS];
    __shared__ c64 sx[OB_NS][6];
    __shared__ int sd[OB_NS];
    const int64_t pt = blockIdx.x * (int64_t)OB_NT + threadIdx.x, r = blockIdx.y;
    const bool valid = pt < n_pts;
    const double t[3] = {valid ? pts[3 * pt] : 0.0, valid ? pts[3 * pt + 1] : 0.0, valid ? pts[3 * pt + 2] : 0.0};
    const int j = valid ? pdom[pt] : -1;
    const c64 k = valid ? dcon[4 * j] : c64{0, 0};
    const c64 ik = {-k.im, k.re};
    c64 acc[3] = {{0, 0}, {0, 0}, {0, 0}}, cur[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int64_t b0 = 0; b0 < N; b0 += OB_NS) {
        const int nb = (int)min((int64_t)OB_NS, N - b0);
        __syncthreads();
        for (int e = threadIdx.x; e < nb; e += blockDim.x) {
            const int64_t b = b0 + e;
            const int d = ndom[b];
            const double n[3] = {nrm[3 * b], nrm[3 * b + 1], nrm[3 * b + 2]};
            for (int q = 0; q < 3; ++q) { sp[e][q] = pos[3 * b + q]; sn[e][q] = n[q]; }
            sw[e] = w[b];
            sd[e] = d;
            const c64 *xb = x + (r * N + b) * 6;
            const c64 td = dcon[4 * d + 1], gd = dcon[4 * d + 2];
            const c64 tn = td * (n[0] * xb[0] + n[1] * xb[1] + n[2] * xb[2]);
            for (int q = 0; q < 3; ++q) {
                sx[e][q] = xb[q] + n[q] * tn;
                sx[e][3 + q] = gd * xb[3 + q];
            }
        }
        __syncthreads();
        if (!valid) continue;
        for (int e = 0; e < nb; ++e) {
            if (sd[e] != j) continue;
            const double rv[3] = {sp[e][0] - t[0], sp[e][1] - t[1], sp[e][2] - t[2]};
            const double R = sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
            const c64 g = cexpd(ik * R) * (1.0 / (4.0 * FMBEM_PI * R));
            const c64 g1 = g * (ik - c64{1.0 / R, 0});  // dg/dR
            const c64 c = g1 * (1.0 / R);                // grad_s g = c (s - r)
            const double *n = sn[e];
            const c64 *v = sx[e], *qv = sx[e] + 3;
            const c64 rP = rv[0] * v[0] + rv[1] * v[1] + rv[2] * v[2];
            const c64 nP = n[0] * v[0] + n[1] * v[1] + n[2] * v[2];
            const double nr = n[0] * rv[0] + n[1] * rv[1] + n[2] * rv[2];
            for (int q = 0; q < 3; ++q) {
                const c64 br = c * (n[q] * rP - nr * v[q] - rv[q] * nP);
                acc[q] += sw[e] * (br - g * qv[q]);
            }
            if (WITH_H) {
                const double iR = 1.0 / R, rh[3] = {rv[0] * iR, rv[1] * iR, rv[2] * iR};
                const c64 q1 = ik - c64{iR, 0};
                const c64 g2 = g * (q1 * q1 + c64{iR * iR, 0});
                const double rn = rh[0] * n[0] + rh[1] * n[1] + rh[2] * n[2];
                const c64 rhP = rP * iR;
                c64 Kn[3], KP[3], av[3];
                for (int q = 0; q < 3; ++q) {
                    Kn[q] = g2 * (rh[q] * rn) + c * (n[q] - rh[q] * rn);
                    KP[q] = g2 * rhP * rh[q] + c * (v[q] - rhP * rh[q]);
                    av[q] = g1 * rh[q];
                }
                cur[0] += sw[e] * (Kn[1] * v[2] - Kn[2] * v[1] + n[1] * KP[2] - n[2] * KP[1] + (av[1] * qv[2] - av[2] * qv[1]));
                cur[1] += sw[e] * (Kn[2] * v[0] - Kn[0] * v[2] + n[2] * KP[0] - n[0] * KP[2] + (av[2] * qv[0] - av[0] * qv[2]));
                cur[2] += sw[e] * (Kn[0] * v[1] - Kn[1] * v[0] + n[0] * KP[1] - n[1] * KP[0] + (av[0] * qv[1] - av[1] * qv[0]));
            }
        }
    }
    if (valid) {
        for (int q = 0; q < 3; ++q) E[(r * n_pts + pt) * 3 + q] = acc[q];
        if (WITH_H)
            for (int q = 0; q < 3; ++q) H[(r * n_pts + pt) * 3 + q] = cdiv(cur[q], dcon[4 * j + 3]);
    }
}

// one source node's term of the exterior representation formula at the point t (and its curl):
// w [n0 (a.Phi) - (n0.a) Phi - a (n0.Phi) + g Psi], n0 = -n, a = grad_s g (as k_near_field)
template <bool WITH_H>
__device__ void exterior_term(const double *t, const double *s, const double *n, double w, const c64 *Phi,
                              const c64 *Psi, c64 ik, c64 *acc, c64 *cur) {
    const double rv[3] = {s[0] - t[0], s[1] - t[1], s[2] - t[2]};
    const double R = sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
    const c64 g = cexpd(ik * R) * (1.0 / (4.0 * FMBEM_PI * R));
    const c64 g1 = g * (ik - c64{1.0 / R, 0});
    const c64 c = g1 * (1.0 / R);
    const double n0[3] = {-n[0], -n[1], -n[2]};
    const c64 rP = rv[0] * Phi[0] + rv[1] * Phi[1] + rv[2] * Phi[2];
    const c64 nP = n0[0] * Phi[0] + n0[1] * Phi[1] + n0[2] * Phi[2];
    const double nr = n0[0] * rv[0] + n0[1] * rv[1] + n0[2] * rv[2];
    for (int q = 0; q < 3; ++q) acc[q] += w * (c * (n0[q] * rP - nr * Phi[q] - rv[q] * nP) + g * Psi[q]);
    if (WITH_H) {
        const double iR = 1.0 / R, rh[3] = {rv[0] * iR, rv[1] * iR, rv[2] * iR};
        const c64 q1 = ik - c64{iR, 0};
        const c64 g2 = g * (q1 * q1 + c64{iR * iR, 0});
        const double rn = rh[0] * n0[0] + rh[1] * n0[1] + rh[2] * n0[2];
        const c64 rhP = rP * iR;
        c64 Kn[3], KP[3], av[3];
        for (int q = 0; q < 3; ++q) {
            Kn[q] = g2 * (rh[q] * rn) + c * (n0[q] - rh[q] * rn);
            KP[q] = g2 * rhP * rh[q] + c * (Phi[q] - rhP * rh[q]);
            av[q] = g1 * rh[q];
        }
        cur[0] += w * (Kn[1] * Phi[2] - Kn[2] * Phi[1] + n0[1] * KP[2] - n0[2] * KP[1] - (av[1] * Psi[2] - av[2] * Psi[1]));
        cur[1] += w * (Kn[2] * Phi[0] - Kn[0] * Phi[2] + n0[2] * KP[0] - n0[0] * KP[2] - (av[2] * Psi[0] - av[0] * Psi[2]));
        cur[2] += w * (Kn[0] * Phi[1] - Kn[1] * Phi[0] + n0[0] * KP[1] - n0[1] * KP[0] - (av[0] * Psi[1] - av[1] * Psi[0]));
    }
}

// Exterior fields through the fast multipole passes (see fmbem_near_field_fmm): a point in leaf g
// takes the far sources from g's local expansion of the background domain (the matvec's D, whose
// L2P gives minus the scattered field: the background rows carry the representation formula with
// the opposite sign), and the sources of g and its Neighbor leaves directly; a point outside
// every leaf sums all nodes directly.  Thread per (point, rhs).
constexpr int FF_PMAX = 20;
template <bool WITH_H>
__global__ void __launch_bounds__(128) k_field_fmm(int64_t N, int64_t nr, int p, int64_t nbox,
                                                 const int32_t *leaf_box, const int32_t *leaf_level,
                                                 const int32_t *leaf_of, const double *box_ctr,
                                                 const int32_t *nbeg, const int32_t *nend, const int32_t *nbr_start,
                                                 const int32_t *nbr_idx, const double *spos, const double *snrm,
                                                 const double *sw, const int32_t *perm, const double *upos,
                                                 const double *unrm, const double *uw, const c64 *x, const c64 *D,
                                                 double kw0, int64_t n_pts, const double *pts, c64 k0, c64 iwmu,
                                                 const double *dir, const c64 *pol, c64 *E, c64 *H) {
    const int64_t pt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, r = blockIdx.y;
    if (pt >= n_pts) return;
    const double t[3] = {pts[3 * pt], pts[3 * pt + 1], pts[3 * pt + 2]};
    const c64 ik = {-k0.im, k0.re};
    c64 acc[3] = {{0, 0}, {0, 0}, {0, 0}}, cur[3] = {{0, 0}, {0, 0}, {0, 0}};
    if (dir != nullptr && pol != nullptr) {
        const double *d = dir + 3 * r;
        const c64 *e = pol + 3 * r;
        const c64 ph = cexpd(ik * (d[0] * t[0] + d[1] * t[1] + d[2] * t[2]));
        for (int q = 0; q < 3; ++q) acc[q] = e[q] * ph;
        if (WITH_H) {
            const c64 de[3] = {d[1] * e[2] - d[2] * e[1], d[2] * e[0] - d[0] * e[2], d[0] * e[1] - d[1] * e[0]};
            for (int q = 0; q < 3; ++q) cur[q] = ik * de[q] * ph;
        }
    }
    const int32_t lf = leaf_of[pt];
    if (lf < 0) {
        for (int64_t b = 0; b < N; ++b)
            exterior_term<WITH_H>(t, upos + 3 * b, unrm + 3 * b, uw[b], x + (r * N + b) * 6, x + (r * N + b) * 6 + 3, ik,
                                  acc, cur);
    } else {
        const int64_t g = leaf_box[lf];
        const double lam = ldexp(kw0, -leaf_level[lf]);  // |k_0| w of the leaf's level
        for (int q = nbr_start[lf]; q < nbr_start[lf + 1]; ++q) {
            const int32_t bx = nbr_idx[q];
            for (int i = nbeg[bx]; i < nend[bx]; ++i) {
                const c64 *xb = x + (r * N + perm[i]) * 6;
                exterior_term<WITH_H>(t, spos + 3 * i, snrm + 3 * i, sw[i], xb, xb + 3, ik, acc, cur);
            }
        }
        // L2P: sum_q D_q R_q(t - c) / lambda^n (and its gradient), subtracted
        const double *c = box_ctr + 3 * g;
        const double rl[3] = {t[0] - c[0], t[1] - c[1], t[2] - c[2]};
        c64 R[(FF_PMAX + 1) * (FF_PMAX + 1)], rad[FF_PMAX + 2];
        double Pb[(FF_PMAX + 2) * (FF_PMAX + 3) / 2];
        wave_functions<false>(p, k0, rl, R, rad, Pb);
        const int p2 = p * p;
        const c64 *Dg = D + (g * 3 * nr + 3 * r) * p2;  // background domain (d = 0)
        c64 grad[3][3] = {{{0, 0}, {0, 0}, {0, 0}}, {{0, 0}, {0, 0}, {0, 0}}, {{0, 0}, {0, 0}, {0, 0}}};  // [component][axis]
        double lpow = 1.0;
        for (int n = 0; n < p; ++n) {
            const double sc = 1.0 / lpow;
            for (int m = -n; m <= n; ++m) {
                const int qi = n * n + n + m;
                c64 gr[3];
                if (WITH_H) grad_regular(p, k0, R, n, m, gr);
                for (int comp = 0; comp < 3; ++comp) {
                    const c64 dq = Dg[comp * p2 + qi] * sc;
                    acc[comp] -= dq * R[qi];
                    if (WITH_H)
                        for (int a = 0; a < 3; ++a) grad[comp][a] += dq * gr[a];
                }
            }
            lpow *= lam;
        }
        if (WITH_H) {  // curl of -sum: subtract the curl of the expansion's field
            cur[0] -= grad[2][1] - grad[1][2];
            cur[1] -= grad[0][2] - grad[2][0];
            cur[2] -= grad[1][0] - grad[0][1];
        }
    }
    for (int q = 0; q < 3; ++q) E[(r * n_pts + pt) * 3 + q] = acc[q];
    if (WITH_H)
        for (int q = 0; q < 3; ++q) H[(r * n_pts + pt) * 3 + q] = cdiv(cur[q], iwmu);
}

// Transposed near-field map (for adjoint gradients of quantities built from exterior fields):
// out[f][b] = sum_p ( cE[f][p] . dE(r_p)/dx_b + cH[f][p] . dH(r_p)/dx_b ), with E, H as in
// k_near_field (no incident part: it does not depend on x).  For c = cE[f][p]:
//   c . dE/dPhi_b = w_b [ (c.n0) a - (n0.a) c - (c.a) n0 ],      c . dE/dPsi_b = w_b g c;
// with c' = cH[f][p] / (i k0 mu_0) and K the Hessian of g in s_b (symmetric):
//   c' . dH/dPhi_b = w_b [ c' x (K n0) + K (c' x n0) ],          c' . dH/dPsi_b = -w_b c' x a.
// One thread per (node, functional); the points staged in shared memory OB_NS at a time.
template <bool WITH_H>
__global__ void __launch_bounds__(OB_NT) k_near_field_functional(int64_t N, const double *pos, const double *nrm,
                                                               const double *w, int64_t n_pts, const double *pts,
                                                               const c64 *cE, const c64 *cH, c64 k0, c64 iwmu,
                                                               c64 *out) {
    __shared__ double spt[OB_NS][3];
    __shared__ c64 sce[OB_NS][3], sch[OB_NS][3];
    const int64_t b = blockIdx.x * (int64_t)OB_NT + threadIdx.x, f = blockIdx.y;
    const bool valid = b < N;
    const double s[3] = {valid ? pos[3 * b] : 0.0, valid ? pos[3 * b + 1] : 0.0, valid ? pos[3 * b + 2] : 0.0};
    const double n0[3] = {valid ? -nrm[3 * b] : 0.0, valid ? -nrm[3 * b + 1] : 0.0, valid ? -nrm[3 * b + 2] : 0.0};
    const c64 ik = {-k0.im, k0.re};
    c64 oP[3] = {{0, 0}, {0, 0}, {0, 0}}, oQ[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int64_t p0 = 0; p0 < n_pts; p0 += OB_NS) {
        const int np = (int)min((int64_t)OB_NS, n_pts - p0);
        __syncthreads();
        for (int e = threadIdx.x; e < np; e += blockDim.x) {
            for (int q = 0; q < 3; ++q) {
                spt[e][q] = pts[3 * (p0 + e) + q];
                sce[e][q] = cE[(f * n_pts + p0 + e) * 3 + q];
                if (WITH_H) sch[e][q] = cdiv(cH[(f * n_pts + p0 + e) * 3 + q], iwmu);
            }
        }
        __syncthreads();
        if (!valid) continue;
        for (int e = 0; e < np; ++e) {
            const double rv[3] = {s[0] - spt[e][0], s[1] - spt[e][1], s[2] - spt[e][2]};
            const double R = sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]), iR = 1.0 / R;
            const c64 g = cexpd(ik * R) * (iR / (4.0 * FMBEM_PI));
            const c64 q1 = ik - c64{iR, 0};
            const c64 g1 = g * q1, c = g1 * iR;
            const double rh[3] = {rv[0] * iR, rv[1] * iR, rv[2] * iR};
            const c64 a[3] = {g1 * rh[0], g1 * rh[1], g1 * rh[2]};
            const c64 *ce = sce[e];
            const c64 cn = ce[0] * n0[0] + ce[1] * n0[1] + ce[2] * n0[2];
            const c64 na = a[0] * n0[0] + a[1] * n0[1] + a[2] * n0[2];
            const c64 ca = ce[0] * a[0] + ce[1] * a[1] + ce[2] * a[2];
            for (int q = 0; q < 3; ++q) {
                oP[q] += cn * a[q] - na * ce[q] - ca * n0[q];
                oQ[q] += g * ce[q];
            }
            if (WITH_H) {
                const c64 *ch = sch[e];
                const c64 g2 = g * (q1 * q1 + c64{iR * iR, 0});
                const double rn = rh[0] * n0[0] + rh[1] * n0[1] + rh[2] * n0[2];
                c64 Kn[3];
                for (int q = 0; q < 3; ++q) Kn[q] = g2 * (rh[q] * rn) + c * (n0[q] - rh[q] * rn);
                const c64 cxn[3] = {ch[1] * n0[2] - ch[2] * n0[1], ch[2] * n0[0] - ch[0] * n0[2], ch[0] * n0[1] - ch[1] * n0[0]};
                const c64 rc = rh[0] * cxn[0] + rh[1] * cxn[1] + rh[2] * cxn[2];
                const c64 cxK[3] = {ch[1] * Kn[2] - ch[2] * Kn[1], ch[2] * Kn[0] - ch[0] * Kn[2], ch[0] * Kn[1] - ch[1] * Kn[0]};
                const c64 cxa[3] = {ch[1] * a[2] - ch[2] * a[1], ch[2] * a[0] - ch[0] * a[2], ch[0] * a[1] - ch[1] * a[0]};
                for (int q = 0; q < 3; ++q) {
                    // K (c' x n0) = g'' rh (rh.(c' x n0)) + g'/R ((c' x n0) - rh (rh.(c' x n0)))
                    const c64 Kc = g2 * rc * rh[q] + c * (cxn[q] - rc * rh[q]);
                    oP[q] += cxK[q] + Kc;
                    oQ[q] += -cxa[q];
                }
            }
        }
    }
    if (valid) {
        c64 *o = out + (f * N + b) * 6;
        for (int q = 0; q < 3; ++q) {
            o[q] = oP[q] * w[b];
            o[3 + q] = oQ[q] * w[b];
        }
    }
}

// Cross sections and the far-zone force of every right-hand side from its far field F[r][dir][3]
// on directions (d_0 .. d_{nr-1}, q_0 .. q_{nq-1}): the forward direction d_r of its own plane wave
// and the quadrature directions q with weights wq (Gauss-Legendre in cos theta x trapezoid in
// phi).  out[r] = (C_ext, C_sca, Fx, Fy, Fz):
//   C_ext = (4 pi / k0) Im[conj(e_r) . F_r(d_r)] (optical theorem), C_sca = sum_q wq |F_r(q)|^2,
//   F = (C_ext d_r - sum_q wq |F_r(q)|^2 q) / 2 (momentum balance in the far zone, vacuum units).
__global__ void __launch_bounds__(OB_TB) k_far_reduce(int64_t nr, int64_t nq, const c64 *F, const double *dirs,
                                                    const c64 *pol, const double *wq, double k0, double *out) {
    __shared__ double red[4][OB_TB];
    const int64_t r = blockIdx.x, ndir = nr + nq;
    double a[4] = {0, 0, 0, 0};
    for (int64_t q = threadIdx.x; q < nq; q += blockDim.x) {
        const c64 *f = F + ((r * ndir) + nr + q) * 3;
        const double f2 = abs2(f[0]) + abs2(f[1]) + abs2(f[2]);
        const double *u = dirs + 3 * (nr + q);
        a[0] += wq[q] * f2;
        for (int c = 0; c < 3; ++c) a[1 + c] += wq[q] * f2 * u[c];
    }
    for (int c = 0; c < 4; ++c) red[c][threadIdx.x] = a[c];
    __syncthreads();
    for (int off = OB_TB / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off)
            for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const c64 *fd = F + (r * ndir + r) * 3;
        double im = 0;
        for (int c = 0; c < 3; ++c) im += (conjg(pol[3 * r + c]) * fd[c]).im;
        const double cext = 4 * FMBEM_PI / k0 * im;
        double *o = out + 5 * r;
        o[0] = cext;
        o[1] = red[0][0];
        for (int c = 0; c < 3; ++c) o[2 + c] = 0.5 * (cext * dirs[3 * r + c] - red[1 + c][0]);
    }
}

// Time-averaged Maxwell-stress force on the surface points p_q = c + R n_q with weights wq
// (R^2 included): F = sum_q wq T n_q, T n = Re[E (E*.n) + H (H*.n) - (|E|^2 + |H|^2) n / 2] / 2
// (vacuum units), E and H the total fields E[r][q][3], H[r][q][3].  out[r][3].
__global__ void __launch_bounds__(OB_TB) k_stress_reduce(int64_t nq, const c64 *E, const c64 *H, const double *nq_dir,
                                                       const double *wq, double *out) {
    __shared__ double red[3][OB_TB];
    const int64_t r = blockIdx.x;
    double a[3] = {0, 0, 0};
    for (int64_t q = threadIdx.x; q < nq; q += blockDim.x) {
        const c64 *e = E + (r * nq + q) * 3, *hh = H + (r * nq + q) * 3;
        const double *n = nq_dir + 3 * q;
        c64 en = {0, 0}, hn = {0, 0};
        for (int c = 0; c < 3; ++c) {
            en += n[c] * conjg(e[c]);
            hn += n[c] * conjg(hh[c]);
        }
        const double u = abs2(e[0]) + abs2(e[1]) + abs2(e[2]) + abs2(hh[0]) + abs2(hh[1]) + abs2(hh[2]);
        for (int c = 0; c < 3; ++c) a[c] += wq[q] * 0.5 * ((e[c] * en).re + (hh[c] * hn).re - 0.5 * u * n[c]);
    }
    for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = a[c];
    __syncthreads();
    for (int off = OB_TB / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off)
            for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) out[3 * r + c] = red[c][0];
}

// Wirtinger coefficients of the stress force's components with respect to the fields at the
// sphere points (see fmbem_force_stress_functional): for component i, point q and field index j,
//   c[i][q][j] = w_q / 4 [delta_ij (conj(F_q) . n_q) + conj(F_q,i) n_q,j - n_q,i conj(F_q,j)],
// F = E (cE) or H (cH); one thread per (i, q, j).
__global__ void k_stress_wirtinger(int64_t nq, const c64 *E, const c64 *H, const double *nq_dir, const double *wq,
                                   c64 *cE, c64 *cH) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= 9 * nq) return;
    const int i = (int)(idx / (3 * nq)), j = (int)(idx % 3);
    const int64_t q = (idx / 3) % nq;
    const double *n = nq_dir + 3 * q;
    for (int f = 0; f < 2; ++f) {
        const c64 *F = (f == 0 ? E : H) + 3 * q;
        c64 fn = {0, 0};
        for (int c = 0; c < 3; ++c) fn += n[c] * conjg(F[c]);
        c64 v = n[j] * conjg(F[i]) - n[i] * conjg(F[j]);
        if (i == j) v += fn;
        (f == 0 ? cE : cH)[idx] = (0.25 * wq[q]) * v;
    }
}

// y = (a - b) * s elementwise over n complex values (central difference of two products)
__global__ void k_cdiff(int64_t n, const c64 *a, const c64 *b, double s, c64 *y) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = s * (a[i] - b[i]);
}

// out[r] = sum_k lam[r][k] y[r][k] (bilinear), one block per right-hand side
__global__ void __launch_bounds__(OB_TB) k_bilinear(int64_t n, const c64 *lam, const c64 *y, c64 *out) {
    __shared__ double red[2][OB_TB];
    const int64_t r = blockIdx.x;
    c64 acc = {0, 0};
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) cfma(acc, lam[r * n + k], y[r * n + k]);
    red[0][threadIdx.x] = acc.re;
    red[1][threadIdx.x] = acc.im;
    __syncthreads();
    for (int off = OB_TB / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            red[0][threadIdx.x] += red[0][threadIdx.x + off];
            red[1][threadIdx.x] += red[1][threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[r] = c64{red[0][0], red[1][0]};
}

}  // namespace

void run_near_field_functional(fmbem *h, int64_t nf, int64_t n_pts, const double *pts_host, const c64 *cE_host,
                               const c64 *cH_host, c64 *out, cudaStream_t s) {
    double *dp = (double *)dev_alloc(h, sizeof(double) * 3 * n_pts);
    c64 *dE = (c64 *)dev_alloc(h, sizeof(c64) * 3 * n_pts * nf);
    c64 *dH = cH_host ? (c64 *)dev_alloc(h, sizeof(c64) * 3 * n_pts * nf) : nullptr;
    auto cleanup = [&] {
        dev_free(h, dp);
        dev_free(h, dE);
        if (dH) dev_free(h, dH);
    };
    try {
        CK(cudaMemcpyAsync(dp, pts_host, sizeof(double) * 3 * n_pts, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dE, cE_host, sizeof(c64) * 3 * n_pts * nf, cudaMemcpyHostToDevice, s));
        if (dH) CK(cudaMemcpyAsync(dH, cH_host, sizeof(c64) * 3 * n_pts * nf, cudaMemcpyHostToDevice, s));
        const dim3 grid((unsigned)((h->N + OB_NT - 1) / OB_NT), (unsigned)nf);
        const c64 iwmu = c64{0, h->k0} * h->mu[0];
        if (dH)
            k_near_field_functional<true><<<grid, OB_NT, 0, s>>>(h->N, h->upos, h->unrm, h->uw, n_pts, dp, dE, dH, h->k[0],
                                                                 iwmu, out);
        else
            k_near_field_functional<false><<<grid, OB_NT, 0, s>>>(h->N, h->upos, h->unrm, h->uw, n_pts, dp, dE, nullptr,
                                                                  h->k[0], iwmu, out);
        CKL("k_near_field_functional");
        CK(cudaStreamSynchronize(s));
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
}

void run_near_field(fmbem *h, const c64 *x, int64_t nr, int64_t n_pts, const double *pts_host, const double *dir_host,
                    const c64 *pol_host, c64 *E_host, c64 *H_host, cudaStream_t s) {
    double *dp = (double *)dev_alloc(h, sizeof(double) * 3 * n_pts);
    c64 *dE = (c64 *)dev_alloc(h, sizeof(c64) * 3 * n_pts * nr);
    c64 *dH = H_host ? (c64 *)dev_alloc(h, sizeof(c64) * 3 * n_pts * nr) : nullptr;
    double *dd = nullptr;
    c64 *dpol = nullptr;
    auto cleanup = [&] {
        dev_free(h, dp);
        dev_free(h, dE);
        if (dH) dev_free(h, dH);
        if (dd) dev_free(h, dd);
        if (dpol) dev_free(h, dpol);
    };
    try {
        CK(cudaMemcpyAsync(dp, pts_host, sizeof(double) * 3 * n_pts, cudaMemcpyHostToDevice, s));
        if (dir_host && pol_host) {
            dd = (double *)dev_alloc(h, sizeof(double) * 3 * nr);
            dpol = (c64 *)dev_alloc(h, sizeof(c64) * 3 * nr);
            CK(cudaMemcpyAsync(dd, dir_host, sizeof(double) * 3 * nr, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(dpol, pol_host, sizeof(c64) * 3 * nr, cudaMemcpyHostToDevice, s));
        }
        const dim3 grid((unsigned)((n_pts + OB_NT - 1) / OB_NT), (unsigned)nr);
        const c64 iwmu = c64{0, h->k0} * h->mu[0];  // i omega mu_0 with omega = k0 (c = 1)
        if (dH)
            k_near_field<true><<<grid, OB_NT, 0, s>>>(h->N, h->upos, h->unrm, h->uw, x, n_pts, dp, h->k[0], iwmu, dd, dpol,
                                                      dE, dH);
        else
            k_near_field<false><<<grid, OB_NT, 0, s>>>(h->N, h->upos, h->unrm, h->uw, x, n_pts, dp, h->k[0], iwmu, dd,
                                                       dpol, dE, nullptr);
        CKL("k_near_field");
        CK(cudaMemcpyAsync(E_host, dE, sizeof(c64) * 3 * n_pts * nr, cudaMemcpyDeviceToHost, s));
        if (dH) CK(cudaMemcpyAsync(H_host, dH, sizeof(c64) * 3 * n_pts * nr, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
}

void run_interior_field(fmbem *h, const c64 *x, int64_t nr, int64_t n_pts, const double *pts_host,
                        const int32_t *dom_host, c64 *E_host, c64 *H_host, cudaStream_t s) {
    if (h->ibc) throw fmbem_error{FMBEM_ERR_INVALID_ARGUMENT, "the impedance boundary does not model the interiors"};
    for (int64_t p = 0; p < n_pts; ++p)
        if (dom_host[p] < 1 || dom_host[p] > h->J)
            throw fmbem_error{FMBEM_ERR_INVALID_ARGUMENT, "point " + std::to_string(p) + ": domain outside 1..n_scatterers"};
    std::vector<c64> dc(4 * (h->J + 1));
    for (int d = 0; d <= h->J; ++d) {
        dc[4 * d] = h->k[d];
        dc[4 * d + 1] = d == 0 ? c64{0, 0} : cdiv(h->eps[0] - h->eps[d], h->eps[d]);  // T_d = I + t_d n n^T
        dc[4 * d + 2] = h->gam[d];
        dc[4 * d + 3] = c64{0, h->k0} * h->mu[d];  // i omega mu_d with omega = k0 (c = 1)
    }
    double *dp = (double *)dev_alloc(h, sizeof(double) * 3 * n_pts);
    int32_t *dd = (int32_t *)dev_alloc(h, sizeof(int32_t) * n_pts);
    c64 *dcon = (c64 *)dev_alloc(h, sizeof(c64) * dc.size());
    c64 *dE = (c64 *)dev_alloc(h, sizeof(c64) * 3 * n_pts * nr);
    c64 *dH = H_host ? (c64 *)dev_alloc(h, sizeof(c64) * 3 * n_pts * nr) : nullptr;
    auto cleanup = [&] {
        dev_free(h, dp);
        dev_free(h, dd);
        dev_free(h, dcon);
        dev_free(h, dE);
        if (dH) dev_free(h, dH);
    };
    try {
        CK(cudaMemcpyAsync(dp, pts_host, sizeof(double) * 3 * n_pts, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dd, dom_host, sizeof(int32_t) * n_pts, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dcon, dc.data(), sizeof(c64) * dc.size(), cudaMemcpyHostToDevice, s));
        const dim3 grid((unsigned)((n_pts + OB_NT - 1) / OB_NT), (unsigned)nr);
        if (dH)
            k_interior_field<true><<<grid, OB_NT, 0, s>>>(h->N, h->upos, h->unrm, h->uw, h->udom, x, n_pts, dp, dd, dcon,
                                                          dE, dH);
        else
            k_interior_field<false><<<grid, OB_NT, 0, s>>>(h->N, h->upos, h->unrm, h->uw, h->udom, x, n_pts, dp, dd,
                                                           dcon, dE, nullptr);
        CKL("k_interior_field");
        CK(cudaMemcpyAsync(E_host, dE, sizeof(c64) * 3 * n_pts * nr, cudaMemcpyDeviceToHost, s));
        if (dH) CK(cudaMemcpyAsync(H_host, dH, sizeof(c64) * 3 * n_pts * nr, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
}

void run_near_field_fmm(fmbem *h, const c64 *x, int64_t nr, int64_t n_pts, const double *pts_host,
                        const double *dir_host, const c64 *pol_host, c64 *E_host, c64 *H_host, cudaStream_t s) {
    if (h->p > FF_PMAX) throw fmbem_error{FMBEM_ERR_INVALID_ARGUMENT, "p above the supported maximum"};
    c64 *yscr = (c64 *)dev_alloc(h, sizeof(c64) * 6 * h->N * nr);
    double *dp = (double *)dev_alloc(h, sizeof(double) * 3 * n_pts);
    int32_t *dl = (int32_t *)dev_alloc(h, sizeof(int32_t) * n_pts);
    c64 *dE = (c64 *)dev_alloc(h, sizeof(c64) * 3 * n_pts * nr);
    c64 *dH = H_host ? (c64 *)dev_alloc(h, sizeof(c64) * 3 * n_pts * nr) : nullptr;
    double *dd = nullptr;
    c64 *dpol = nullptr;
    auto cleanup = [&] {
        for (void *q : {(void *)yscr, (void *)dp, (void *)dl, (void *)dE, (void *)dH, (void *)dd, (void *)dpol})
            if (q) dev_free(h, q);
    };
    try {
        // the passes of one FP64 product leave the local expansions of x's background sums in D
        run_matvec(h, x, yscr, nr, FMBEM_FP64, s);
        CK(cudaMemcpyAsync(dp, pts_host, sizeof(double) * 3 * n_pts, cudaMemcpyHostToDevice, s));
        if (dir_host && pol_host) {
            dd = (double *)dev_alloc(h, sizeof(double) * 3 * nr);
            dpol = (c64 *)dev_alloc(h, sizeof(c64) * 3 * nr);
            CK(cudaMemcpyAsync(dd, dir_host, sizeof(double) * 3 * nr, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(dpol, pol_host, sizeof(c64) * 3 * nr, cudaMemcpyHostToDevice, s));
        }
        run_locate_leaves(h, dp, n_pts, dl, s);
        const double kw0 = cabsd(h->k[0]) * h->lev[0].w;  // the scale of level l is kw0 / 2^l
        const c64 iwmu = c64{0, h->k0} * h->mu[0];
        const dim3 grid((unsigned)((n_pts + 127) / 128), (unsigned)nr);
        if (dH)
            k_field_fmm<true><<<grid, 128, 0, s>>>(h->N, nr, h->p, h->nbox, h->leaf_box, h->leaf_level, dl, h->box_ctr, h->box_nbeg,
                                                   h->box_nend, h->nbr_start, h->nbr_idx, h->pos, h->nrm, h->w,
                                                   h->perm, h->upos, h->unrm, h->uw, x, (const c64 *)h->Dexp, kw0,
                                                   n_pts, dp, h->k[0], iwmu, dd, dpol, dE, dH);
        else
            k_field_fmm<false><<<grid, 128, 0, s>>>(h->N, nr, h->p, h->nbox, h->leaf_box, h->leaf_level, dl, h->box_ctr, h->box_nbeg,
                                                    h->box_nend, h->nbr_start, h->nbr_idx, h->pos, h->nrm, h->w,
                                                    h->perm, h->upos, h->unrm, h->uw, x, (const c64 *)h->Dexp, kw0,
                                                    n_pts, dp, h->k[0], iwmu, dd, dpol, dE, nullptr);
        CKL("k_field_fmm");
        CK(cudaMemcpyAsync(E_host, dE, sizeof(c64) * 3 * n_pts * nr, cudaMemcpyDeviceToHost, s));
        if (dH) CK(cudaMemcpyAsync(H_host, dH, sizeof(c64) * 3 * n_pts * nr, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
}

void run_far_field(fmbem *h, const c64 *x, int64_t nr, int64_t n_dir, const double *rhat_host, c64 *F_host,
                   cudaStream_t s) {
    double *dr = (double *)dev_alloc(h, sizeof(double) * 3 * n_dir);
    c64 *dF = (c64 *)dev_alloc(h, sizeof(c64) * 3 * n_dir * nr);
    try {
        CK(cudaMemcpyAsync(dr, rhat_host, sizeof(double) * 3 * n_dir, cudaMemcpyHostToDevice, s));
        k_far_field<<<dim3((unsigned)n_dir, (unsigned)nr), OB_TB, 0, s>>>(h->N, h->upos, h->unrm, h->uw, x, dr, h->k[0],
                                                                         n_dir, dF);
        CKL("k_far_field");
        CK(cudaMemcpyAsync(F_host, dF, sizeof(c64) * 3 * n_dir * nr, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    } catch (...) {
        dev_free(h, dr);
        dev_free(h, dF);
        throw;
    }
    dev_free(h, dr);
    dev_free(h, dF);
}

void run_far_field_functional(fmbem *h, int64_t nr, const double *rhat_host, const c64 *coef_host, c64 *out,
                              cudaStream_t s) {
    double *dr = (double *)dev_alloc(h, sizeof(double) * 3 * nr);
    c64 *dc = (c64 *)dev_alloc(h, sizeof(c64) * 3 * nr);
    try {
        CK(cudaMemcpyAsync(dr, rhat_host, sizeof(double) * 3 * nr, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dc, coef_host, sizeof(c64) * 3 * nr, cudaMemcpyHostToDevice, s));
        k_far_field_functional<<<dim3((unsigned)((h->N + 127) / 128), (unsigned)nr), 128, 0, s>>>(
            h->N, nr, h->upos, h->unrm, h->uw, dr, dc, h->k[0], out);
        CKL("k_far_field_functional");
        CK(cudaStreamSynchronize(s));
    } catch (...) {
        dev_free(h, dr);
        dev_free(h, dc);
        throw;
    }
    dev_free(h, dr);
    dev_free(h, dc);
}

void run_absorption(fmbem *h, const c64 *x, int64_t nr, double *out_host, cudaStream_t s) {
    double *d = (double *)dev_alloc(h, sizeof(double) * nr);
    try {
        k_absorption<<<(unsigned)nr, OB_TB, 0, s>>>(h->N, h->uw, x, d);
        CKL("k_absorption");
        CK(cudaMemcpyAsync(out_host, d, sizeof(double) * nr, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    } catch (...) {
        dev_free(h, d);
        throw;
    }
    dev_free(h, d);
}

// unit directions and weights of the Gauss-Legendre (cos theta) x trapezoid (phi) rule on the sphere
static void sphere_rule(int nt, int np, std::vector<double> &dirs, std::vector<double> &w) {
    std::vector<double> x, gw;
    gauss_legendre(nt, x, gw);
    dirs.resize(3 * (size_t)nt * np);
    w.resize((size_t)nt * np);
    for (int i = 0; i < nt; ++i)
        for (int j = 0; j < np; ++j) {
            const double ct = x[i], st = std::sqrt(std::max(0.0, 1 - ct * ct)), ph = 2 * FMBEM_PI * j / np;
            const size_t q = (size_t)i * np + j;
            dirs[3 * q] = st * std::cos(ph);
            dirs[3 * q + 1] = st * std::sin(ph);
            dirs[3 * q + 2] = ct;
            w[q] = gw[i] * 2 * FMBEM_PI / np;
        }
}

// C_ext, C_sca, C_abs and the far-zone force of the plane waves (dir, pol) that produced x
// (see fmbem_cross_sections); out_host [nr][6] = (C_ext, C_sca, C_abs, Fx, Fy, Fz)
void run_cross_sections(fmbem *h, const c64 *x, int64_t nr, const double *dir_host, const c64 *pol_host, int nt, int np,
                        double *out_host, cudaStream_t s) {
    if (h->k[0].im != 0.0 || !(h->k[0].re > 0))
        throw fmbem_error{FMBEM_ERR_INVALID_ARGUMENT, "cross sections need a lossless background"};
    std::vector<double> q, wq;
    sphere_rule(nt, np, q, wq);
    const int64_t nq = (int64_t)wq.size(), ndir = nr + nq;
    std::vector<double> dirs(3 * ndir);
    std::copy(dir_host, dir_host + 3 * nr, dirs.begin());
    std::copy(q.begin(), q.end(), dirs.begin() + 3 * nr);
    double *dd = (double *)dev_alloc(h, sizeof(double) * 3 * ndir);
    double *dw = (double *)dev_alloc(h, sizeof(double) * nq);
    c64 *dp = (c64 *)dev_alloc(h, sizeof(c64) * 3 * nr);
    c64 *dF = (c64 *)dev_alloc(h, sizeof(c64) * 3 * ndir * nr);
    double *dout = (double *)dev_alloc(h, sizeof(double) * 5 * nr);
    double *dabs = (double *)dev_alloc(h, sizeof(double) * nr);
    auto cleanup = [&] {
        for (void *p : {(void *)dd, (void *)dw, (void *)dp, (void *)dF, (void *)dout, (void *)dabs}) dev_free(h, p);
    };
    try {
        CK(cudaMemcpyAsync(dd, dirs.data(), sizeof(double) * 3 * ndir, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dw, wq.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dp, pol_host, sizeof(c64) * 3 * nr, cudaMemcpyHostToDevice, s));
        k_far_field<<<dim3((unsigned)ndir, (unsigned)nr), OB_TB, 0, s>>>(h->N, h->upos, h->unrm, h->uw, x, dd, h->k[0],
                                                                        ndir, dF);
        CKL("k_far_field");
        k_far_reduce<<<(unsigned)nr, OB_TB, 0, s>>>(nr, nq, dF, dd, dp, dw, h->k[0].re, dout);
        CKL("k_far_reduce");
        k_absorption<<<(unsigned)nr, OB_TB, 0, s>>>(h->N, h->uw, x, dabs);
        CKL("k_absorption");
        std::vector<double> o(5 * nr), a(nr);
        CK(cudaMemcpyAsync(o.data(), dout, sizeof(double) * 5 * nr, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(a.data(), dabs, sizeof(double) * nr, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int64_t r = 0; r < nr; ++r) {
            double *row = out_host + 6 * r;
            row[0] = o[5 * r];
            row[1] = o[5 * r + 1];
            row[2] = -a[r] / h->k[0].re;  // Eq. (4.2): C_abs = -(1/k0) sum w Im(Phi . conj(Psi))
            for (int c = 0; c < 3; ++c) row[3 + c] = o[5 * r + 2 + c];
        }
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
}

// Maxwell-stress force on the scatterers inside the sphere (center, radius) in the plane waves
// (dir, pol): total E and H on the sphere's quadrature points by direct summation, then the
// stress-tensor reduction (see fmbem_force_stress); out_host [nr][3]
void run_force_stress(fmbem *h, const c64 *x, int64_t nr, const double *dir_host, const c64 *pol_host,
                      const double *center, double radius, int nt, int np, double *out_host, cudaStream_t s) {
    std::vector<double> q, wq;
    sphere_rule(nt, np, q, wq);
    const int64_t nq = (int64_t)wq.size();
    std::vector<double> pts(3 * nq);
    for (int64_t i = 0; i < nq; ++i) {
        for (int c = 0; c < 3; ++c) pts[3 * i + c] = center[c] + radius * q[3 * i + c];
        wq[i] *= radius * radius;
    }
    double *dpts = (double *)dev_alloc(h, sizeof(double) * 3 * nq);
    double *dq = (double *)dev_alloc(h, sizeof(double) * 3 * nq);
    double *dw = (double *)dev_alloc(h, sizeof(double) * nq);
    double *ddir = (double *)dev_alloc(h, sizeof(double) * 3 * nr);
    c64 *dpol = (c64 *)dev_alloc(h, sizeof(c64) * 3 * nr);
    c64 *dE = (c64 *)dev_alloc(h, sizeof(c64) * 3 * nq * nr);
    c64 *dH = (c64 *)dev_alloc(h, sizeof(c64) * 3 * nq * nr);
    double *dout = (double *)dev_alloc(h, sizeof(double) * 3 * nr);
    auto cleanup = [&] {
        for (void *p : {(void *)dpts, (void *)dq, (void *)dw, (void *)ddir, (void *)dpol, (void *)dE, (void *)dH,
                        (void *)dout})
            dev_free(h, p);
    };
    try {
        CK(cudaMemcpyAsync(dpts, pts.data(), sizeof(double) * 3 * nq, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dq, q.data(), sizeof(double) * 3 * nq, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dw, wq.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ddir, dir_host, sizeof(double) * 3 * nr, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dpol, pol_host, sizeof(c64) * 3 * nr, cudaMemcpyHostToDevice, s));
        const dim3 grid((unsigned)((nq + OB_NT - 1) / OB_NT), (unsigned)nr);
        const c64 iwmu = c64{0, h->k0} * h->mu[0];
        k_near_field<true><<<grid, OB_NT, 0, s>>>(h->N, h->upos, h->unrm, h->uw, x, nq, dpts, h->k[0], iwmu, ddir, dpol,
                                                  dE, dH);
        CKL("k_near_field");
        k_stress_reduce<<<(unsigned)nr, OB_TB, 0, s>>>(nq, dE, dH, dq, dw, dout);
        CKL("k_stress_reduce");
        CK(cudaMemcpyAsync(out_host, dout, sizeof(double) * 3 * nr, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
}

// the stress force of one plane wave and, on the device, the near-field functionals of its three
// components' Wirtinger coefficients (see fmbem_force_stress_functional)
void run_force_stress_functional(fmbem *h, const c64 *x, const double *dir_host, const c64 *pol_host,
                                 const double *center, double radius, int nt, int np, double *force_host,
                                 double *pts_host, c64 *cE_host, c64 *cH_host, c64 *L, cudaStream_t s) {
    std::vector<double> q, wq;
    sphere_rule(nt, np, q, wq);
    const int64_t nq = (int64_t)wq.size();
    std::vector<double> pts(3 * nq);
    for (int64_t i = 0; i < nq; ++i) {
        for (int c = 0; c < 3; ++c) pts[3 * i + c] = center[c] + radius * q[3 * i + c];
        wq[i] *= radius * radius;
    }
    double *dpts = (double *)dev_alloc(h, sizeof(double) * 3 * nq);
    double *dq = (double *)dev_alloc(h, sizeof(double) * 3 * nq);
    double *dw = (double *)dev_alloc(h, sizeof(double) * nq);
    double *ddir = (double *)dev_alloc(h, sizeof(double) * 3);
    c64 *dpol = (c64 *)dev_alloc(h, sizeof(c64) * 3);
    c64 *dE = (c64 *)dev_alloc(h, sizeof(c64) * 3 * nq);
    c64 *dH = (c64 *)dev_alloc(h, sizeof(c64) * 3 * nq);
    c64 *dcE = (c64 *)dev_alloc(h, sizeof(c64) * 9 * nq);
    c64 *dcH = (c64 *)dev_alloc(h, sizeof(c64) * 9 * nq);
    double *dout = (double *)dev_alloc(h, sizeof(double) * 3);
    auto cleanup = [&] {
        for (void *p : {(void *)dpts, (void *)dq, (void *)dw, (void *)ddir, (void *)dpol, (void *)dE, (void *)dH,
                        (void *)dcE, (void *)dcH, (void *)dout})
            dev_free(h, p);
    };
    try {
        CK(cudaMemcpyAsync(dpts, pts.data(), sizeof(double) * 3 * nq, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dq, q.data(), sizeof(double) * 3 * nq, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dw, wq.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ddir, dir_host, sizeof(double) * 3, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dpol, pol_host, sizeof(c64) * 3, cudaMemcpyHostToDevice, s));
        const c64 iwmu = c64{0, h->k0} * h->mu[0];
        k_near_field<true><<<dim3((unsigned)((nq + OB_NT - 1) / OB_NT), 1), OB_NT, 0, s>>>(
            h->N, h->upos, h->unrm, h->uw, x, nq, dpts, h->k[0], iwmu, ddir, dpol, dE, dH);
        CKL("k_near_field");
        k_stress_reduce<<<1, OB_TB, 0, s>>>(nq, dE, dH, dq, dw, dout);
        CKL("k_stress_reduce");
        k_stress_wirtinger<<<(unsigned)((9 * nq + 255) / 256), 256, 0, s>>>(nq, dE, dH, dq, dw, dcE, dcH);
        CKL("k_stress_wirtinger");
        // the scattered-field functional of the three components (the incident wave does not
        // depend on the solution)
        k_near_field_functional<true><<<dim3((unsigned)((h->N + OB_NT - 1) / OB_NT), 3), OB_NT, 0, s>>>(
            h->N, h->upos, h->unrm, h->uw, nq, dpts, dcE, dcH, h->k[0], iwmu, L);
        CKL("k_near_field_functional");
        CK(cudaMemcpyAsync(force_host, dout, sizeof(double) * 3, cudaMemcpyDeviceToHost, s));
        if (cE_host) CK(cudaMemcpyAsync(cE_host, dcE, sizeof(c64) * 9 * nq, cudaMemcpyDeviceToHost, s));
        if (cH_host) CK(cudaMemcpyAsync(cH_host, dcH, sizeof(c64) * 9 * nq, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (pts_host) std::copy(pts.begin(), pts.end(), pts_host);
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
}

// s[r] = lam_r^T (dA/deps_j) x_r with dA/deps_j the central difference of the operators with
// eps_j +- step (handles built once per (j, step) and kept, same mesh and options)
void run_eps_sensitivity(fmbem *h, int j, const c64 *x, const c64 *lam, int64_t nr, double step, c64 *out_host,
                         cudaStream_t s) {
    if (h->mesh_V.empty()) throw fmbem_error{FMBEM_ERR_INVALID_ARGUMENT, "the handle keeps no mesh copy"};
    if (h->eps_j != j || h->eps_step != step || !h->eps_plus || !h->eps_minus) {
        if (h->eps_plus) fmbem_destroy(h->eps_plus);
        if (h->eps_minus) fmbem_destroy(h->eps_minus);
        h->eps_plus = h->eps_minus = nullptr;
        const fmbem_mesh m{(int64_t)h->mesh_V.size() / 3, h->mesh_V.data(), (int64_t)h->mesh_F.size() / 3,
                           h->mesh_F.data(), h->mesh_D.data(), (int32_t)h->J};
        std::vector<fmbem_c64> ep(h->J + 1), em(h->J + 1), mu(h->J + 1);
        for (int d = 0; d <= h->J; ++d) {
            ep[d] = em[d] = fmbem_c64{h->eps_user[d].re, h->eps_user[d].im};
            mu[d] = fmbem_c64{h->mu_user[d].re, h->mu_user[d].im};
        }
        ep[j].re += step;
        em[j].re -= step;
        fmbem_options o = h->opt;
        o.near_cache = 0;
        o.profile_phases = 0;
        fmbem_status st = fmbem_create(&m, ep.data(), mu.data(), h->k0, &o, s, &h->eps_plus);
        if (st == FMBEM_OK) st = fmbem_create(&m, em.data(), mu.data(), h->k0, &o, s, &h->eps_minus);
        if (st != FMBEM_OK) throw fmbem_error{st, std::string("perturbed operator: ") + fmbem_last_error(nullptr)};
        h->eps_j = j;
        h->eps_step = step;
    }
    const int64_t n = 6 * h->N;
    c64 *yp = (c64 *)dev_alloc(h, sizeof(c64) * n * nr);
    c64 *ym = (c64 *)dev_alloc(h, sizeof(c64) * n * nr);
    c64 *dout = (c64 *)dev_alloc(h, sizeof(c64) * nr);
    auto cleanup = [&] {
        dev_free(h, yp);
        dev_free(h, ym);
        dev_free(h, dout);
    };
    try {
        run_matvec(h->eps_plus, x, yp, nr, FMBEM_FP64, s);
        run_matvec(h->eps_minus, x, ym, nr, FMBEM_FP64, s);
        k_cdiff<<<(unsigned)((n * nr + 255) / 256), 256, 0, s>>>(n * nr, yp, ym, 0.5 / step, yp);
        CKL("k_cdiff");
        k_bilinear<<<(unsigned)nr, OB_TB, 0, s>>>(n, lam, yp, dout);
        CKL("k_bilinear");
        CK(cudaMemcpyAsync(out_host, dout, sizeof(c64) * nr, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
}
