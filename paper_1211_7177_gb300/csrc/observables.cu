// observables.cu -- quantities of a solution: the far-field amplitude of the scattered field and
// the absorbed power (Section 4; representation formula of Appendix A in the far zone).
//
// Far field: with n0 = -n (the outward normal of the background) and Psi0 = -Psi,
//   F(u) = 1/(4 pi) sum_b w_b exp(-i k0 u.s_b) { (-i k0) [n0 (u.Phi_b) - (n0.u) Phi_b - u (n0.Phi_b)]
//                                                 - Psi0_b },
// so that the scattered field behaves as E_sca ~ exp(i k0 r)/r F(u) in direction u.
// Absorption: the inward flux of the time-averaged Poynting vector through the surface, Eq. (4.2),
// with n x curl E = Psi, reduces to C_abs = -(1/k0) sum_b w_b Im(Phi_b . conj(Psi_b)).
#include "fmbem_internal.cuh"

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

}  // namespace

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
