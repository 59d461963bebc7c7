// solver.cu -- right-preconditioned restarted GMRES for A x = b (Eqs. 2.9, 3.1) with the
// block-diagonal preconditioner M = A_self (Eq. 3.2).  Each right-hand side has its own Krylov
// space; all of them share one batched matvec per iteration.  Device kernels do every vector
// operation in double precision (classical Gram-Schmidt applied twice for the Arnoldi step);
// the host runs the small Hessenberg/Givens recurrences and the convergence tests.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "fmbem_internal.cuh"

namespace {

using cd = std::complex<double>;
constexpr int DOT_TB = 256;

inline unsigned nblk(int64_t n, int tb) { return (unsigned)((n + tb - 1) / tb); }

// partial[r][i][blk] = sum over the block's chunk of conj(V_i[r]) w[r]   (i = 0..nv-1)
// V_i[r] at V + (i * nr + r) * n
__global__ void k_multidot(const c64 *V, int nv, const c64 *w, int64_t n, int64_t nr, int nblocks, c64 *partial) {
    __shared__ double sre[DOT_TB], sim[DOT_TB];
    int i = blockIdx.y;
    int64_t r = blockIdx.z;
    const c64 *a = V + ((int64_t)i * nr + r) * n, *b = w + r * n;
    double re = 0, im = 0;
    for (int64_t q = blockIdx.x * (int64_t)DOT_TB + threadIdx.x; q < n; q += (int64_t)nblocks * DOT_TB) {
        c64 x = a[q], y = b[q];
        re += x.re * y.re + x.im * y.im;
        im += x.re * y.im - x.im * y.re;
    }
    sre[threadIdx.x] = re;
    sim[threadIdx.x] = im;
    __syncthreads();
    for (int off = DOT_TB / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) { sre[threadIdx.x] += sre[threadIdx.x + off]; sim[threadIdx.x] += sim[threadIdx.x + off]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[((int64_t)r * nv + i) * nblocks + blockIdx.x] = c64{sre[0], sim[0]};
}
__global__ void k_reduce_partials(const c64 *partial, int nblocks, int64_t count, c64 *out) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= count) return;
    c64 s = {0, 0};
    for (int b = 0; b < nblocks; ++b) s += partial[e * nblocks + b];
    out[e] = s;
}
// w[r] -= sum_i h[r][i] V_i[r]
__global__ void k_subtract(const c64 *V, int nv, const c64 *hcoef, c64 *w, int64_t n, int64_t nr) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t r = blockIdx.y;
    if (q >= n) return;
    c64 acc = w[r * n + q];
    for (int i = 0; i < nv; ++i) acc -= hcoef[r * nv + i] * V[((int64_t)i * nr + r) * n + q];
    w[r * n + q] = acc;
}
// out[r] = sum_i y[r][i] V_i[r]
__global__ void k_combine(const c64 *V, int nv, const c64 *ycoef, c64 *out, int64_t n, int64_t nr) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t r = blockIdx.y;
    if (q >= n) return;
    c64 acc = {0, 0};
    for (int i = 0; i < nv; ++i) acc += ycoef[r * nv + i] * V[((int64_t)i * nr + r) * n + q];
    out[r * n + q] = acc;
}
// y[r] = a[r] * x[r] (per-rhs complex scale), or y = x - y (residual) with mode 1, or y += x (mode 2)
__global__ void k_axpy(int mode, const c64 *scale, const c64 *x, c64 *y, int64_t n, int64_t nr) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t r = blockIdx.y;
    if (q >= n) return;
    int64_t e = r * n + q;
    if (mode == 0) y[e] = scale[r] * x[e];
    else if (mode == 1) y[e] = x[e] - y[e];
    else y[e] = y[e] + x[e];
}

struct Work {
    fmbem *h;
    cudaStream_t s;
    int64_t n, nr;
    int nblocks;
    c64 *partial, *dres, *dcoef;
    std::vector<c64> hres;
    // dots[r][i] = <V_i[r], w[r]> for i < nv
    void dots(const c64 *V, int nv, const c64 *w, std::vector<cd> &out) {
        k_multidot<<<dim3(nblocks, nv, (unsigned)nr), DOT_TB, 0, s>>>(V, nv, w, n, nr, nblocks, partial);
        CKL("k_multidot");
        int64_t cnt = nr * nv;
        k_reduce_partials<<<nblk(cnt, 128), 128, 0, s>>>(partial, nblocks, cnt, dres);
        CKL("k_reduce_partials");
        hres.resize(cnt);
        CK(cudaMemcpyAsync(hres.data(), dres, sizeof(c64) * cnt, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        out.resize(cnt);
        for (int64_t e = 0; e < cnt; ++e) out[e] = cd(hres[e].re, hres[e].im);
    }
    void upload(const std::vector<cd> &c) {
        hres.resize(c.size());
        for (size_t e = 0; e < c.size(); ++e) hres[e] = c64{c[e].real(), c[e].imag()};
        CK(cudaMemcpyAsync(dcoef, hres.data(), sizeof(c64) * c.size(), cudaMemcpyHostToDevice, s));
    }
    void norms(const c64 *x, std::vector<double> &out) {
        std::vector<cd> d;
        dots(x, 1, x, d);  // with nv = 1 and V = x: per rhs <x_r, x_r>
        out.resize(nr);
        for (int64_t r = 0; r < nr; ++r) out[r] = std::sqrt(std::max(0.0, d[r].real()));
    }
};

}  // namespace

// one restarted GMRES solve of A x = rhs with the operator of the given precision; returns
// the iterations used per rhs; x is updated in place.  tol relative to ||rhs||.
static void gmres(fmbem *h, Work &W, int precision, const c64 *rhs, c64 *x, double tol, int max_iter,
                  std::vector<int> &its, std::vector<double> &relres, std::vector<char> &conv, bool &breakdown) {
    const int64_t n = W.n, nr = W.nr;
    const int m = std::max(1, h->opt.gmres_restart);
    c64 *V = h->sv;                       // (m+1) * nr * n
    c64 *z = V + (int64_t)(m + 1) * nr * n;
    c64 *w = z + nr * n;
    cudaStream_t s = W.s;
    std::vector<double> bn;
    W.norms(rhs, bn);
    its.assign(nr, 0);
    relres.assign(nr, 1.0);
    conv.assign(nr, 0);
    std::vector<double> rn;
    int total = 0;
    for (;;) {
        // true residual r = rhs - A x
        run_matvec(h, x, w, nr, precision, s);
        k_axpy<<<dim3(nblk(n, 256), (unsigned)nr), 256, 0, s>>>(1, nullptr, rhs, w, n, nr);
        CKL("k_axpy");
        W.norms(w, rn);
        bool all = true;
        for (int64_t r = 0; r < nr; ++r) {
            relres[r] = bn[r] > 0 ? rn[r] / bn[r] : 0.0;
            if (!std::isfinite(relres[r])) breakdown = true;
            conv[r] = relres[r] <= tol;
            all = all && conv[r];
        }
        if (all || breakdown || total >= max_iter) break;
        // V_0 = r / ||r||
        std::vector<cd> sc(nr);
        for (int64_t r = 0; r < nr; ++r) sc[r] = rn[r] > 0 ? cd(1.0 / rn[r], 0) : cd(0, 0);
        W.upload(sc);
        k_axpy<<<dim3(nblk(n, 256), (unsigned)nr), 256, 0, s>>>(0, W.dcoef, w, V, n, nr);
        CKL("k_axpy");
        std::vector<std::vector<cd>> H(nr, std::vector<cd>((m + 1) * m, cd(0, 0)));
        std::vector<std::vector<cd>> cs(nr, std::vector<cd>(m)), sn(nr, std::vector<cd>(m));
        std::vector<std::vector<cd>> g(nr, std::vector<cd>(m + 1, cd(0, 0)));
        for (int64_t r = 0; r < nr; ++r) g[r][0] = rn[r];
        int jdone = 0;
        for (int j = 0; j < m && total < max_iter; ++j) {
            run_precond(h, V + (int64_t)j * nr * n, z, nr, s);
            run_matvec(h, z, w, nr, precision, s);
            ++total;
            // classical Gram-Schmidt, twice
            std::vector<cd> hc(nr * (j + 1), cd(0, 0));
            for (int pass = 0; pass < 2; ++pass) {
                std::vector<cd> d;
                W.dots(V, j + 1, w, d);
                W.upload(d);
                k_subtract<<<dim3(nblk(n, 256), (unsigned)nr), 256, 0, s>>>(V, j + 1, W.dcoef, w, n, nr);
                CKL("k_subtract");
                for (size_t e = 0; e < d.size(); ++e) hc[e] += d[e];
            }
            std::vector<double> wn;
            W.norms(w, wn);
            for (int64_t r = 0; r < nr; ++r) {
                sc[r] = wn[r] > 1e-300 ? cd(1.0 / wn[r], 0) : cd(0, 0);
                if (!std::isfinite(wn[r])) breakdown = true;
            }
            W.upload(sc);
            k_axpy<<<dim3(nblk(n, 256), (unsigned)nr), 256, 0, s>>>(0, W.dcoef, w, V + (int64_t)(j + 1) * nr * n, n, nr);
            CKL("k_axpy");
            bool all = true;
            for (int64_t r = 0; r < nr; ++r) {
                std::vector<cd> &Hr = H[r];
                for (int i = 0; i <= j; ++i) Hr[i * m + j] = hc[r * (j + 1) + i];
                Hr[(j + 1) * m + j] = wn[r];
                for (int i = 0; i < j; ++i) {  // previous rotations
                    cd t = cs[r][i] * Hr[i * m + j] + sn[r][i] * Hr[(i + 1) * m + j];
                    Hr[(i + 1) * m + j] = -std::conj(sn[r][i]) * Hr[i * m + j] + std::conj(cs[r][i]) * Hr[(i + 1) * m + j];
                    Hr[i * m + j] = t;
                }
                cd a = Hr[j * m + j], b = Hr[(j + 1) * m + j];
                double den = std::sqrt(std::norm(a) + std::norm(b));
                if (den == 0) { cs[r][j] = 1; sn[r][j] = 0; }
                else { cs[r][j] = std::conj(a) / den; sn[r][j] = std::conj(b) / den; }
                Hr[j * m + j] = cs[r][j] * a + sn[r][j] * b;
                Hr[(j + 1) * m + j] = 0;
                g[r][j + 1] = -std::conj(sn[r][j]) * g[r][j];
                g[r][j] = cs[r][j] * g[r][j];
                double est = bn[r] > 0 ? std::abs(g[r][j + 1]) / bn[r] : 0.0;
                if (!std::isfinite(est)) breakdown = true;
                all = all && (est <= tol || wn[r] <= 1e-300);
            }
            jdone = j + 1;
            for (int64_t r = 0; r < nr; ++r) its[r] = total;
            if (all || breakdown) break;
        }
        // x += M^-1 V y
        std::vector<cd> yc(nr * jdone, cd(0, 0));
        for (int64_t r = 0; r < nr; ++r) {
            for (int i = jdone - 1; i >= 0; --i) {
                cd acc = g[r][i];
                for (int q = i + 1; q < jdone; ++q) acc -= H[r][i * m + q] * yc[r * jdone + q];
                cd d = H[r][i * m + i];
                yc[r * jdone + i] = std::abs(d) > 0 ? acc / d : cd(0, 0);
            }
        }
        W.upload(yc);
        k_combine<<<dim3(nblk(n, 256), (unsigned)nr), 256, 0, s>>>(V, jdone, W.dcoef, w, n, nr);
        CKL("k_combine");
        run_precond(h, w, z, nr, s);
        k_axpy<<<dim3(nblk(n, 256), (unsigned)nr), 256, 0, s>>>(2, nullptr, z, x, n, nr);
        CKL("k_axpy");
        if (breakdown) break;
    }
    for (int64_t r = 0; r < nr; ++r) its[r] = total;
}

fmbem_status run_solve(fmbem *h, const c64 *b, c64 *x, int64_t nr, double tol, int max_iter, int32_t *iters,
                       double *relres, cudaStream_t s) {
    const int m = std::max(1, h->opt.gmres_restart);
    const int64_t n = 6 * h->N;
    const bool refine = h->opt.solve_precision != FMBEM_FP64;
    size_t need = sizeof(c64) * ((size_t)(m + 1) * nr * n + 2 * nr * n + (refine ? 3 * nr * n : 0));
    if (h->sv_bytes < need) {
        if (h->sv) dev_free(h, h->sv);
        h->sv = (c64 *)dev_alloc(h, need);
        h->sv_bytes = need;
    }
    Work W;
    W.h = h;
    W.s = s;
    W.n = n;
    W.nr = nr;
    W.nblocks = (int)std::min<int64_t>(nblk(n, DOT_TB), 512);
    size_t pb = sizeof(c64) * (size_t)nr * (m + 1) * W.nblocks;
    W.partial = (c64 *)dev_alloc(h, pb);
    W.dres = (c64 *)dev_alloc(h, sizeof(c64) * nr * (m + 1));
    W.dcoef = (c64 *)dev_alloc(h, sizeof(c64) * nr * (m + 1));
    std::vector<int> its;
    std::vector<double> rr;
    std::vector<char> conv;
    bool breakdown = false;
    fmbem_status st = FMBEM_OK;
    try {
        if (!refine) {
            gmres(h, W, FMBEM_FP64, b, x, tol, max_iter, its, rr, conv, breakdown);
        } else {
            // iterative refinement: r = b - A x (outer_precision passes, FP64 vectors); solve
            // A32 d = r to inner_tol with the FP32 operator; x += d
            c64 *base = h->sv + (size_t)(m + 1) * nr * n + 2 * nr * n;
            c64 *r = base, *d = base + nr * n;
            std::vector<int> itot(nr, 0);
            std::vector<double> bn;
            W.norms(b, bn);
            for (int outer = 0;; ++outer) {
                run_matvec(h, x, r, nr, h->opt.outer_precision, s);
                k_axpy<<<dim3(nblk(n, 256), (unsigned)nr), 256, 0, s>>>(1, nullptr, b, r, n, nr);
                CKL("k_axpy");
                std::vector<double> rn;
                W.norms(r, rn);
                bool all = true;
                rr.assign(nr, 0);
                conv.assign(nr, 0);
                for (int64_t q = 0; q < nr; ++q) {
                    rr[q] = bn[q] > 0 ? rn[q] / bn[q] : 0.0;
                    if (!std::isfinite(rr[q])) breakdown = true;
                    conv[q] = rr[q] <= tol;
                    all = all && conv[q];
                }
                int used = *std::max_element(itot.begin(), itot.end());
                if (all || breakdown || used >= max_iter || outer > 50) break;
                CK(cudaMemsetAsync(d, 0, sizeof(c64) * nr * n, s));
                std::vector<int> ii;
                std::vector<double> ir;
                std::vector<char> ic;
                double itol = std::max(h->opt.inner_tol, 0.5 * tol);
                gmres(h, W, h->opt.solve_precision, r, d, itol, max_iter - used, ii, ir, ic, breakdown);
                for (int64_t q = 0; q < nr; ++q) itot[q] += ii[q];
                k_axpy<<<dim3(nblk(n, 256), (unsigned)nr), 256, 0, s>>>(2, nullptr, d, x, n, nr);
                CKL("k_axpy");
            }
            its = itot;
        }
        CK(cudaStreamSynchronize(s));
    } catch (...) {
        dev_free(h, W.partial);
        dev_free(h, W.dres);
        dev_free(h, W.dcoef);
        throw;
    }
    dev_free(h, W.partial);
    dev_free(h, W.dres);
    dev_free(h, W.dcoef);
    for (int64_t r = 0; r < nr; ++r) {
        if (iters) iters[r] = its[r];
        if (relres) relres[r] = rr[r];
        if (!conv[r]) st = FMBEM_ERR_NOT_CONVERGED;
    }
    if (breakdown) st = FMBEM_ERR_BREAKDOWN;
    return st;
}
