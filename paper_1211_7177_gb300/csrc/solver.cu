// solver.cu -- right-preconditioned restarted GMRES for A x = b (Eqs. 2.9, 3.1) with the
// block-diagonal preconditioner M = A_self (Eq. 3.2).  Each right-hand side has its own Krylov
// space; all of them share one batched matvec per iteration.  The host runs the small
// Hessenberg/Givens recurrences and the convergence tests in double precision.
//
// Two Krylov-basis precisions.  The plain solve keeps its basis in double precision and does
// every vector operation (classical Gram-Schmidt applied twice for the Arnoldi step) in double
// precision.  The inner iterations of the refined solve, which only have to reach a loose
// tolerance against a single-precision operator, keep the basis in single precision and do the
// vector arithmetic in single precision, with the per-block partial sums of the inner products
// combined in double precision; GB300 runs FP64 at 1/62 of its FP32 rate, so double-precision
// Gram-Schmidt over 128 right-hand sides would cost as much as the matvec itself.  The outer
// residuals, corrections and the solution of the refined solve stay in double precision.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "fmbem_internal.cuh"

namespace {

using cd = std::complex<double>;
constexpr int DOT_TB = 256;
// elements of each vector per thread in the inner products: 16 when that still gives several
// blocks per SM (batches), 4 otherwise (a single right-hand side)
constexpr int MD_E_BIG = 16, MD_E_SMALL = 4;
constexpr int MD_G = 8;  // basis vectors per block reduction

inline unsigned nblk(int64_t n, int tb) { return (unsigned)((n + tb - 1) / tb); }

template <typename R, typename T>
__device__ __forceinline__ cx<R> load_as(const T *p, int64_t i) {
    const T v = p[i];
    return cx<R>{(R)v.re, (R)v.im};
}

// partial[r][i][blk] = sum over the block's DOT_TB * MD_E elements of conj(V_i[r]) w[r] for
// i = 0..nv-1 (V_i[r] at V + (i * nr + r) * n), in arithmetic R; the warps' sums are combined
// in double precision.  The block keeps its slice of w in registers and walks the basis vectors
// MD_G at a time, so w is read once and every basis vector once.
template <typename TV, typename TW, typename R, int MD_E>
__global__ void __launch_bounds__(DOT_TB) k_multidot(const TV *V, int nv, const TW *w, int64_t n, int64_t nr,
                                                    c64 *partial) {
    __shared__ double sre[MD_G][DOT_TB / 32], sim[MD_G][DOT_TB / 32];
    const int64_t r = blockIdx.y;
    const int nblocks = gridDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t q0 = (int64_t)blockIdx.x * DOT_TB * MD_E + threadIdx.x;
    cx<R> wv[MD_E];
#pragma unroll
    for (int e = 0; e < MD_E; ++e) {
        const int64_t q = q0 + (int64_t)e * DOT_TB;
        wv[e] = q < n ? load_as<R>(w, r * n + q) : cx<R>{0, 0};
    }
    for (int i0 = 0; i0 < nv; i0 += MD_G) {
        R re[MD_G], im[MD_G];
#pragma unroll
        for (int gI = 0; gI < MD_G; ++gI) {
            re[gI] = 0;
            im[gI] = 0;
            if (i0 + gI < nv) {
                const TV *a = V + ((int64_t)(i0 + gI) * nr + r) * n;
#pragma unroll
                for (int e = 0; e < MD_E; ++e) {
                    const int64_t q = q0 + (int64_t)e * DOT_TB;
                    if (q < n) {
                        const cx<R> x = load_as<R>(a, q);
                        re[gI] += x.re * wv[e].re + x.im * wv[e].im;
                        im[gI] += x.re * wv[e].im - x.im * wv[e].re;
                    }
                }
            }
        }
#pragma unroll
        for (int gI = 0; gI < MD_G; ++gI)
            for (int off = 16; off > 0; off >>= 1) {
                re[gI] += __shfl_xor_sync(0xffffffffu, re[gI], off);
                im[gI] += __shfl_xor_sync(0xffffffffu, im[gI], off);
            }
        if (lane == 0)
#pragma unroll
            for (int gI = 0; gI < MD_G; ++gI) {
                sre[gI][warp] = (double)re[gI];
                sim[gI][warp] = (double)im[gI];
            }
        __syncthreads();
        if (threadIdx.x < MD_G && i0 + (int)threadIdx.x < nv) {
            double a = 0, b = 0;
            for (int k = 0; k < DOT_TB / 32; ++k) {
                a += sre[threadIdx.x][k];
                b += sim[threadIdx.x][k];
            }
            partial[(r * nv + i0 + threadIdx.x) * nblocks + blockIdx.x] = c64{a, b};
        }
        __syncthreads();
    }
}
// out[e] = sum over blocks of partial[e][blk], one warp per output, fixed order
__global__ void k_reduce_partials(const c64 *partial, int nblocks, int64_t count, c64 *out) {
    const int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (e >= count) return;
    double re = 0, im = 0;
    for (int b = lane; b < nblocks; b += 32) {
        const c64 v = partial[e * nblocks + b];
        re += v.re;
        im += v.im;
    }
    for (int off = 16; off > 0; off >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, off);
        im += __shfl_xor_sync(0xffffffffu, im, off);
    }
    if (lane == 0) out[e] = c64{re, im};
}
// w[r] -= sum_i h[r][i] V_i[r], arithmetic R (coefficients given in R)
template <typename TV, typename R>
__global__ void k_subtract(const TV *V, int nv, const cx<R> *hcoef, c64 *w, int64_t n, int64_t nr) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t r = blockIdx.y;
    if (q >= n) return;
    cx<R> acc = load_as<R>(w, r * n + q);
    for (int i = 0; i < nv; ++i) acc -= hcoef[r * nv + i] * load_as<R>(V, ((int64_t)i * nr + r) * n + q);
    w[r * n + q] = c64{(double)acc.re, (double)acc.im};
}
// out[r] = sum_i y[r][i] V_i[r], arithmetic R, out of element type TO
template <typename TV, typename R, typename TO>
__global__ void k_combine(const TV *V, int nv, const cx<R> *ycoef, TO *out, int64_t n, int64_t nr) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t r = blockIdx.y;
    if (q >= n) return;
    cx<R> acc = {0, 0};
    for (int i = 0; i < nv; ++i) acc += ycoef[r * nv + i] * load_as<R>(V, ((int64_t)i * nr + r) * n + q);
    out[r * n + q] = TO{acc.re, acc.im};
}
// y[r] = a[r] x[r] (per-rhs complex scale), arithmetic R, y of element type TV
template <typename R, typename TV>
__global__ void k_scale(const cx<R> *scale, const c64 *x, TV *y, int64_t n, int64_t nr) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t r = blockIdx.y;
    if (q >= n) return;
    const cx<R> v = scale[r] * load_as<R>(x, r * n + q);
    y[r * n + q] = TV{v.re, v.im};
}
// y = x - y (residual) with mode 1, or y += x (mode 2)
__global__ void k_axpy(int mode, const c64 *x, c64 *y, int64_t n, int64_t nr) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t r = blockIdx.y;
    if (q >= n) return;
    const int64_t e = r * n + q;
    if (mode == 1) y[e] = x[e] - y[e];
    else y[e] = y[e] + x[e];
}

struct Work {
    fmbem *h;
    cudaStream_t s;
    int64_t n, nr;
    int nblocks, md_e;
    c64 *partial, *dres;
    void *dcoef;
    std::vector<c64> hres;
    std::vector<c32> hres32;
    // dots[r][i] = <V_i[r], w[r]> for i < nv, arithmetic R
    template <typename R, typename TV, typename TW>
    void dots(const TV *V, int nv, const TW *w, std::vector<cd> &out) {
        if (md_e == MD_E_BIG)
            k_multidot<TV, TW, R, MD_E_BIG><<<dim3(nblocks, (unsigned)nr), DOT_TB, 0, s>>>(V, nv, w, n, nr, partial);
        else
            k_multidot<TV, TW, R, MD_E_SMALL><<<dim3(nblocks, (unsigned)nr), DOT_TB, 0, s>>>(V, nv, w, n, nr, partial);
        CKL("k_multidot");
        const int64_t cnt = nr * nv;
        k_reduce_partials<<<nblk(cnt * 32, 256), 256, 0, s>>>(partial, nblocks, cnt, dres);
        CKL("k_reduce_partials");
        hres.resize(cnt);
        CK(cudaMemcpyAsync(hres.data(), dres, sizeof(c64) * cnt, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        out.resize(cnt);
        for (int64_t e = 0; e < cnt; ++e) out[e] = cd(hres[e].re, hres[e].im);
    }
    // coefficients to the device in arithmetic R
    template <typename R>
    const cx<R> *upload(const std::vector<cd> &c) {
        if (sizeof(R) == sizeof(double)) {
            hres.resize(c.size());
            for (size_t e = 0; e < c.size(); ++e) hres[e] = c64{c[e].real(), c[e].imag()};
            CK(cudaMemcpyAsync(dcoef, hres.data(), sizeof(c64) * c.size(), cudaMemcpyHostToDevice, s));
        } else {
            hres32.resize(c.size());
            for (size_t e = 0; e < c.size(); ++e) hres32[e] = c32{(float)c[e].real(), (float)c[e].imag()};
            CK(cudaMemcpyAsync(dcoef, hres32.data(), sizeof(c32) * c.size(), cudaMemcpyHostToDevice, s));
        }
        return (const cx<R> *)dcoef;
    }
    template <typename R>
    void norms(const c64 *x, std::vector<double> &out) {
        std::vector<cd> d;
        dots<R>(x, 1, x, d);  // with nv = 1 and V = x: per rhs <x_r, x_r>
        out.resize(nr);
        for (int64_t r = 0; r < nr; ++r) out[r] = std::sqrt(std::max(0.0, d[r].real()));
    }
};

// M^-1 (or M^-T for the adjoint solve) applied to a basis vector: the LU of Eq. (3.2) in double
// precision for a double basis, the single-precision explicit inverse for a single basis
void precond(fmbem *h, const c64 *v, c64 *z, int64_t nr, cudaStream_t s, bool tr) {
    if (tr) run_precond_t(h, v, z, nr, s);
    else run_precond(h, v, z, nr, s);
}
void precond(fmbem *h, const c32 *v, c64 *z, int64_t nr, cudaStream_t s, bool tr) { run_precond32(h, v, z, nr, s, tr); }

// the operator of the solve: A (Eq. 2.9) or, for the adjoint solve, A^T
void apply_op(fmbem *h, const c64 *x, c64 *y, int64_t nr, int precision, cudaStream_t s, bool tr) {
    if (tr) run_adjoint_matvec(h, x, y, nr, precision, s);
    else run_matvec(h, x, y, nr, precision, s);
}

// basis element type -> arithmetic of its vector operations
template <typename TV>
struct ArithOf;
template <>
struct ArithOf<c64> {
    using R = double;
};
template <>
struct ArithOf<c32> {
    using R = float;
};

// one restarted GMRES solve of A x = rhs with the operator of the given precision and a Krylov
// basis of element type TV; returns the iterations used per rhs; x is updated in place.  tol is
// relative to ||rhs||.  V holds (m + 2) vectors of nr * n elements of TV (the last one is scratch
// for the final combination); z and w are nr * n double vectors.
template <typename TV>
// x_zero: x is zero on entry, so the first residual is the right-hand side (no product)
void gmres(fmbem *h, Work &W, int precision, bool tr, const c64 *rhs, c64 *x, double tol, int max_iter, TV *V, c64 *z,
           c64 *w, std::vector<int> &its, std::vector<double> &relres, std::vector<char> &conv, bool &breakdown,
           bool x_zero) {
    using R = typename ArithOf<TV>::R;
    const int64_t n = W.n, nr = W.nr;
    const int m = std::max(1, h->opt.gmres_restart);
    TV *tmp = V + (int64_t)(m + 1) * nr * n;
    cudaStream_t s = W.s;
    const dim3 grid(nblk(n, 256), (unsigned)nr);
    std::vector<double> bn;
    W.norms<double>(rhs, bn);
    its.assign(nr, 0);
    relres.assign(nr, 1.0);
    conv.assign(nr, 0);
    std::vector<double> rn;
    int total = 0;
    bool first = true;
    for (;;) {
        // true residual r = rhs - A x
        if (first && x_zero) CK(cudaMemsetAsync(w, 0, sizeof(c64) * (size_t)nr * n, s));
        else apply_op(h, x, w, nr, precision, s, tr);
        first = false;
        k_axpy<<<grid, 256, 0, s>>>(1, rhs, w, n, nr);
        CKL("k_axpy");
        W.norms<double>(w, rn);
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
        k_scale<R, TV><<<grid, 256, 0, s>>>(W.upload<R>(sc), w, V, n, nr);
        CKL("k_scale");
        std::vector<std::vector<cd>> H(nr, std::vector<cd>((m + 1) * m, cd(0, 0)));
        std::vector<std::vector<cd>> cs(nr, std::vector<cd>(m)), sn(nr, std::vector<cd>(m));
        std::vector<std::vector<cd>> g(nr, std::vector<cd>(m + 1, cd(0, 0)));
        for (int64_t r = 0; r < nr; ++r) g[r][0] = rn[r];
        int jdone = 0;
        for (int j = 0; j < m && total < max_iter; ++j) {
            precond(h, V + (int64_t)j * nr * n, z, nr, s, tr);
            apply_op(h, z, w, nr, precision, s, tr);
            ++total;
            // classical Gram-Schmidt, twice (a Daniel-Gragg-Kaufman-Stewart test for skipping the
            // second pass found it needed in 199 of 202 iterations of the 128-RHS torus solve)
            std::vector<cd> hc(nr * (j + 1), cd(0, 0));
            for (int pass = 0; pass < 2; ++pass) {
                std::vector<cd> d;
                W.dots<R>(V, j + 1, w, d);
                k_subtract<TV, R><<<grid, 256, 0, s>>>(V, j + 1, W.upload<R>(d), w, n, nr);
                CKL("k_subtract");
                for (size_t e = 0; e < d.size(); ++e) hc[e] += d[e];
            }
            std::vector<double> wn;
            W.norms<R>(w, wn);
            for (int64_t r = 0; r < nr; ++r) {
                sc[r] = wn[r] > 1e-300 ? cd(1.0 / wn[r], 0) : cd(0, 0);
                if (!std::isfinite(wn[r])) breakdown = true;
            }
            k_scale<R, TV><<<grid, 256, 0, s>>>(W.upload<R>(sc), w, V + (int64_t)(j + 1) * nr * n, n, nr);
            CKL("k_scale");
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
        k_combine<TV, R, TV><<<grid, 256, 0, s>>>(V, jdone, W.upload<R>(yc), tmp, n, nr);
        CKL("k_combine");
        precond(h, tmp, z, nr, s, tr);
        k_axpy<<<grid, 256, 0, s>>>(2, z, x, n, nr);
        CKL("k_axpy");
        if (breakdown) break;
    }
    for (int64_t r = 0; r < nr; ++r) its[r] = total;
}

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

fmbem_status run_solve(fmbem *h, const c64 *b, c64 *x, int64_t nr, double tol, int max_iter, int32_t *iters,
                       double *relres, cudaStream_t s, bool transpose) {
    const int m = std::max(1, h->opt.gmres_restart);
    const int64_t n = 6 * h->N;
    const bool refine = h->opt.solve_precision != FMBEM_FP64;
    // [basis: (m + 2) vectors of the basis type][z][w][refined solve: r, d], double vectors
    const size_t vec = sizeof(c64) * (size_t)nr * n;
    const size_t basis_bytes = round256((refine ? sizeof(c32) : sizeof(c64)) * (size_t)(m + 2) * nr * n);
    const size_t need = basis_bytes + (refine ? 4 : 2) * vec;
    if (h->sv_bytes < need) {
        if (h->sv) dev_free(h, h->sv);
        h->sv = nullptr;
        h->sv_bytes = 0;
        h->sv = (c64 *)dev_alloc(h, need);
        h->sv_bytes = need;
    }
    unsigned char *base = (unsigned char *)h->sv;
    c64 *z = (c64 *)(base + basis_bytes), *w = z + nr * n;
    Work W;
    W.h = h;
    W.s = s;
    W.n = n;
    W.nr = nr;
    W.md_e = (int64_t)nr * nblk(n, DOT_TB * MD_E_BIG) >= 8 * 152 ? MD_E_BIG : MD_E_SMALL;
    W.nblocks = (int)nblk(n, DOT_TB * W.md_e);
    const size_t pb = sizeof(c64) * (size_t)nr * (m + 1) * W.nblocks;
    W.partial = (c64 *)dev_alloc(h, pb);
    W.dres = (c64 *)dev_alloc(h, sizeof(c64) * nr * (m + 1));
    W.dcoef = dev_alloc(h, sizeof(c64) * nr * (m + 1));
    std::vector<int> its;
    std::vector<double> rr;
    std::vector<char> conv;
    bool breakdown = false;
    fmbem_status st = FMBEM_OK;
    const dim3 grid(nblk(n, 256), (unsigned)nr);
    try {
        // a zero initial guess (the usual one) makes the first residual b itself
        std::vector<double> xn;
        W.norms<double>(x, xn);
        const bool x_zero = std::all_of(xn.begin(), xn.end(), [](double v) { return v == 0.0; });
        if (!refine) {
            gmres<c64>(h, W, FMBEM_FP64, transpose, b, x, tol, max_iter, (c64 *)base, z, w, its, rr, conv, breakdown,
                       x_zero);
        } else {
            // iterative refinement: r = b - A x (outer_precision passes, double vectors); solve
            // A' d = r to inner_tol with the FP32 or TF32 operator and a single-precision basis;
            // x += d
            c64 *r = w + nr * n, *d = r + nr * n;
            std::vector<int> itot(nr, 0);
            std::vector<double> bn;
            W.norms<double>(b, bn);
            for (int outer = 0;; ++outer) {
                if (outer == 0 && x_zero) CK(cudaMemsetAsync(r, 0, vec, s));
                else apply_op(h, x, r, nr, h->opt.outer_precision, s, transpose);
                k_axpy<<<grid, 256, 0, s>>>(1, b, r, n, nr);
                CKL("k_axpy");
                std::vector<double> rn;
                W.norms<double>(r, rn);
                bool all = true;
                rr.assign(nr, 0);
                conv.assign(nr, 0);
                for (int64_t q = 0; q < nr; ++q) {
                    rr[q] = bn[q] > 0 ? rn[q] / bn[q] : 0.0;
                    if (!std::isfinite(rr[q])) breakdown = true;
                    conv[q] = rr[q] <= tol;
                    all = all && conv[q];
                }
                const int used = *std::max_element(itot.begin(), itot.end());
                if (all || breakdown || used >= max_iter || outer > 50) break;
                CK(cudaMemsetAsync(d, 0, vec, s));
                std::vector<int> ii;
                std::vector<double> ir;
                std::vector<char> ic;
                const double itol = std::max(h->opt.inner_tol, 0.5 * tol);
                gmres<c32>(h, W, h->opt.solve_precision, transpose, r, d, itol, max_iter - used, (c32 *)base, z, w, ii,
                           ir, ic, breakdown, true);  // d = 0
                for (int64_t q = 0; q < nr; ++q) itot[q] += ii[q];
                k_axpy<<<grid, 256, 0, s>>>(2, d, x, n, nr);
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
