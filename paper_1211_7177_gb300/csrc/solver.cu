// solver.cu -- right-preconditioned restarted GMRES for A x = b (Eqs. 2.9, 3.1) with the
// block-diagonal preconditioner M = A_self (Eq. 3.2).  Each right-hand side has its own Krylov
// space; all of them share one batched matvec per iteration.  The host runs the small
// Hessenberg/Givens recurrences and the convergence tests in double precision.
//
// Two Krylov-basis precisions.  The plain solve keeps its basis in double precision and does
// every vector operation (classical Gram-Schmidt applied twice for the Arnoldi step, the second
// pass delayed by one step so that each step reads the basis twice) in double precision.  The
// inner iterations of the refined solve, which only have to reach a loose
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
// The same reduction with two right-hand vectors read in one pass over the basis: for
// i = 0..nv-1, partial[r][0][i][blk] = block sum of conj(V_i[r]) u[r] and partial[r][1][i][blk]
// of conj(V_i[r]) w[r] (u a basis-type vector, w a double vector)
template <typename TV, typename R, int MD_E>
__global__ void __launch_bounds__(DOT_TB) k_multidot2(const TV *V, int nv, const TV *u, const c64 *w, int64_t n,
                                                     int64_t nr, c64 *partial) {
    constexpr int G = MD_G / 2;
    __shared__ double sre[2 * G][DOT_TB / 32], sim[2 * G][DOT_TB / 32];
    const int64_t r = blockIdx.y;
    const int nblocks = gridDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t q0 = (int64_t)blockIdx.x * DOT_TB * MD_E + threadIdx.x;
    cx<R> uv[MD_E], wv[MD_E];
#pragma unroll
    for (int e = 0; e < MD_E; ++e) {
        const int64_t q = q0 + (int64_t)e * DOT_TB;
        uv[e] = q < n ? load_as<R>(u, r * n + q) : cx<R>{0, 0};
        wv[e] = q < n ? load_as<R>(w, r * n + q) : cx<R>{0, 0};
    }
    for (int i0 = 0; i0 < nv; i0 += G) {
        R re[2 * G], im[2 * G];
#pragma unroll
        for (int gI = 0; gI < G; ++gI) {
            re[gI] = im[gI] = re[G + gI] = im[G + gI] = 0;
            if (i0 + gI < nv) {
                const TV *a = V + ((int64_t)(i0 + gI) * nr + r) * n;
#pragma unroll
                for (int e = 0; e < MD_E; ++e) {
                    const int64_t q = q0 + (int64_t)e * DOT_TB;
                    if (q < n) {
                        const cx<R> x = load_as<R>(a, q);
                        re[gI] += x.re * uv[e].re + x.im * uv[e].im;
                        im[gI] += x.re * uv[e].im - x.im * uv[e].re;
                        re[G + gI] += x.re * wv[e].re + x.im * wv[e].im;
                        im[G + gI] += x.re * wv[e].im - x.im * wv[e].re;
                    }
                }
            }
        }
#pragma unroll
        for (int gI = 0; gI < 2 * G; ++gI)
            for (int off = 16; off > 0; off >>= 1) {
                re[gI] += __shfl_xor_sync(0xffffffffu, re[gI], off);
                im[gI] += __shfl_xor_sync(0xffffffffu, im[gI], off);
            }
        if (lane == 0)
#pragma unroll
            for (int gI = 0; gI < 2 * G; ++gI) {
                sre[gI][warp] = (double)re[gI];
                sim[gI][warp] = (double)im[gI];
            }
        __syncthreads();
        if (threadIdx.x < 2 * G) {
            const int k = threadIdx.x / G, gI = threadIdx.x % G;
            if (i0 + gI < nv) {
                double a = 0, b = 0;
                for (int t = 0; t < DOT_TB / 32; ++t) {
                    a += sre[threadIdx.x][t];
                    b += sim[threadIdx.x][t];
                }
                partial[((r * 2 + k) * nv + i0 + gI) * nblocks + blockIdx.x] = c64{a, b};
            }
        }
        __syncthreads();
    }
}
// The update of one delayed-CGS2 Arnoldi step (slot j of V holds u_j, the once-orthogonalised
// remainder of the previous step; w = A M^-1 u_j):
//   V_j     <- (u_j - sum_{i<j} s_i V_i) / alpha                       (u_j reorthogonalised)
//   V_{j+1} <- sw w - sum_{i<j} c_i V_i - cu u_j                       (w orthogonalised once,
//                                                                     c, cu and sw scaled by 1/|w|)
// coefficients per right-hand side: coef[r] = [s (j), c (j), cu, 1/alpha, sw], arithmetic R (all
// zero for a right-hand side frozen at an invariant space: both slots become zero)
template <typename TV, typename R>
__global__ void k_dcgs2_update(TV *V, int j, const cx<R> *coef, const c64 *w, int64_t n, int64_t nr) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t r = blockIdx.y;
    if (q >= n) return;
    const cx<R> *cs = coef + r * (2 * j + 3), *cc = cs + j;
    const cx<R> u = load_as<R>(V, ((int64_t)j * nr + r) * n + q);
    cx<R> v = u, x = cc[j + 2].re * load_as<R>(w, r * n + q);
    for (int i = 0; i < j; ++i) {
        const cx<R> a = load_as<R>(V, ((int64_t)i * nr + r) * n + q);
        v -= cs[i] * a;
        x -= cc[i] * a;
    }
    x -= cc[j] * u;
    v = cc[j + 1].re * v;
    V[((int64_t)j * nr + r) * n + q] = TV{v.re, v.im};
    V[((int64_t)(j + 1) * nr + r) * n + q] = TV{x.re, x.im};
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
    // d1[r][i] = <V_i[r], u[r]>, d2[r][i] = <V_i[r], w[r]> for i < nv, in one pass over V
    template <typename R, typename TV>
    void dots2(const TV *V, int nv, const TV *u, const c64 *w, std::vector<cd> &d1, std::vector<cd> &d2) {
        if (md_e == MD_E_BIG)
            k_multidot2<TV, R, MD_E_BIG><<<dim3(nblocks, (unsigned)nr), DOT_TB, 0, s>>>(V, nv, u, w, n, nr, partial);
        else
            k_multidot2<TV, R, MD_E_SMALL><<<dim3(nblocks, (unsigned)nr), DOT_TB, 0, s>>>(V, nv, u, w, n, nr, partial);
        CKL("k_multidot2");
        const int64_t cnt = nr * 2 * nv;
        k_reduce_partials<<<nblk(cnt * 32, 256), 256, 0, s>>>(partial, nblocks, cnt, dres);
        CKL("k_reduce_partials");
        hres.resize(cnt);
        CK(cudaMemcpyAsync(hres.data(), dres, sizeof(c64) * cnt, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        d1.resize(nr * nv);
        d2.resize(nr * nv);
        for (int64_t r = 0; r < nr; ++r)
            for (int i = 0; i < nv; ++i) {
                const c64 a = hres[(r * 2 + 0) * nv + i], b = hres[(r * 2 + 1) * nv + i];
                d1[r * nv + i] = cd(a.re, a.im);
                d2[r * nv + i] = cd(b.re, b.im);
            }
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
        // Arnoldi with classical Gram-Schmidt applied twice, the second pass delayed by one step
        // (DCGS2): slot j holds u_j, the previous step's remainder orthogonalised once; step j
        // forms w = A M^-1 u_j, then ONE reduction over slots 0..j gives s = V_{<j}^H u_j,
        // nu = |u_j|^2, t = V_{<j}^H w, tau = u_j^H w, and ONE update pass writes the twice-
        // orthogonalised v_j = (u_j - V s) / alpha (alpha^2 = nu - |s|^2) and the remainder
        // u_{j+1} = w - V_{<j} (t - s beta / alpha) - u_j beta / alpha (beta = v_j^H w).  Each step
        // reads the basis twice where two full passes read it four times.  Since u_j = V_{<j} s +
        // alpha v_j, column j - 1 of the Hessenberg matrix is known at step j:
        //   H[0..j-1][j-1] = ([t; beta]_{j-1} + s_j - H[0..j-1][0..j-2] s_{j-1}) / alpha_{j-1},
        //   H[j][j-1] = alpha_j / alpha_{j-1},
        // so the Givens rotation and the residual estimate of the j-dimensional space follow one
        // step behind the matvec (a converged cycle has made one matvec more than it uses); at
        // the restart a reduction over u_m alone closes the last column.
        std::vector<std::vector<cd>> H(nr, std::vector<cd>((m + 1) * m, cd(0, 0)));  // raw columns
        std::vector<std::vector<cd>> Hr(nr, std::vector<cd>((m + 1) * m, cd(0, 0)));  // rotated
        std::vector<std::vector<cd>> cs(nr, std::vector<cd>(m)), sn(nr, std::vector<cd>(m));
        std::vector<std::vector<cd>> g(nr, std::vector<cd>(m + 1, cd(0, 0)));
        std::vector<std::vector<double>> alpha(nr, std::vector<double>(m + 2, 1.0));
        // slot j + 1 holds sigma_{j+1} (w - ...) with sigma_{j+1} = 1 / |w| of step j, so that the
        // unnormalised remainders keep their size from step to step; the closure divides it out
        std::vector<std::vector<double>> sigma(nr, std::vector<double>(m + 2, 1.0));
        std::vector<std::vector<cd>> tb_prev(nr), s_prev(nr);
        // a right-hand side whose Krylov space has become invariant (u_j in the span of the basis
        // to rounding: alpha below eps_inv times the norm of the vector it came from) is frozen for
        // the rest of the cycle: H[j][j-1] = 0 (its estimate is then exact), and its later basis
        // vectors and columns are zero
        const double eps_inv = 64.0 * (sizeof(R) == 4 ? 5.96e-8 : 1.11e-16);
        std::vector<char> frozen(nr, 0);
        for (int64_t r = 0; r < nr; ++r) {
            g[r][0] = rn[r];
            if (!(rn[r] > 0)) frozen[r] = 1;
        }
        // closes column j - 1 from the reduction over u_j (sv = V_{<j}^H u_j, nu = |u_j|^2), sets
        // alpha_j (0 if frozen) and returns the residual estimate of the j-dimensional space
        auto close_column = [&](int64_t r, int j, const cd *sv, double nu) {
            std::vector<cd> &Hw = H[r], &R = Hr[r];
            const int c = j - 1;
            double a = 0;
            if (!frozen[r]) {
                const double sg = sigma[r][j];
                double ss = 0, pn = 0;
                for (int i = 0; i < j; ++i) ss += std::norm(sv[i]);
                for (const cd &v : tb_prev[r]) pn += std::norm(v);
                if (!std::isfinite(nu) || !std::isfinite(ss)) breakdown = true;
                a = std::sqrt(std::max(nu - ss, 0.0));
                for (int i = 0; i < j; ++i) {
                    cd v = tb_prev[r][i] + sv[i] / sg;
                    for (int k = 0; k < c; ++k) v -= Hw[i * m + k] * s_prev[r][k];
                    Hw[i * m + c] = v / alpha[r][c];
                }
                // |w_{j-1}|^2 = |[t; beta]|^2 + |u_j / sigma_j|^2
                if (a <= eps_inv * std::sqrt(nu + sg * sg * pn) || a <= 1e-300) {
                    frozen[r] = 1;
                    a = 0;
                }
                Hw[j * m + c] = a / sg / alpha[r][c];
            } else {
                for (int i = 0; i <= j; ++i) Hw[i * m + c] = 0;
            }
            alpha[r][j] = a;
            for (int i = 0; i <= j; ++i) R[i * m + c] = Hw[i * m + c];
            for (int i = 0; i < c; ++i) {  // previous rotations
                const cd t = cs[r][i] * R[i * m + c] + sn[r][i] * R[(i + 1) * m + c];
                R[(i + 1) * m + c] = -std::conj(sn[r][i]) * R[i * m + c] + std::conj(cs[r][i]) * R[(i + 1) * m + c];
                R[i * m + c] = t;
            }
            const cd x = R[c * m + c], y = R[(c + 1) * m + c];
            const double den = std::sqrt(std::norm(x) + std::norm(y));
            if (den == 0) { cs[r][c] = 1; sn[r][c] = 0; }
            else { cs[r][c] = std::conj(x) / den; sn[r][c] = std::conj(y) / den; }
            R[c * m + c] = cs[r][c] * x + sn[r][c] * y;
            R[(c + 1) * m + c] = 0;
            g[r][c + 1] = -std::conj(sn[r][c]) * g[r][c];
            g[r][c] = cs[r][c] * g[r][c];
            const double est = bn[r] > 0 ? std::abs(g[r][c + 1]) / bn[r] : 0.0;
            if (!std::isfinite(est)) breakdown = true;
            return est;
        };
        int jdone = 0;
        for (int j = 0; j <= m; ++j) {
            TV *u = V + (int64_t)j * nr * n;
            if (j == m || total >= max_iter) {  // close the last column: reduction over u_j only
                if (j > 0) {
                    std::vector<cd> d;
                    W.dots<R>(V, j + 1, u, d);
                    for (int64_t r = 0; r < nr; ++r) close_column(r, j, &d[r * (j + 1)], d[r * (j + 1) + j].real());
                }
                jdone = j;
                break;
            }
            precond(h, u, z, nr, s, tr);
            apply_op(h, z, w, nr, precision, s, tr);
            ++total;
            std::vector<cd> d1, d2;
            W.dots2<R>(V, j + 1, u, w, d1, d2);
            // per right-hand side [s (j), c (j), cu, 1 / alpha, w scale] for k_dcgs2_update
            const int nc = 2 * j + 3;
            std::vector<cd> coef(nr * nc, cd(0, 0));
            bool all = j > 0;
            for (int64_t r = 0; r < nr; ++r) {
                const cd *sv = &d1[r * (j + 1)], *tv = &d2[r * (j + 1)];
                if (j > 0) {
                    const double est = close_column(r, j, sv, d1[r * (j + 1) + j].real());
                    all = all && est <= tol;
                }
                if (frozen[r]) continue;  // its slots j and j + 1 become zero
                const double a = alpha[r][j];
                cd st(0, 0);
                for (int i = 0; i < j; ++i) st += std::conj(sv[i]) * tv[i];
                const cd beta = (d2[r * (j + 1) + j] - st) / a;
                const cd bs = beta / a;
                cd *cf = &coef[r * nc];
                for (int i = 0; i < j; ++i) {
                    cf[i] = sv[i];
                    cf[j + i] = tv[i] - sv[i] * bs;
                }
                cf[2 * j] = bs;
                cf[2 * j + 1] = cd(1.0 / a, 0);
                cf[2 * j + 2] = cd(1.0, 0);
                tb_prev[r].assign(tv, tv + j);
                tb_prev[r].push_back(beta);
                s_prev[r].assign(sv, sv + j);
            }
            for (int64_t r = 0; r < nr; ++r) its[r] = total;
            if (all || breakdown) {  // the space of dimension j suffices: the update is not needed
                jdone = j;
                break;
            }
            std::vector<double> wn;
            W.norms<R>(w, wn);
            for (int64_t r = 0; r < nr; ++r) {
                if (frozen[r]) continue;
                if (!std::isfinite(wn[r])) breakdown = true;
                const double sg = wn[r] > 1e-300 ? 1.0 / wn[r] : 0.0;
                sigma[r][j + 1] = sg;
                if (sg == 0) frozen[r] = 1;  // w = 0: the next column is zero
                cd *cf = &coef[r * nc];
                for (int i = 0; i < j; ++i) cf[j + i] *= sg;
                cf[2 * j] *= sg;
                cf[2 * j + 2] *= sg;
            }
            k_dcgs2_update<TV, R><<<grid, 256, 0, s>>>(V, j, W.upload<R>(coef), w, n, nr);
            CKL("k_dcgs2_update");
        }
        if (jdone == 0) break;
        // x += M^-1 V y
        std::vector<cd> yc(nr * jdone, cd(0, 0));
        for (int64_t r = 0; r < nr; ++r) {
            for (int i = jdone - 1; i >= 0; --i) {
                cd acc = g[r][i];
                for (int q = i + 1; q < jdone; ++q) acc -= Hr[r][i * m + q] * yc[r * jdone + q];
                cd d = Hr[r][i * m + i];
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
    // two right-hand vectors per reduction (k_multidot2), 2 m + 1 coefficients per right-hand side
    const size_t pb = sizeof(c64) * (size_t)nr * 2 * (m + 1) * W.nblocks;
    W.partial = (c64 *)dev_alloc(h, pb);
    W.dres = (c64 *)dev_alloc(h, sizeof(c64) * nr * 2 * (m + 1));
    W.dcoef = dev_alloc(h, sizeof(c64) * nr * (2 * m + 4));
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
