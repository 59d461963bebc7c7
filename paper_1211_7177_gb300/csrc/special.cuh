// special.cuh -- double-precision special functions for the multipole bases of Eqs. (2.14)-(2.16),
// evaluated on the device at set-up time.
//
//   Y_n^m(theta, phi) = (-1)^m sqrt((2n+1)/(4 pi) (n-|m|)!/(n+|m|)!) P_n^{|m|}(cos theta) e^{i m phi}
//   (Eq. 2.15; P_n^m without the Condon-Shortley phase), so that conj(Y_n^m) = Y_n^{-m} and the
//   addition theorem (2.14) holds with R_n^{-m} S_n^m.
//   R_n^m(r) = j_n(k|r|) Y_n^m(rhat),  S_n^m(r) = h_n^(1)(k|r|) Y_n^m(rhat)   (Eq. 2.16)
//   for complex k.
//
// Coefficient index of (n, m): n*n + n + m, n = 0..p-1.
#pragma once
#include "fmbem_internal.cuh"

__host__ __device__ __forceinline__ int nm_index(int n, int m) { return n * n + n + m; }

// fully normalised associated Legendre values Pb[n][m] = sqrt((2n+1)/(4pi)(n-m)!/(n+m)!) P_n^m(x),
// 0 <= m <= n <= nmax, unphased, by the standard three-term recurrences in n.
// Storage: Pb[n*(n+1)/2 + m].
__device__ inline void legendre_bar(int nmax, double x, double *Pb) {
    double s = sqrt(fmax(0.0, 1.0 - x * x));
    Pb[0] = 0.28209479177387814347;  // 1/sqrt(4 pi)
    for (int m = 1; m <= nmax; ++m) {
        int i = m * (m + 1) / 2 + m, j = (m - 1) * m / 2 + (m - 1);
        Pb[i] = sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * Pb[j];
    }
    for (int m = 0; m < nmax; ++m) {
        int i = (m + 1) * (m + 2) / 2 + m, j = m * (m + 1) / 2 + m;
        Pb[i] = sqrt(2.0 * m + 3.0) * x * Pb[j];
    }
    for (int m = 0; m <= nmax; ++m)
        for (int n = m + 2; n <= nmax; ++n) {
            double a = sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
            double b = sqrt(((n - 1.0) * (n - 1.0) - (double)m * m) / (4.0 * (n - 1.0) * (n - 1.0) - 1.0));
            Pb[n * (n + 1) / 2 + m] = a * (x * Pb[(n - 1) * n / 2 + m] - b * Pb[(n - 2) * (n - 1) / 2 + m]);
        }
}

// spherical Bessel j_n(z), n = 0..nmax, complex z.  |z| < 1: power series
//   j_n(z) = z^n/(2n+1)!! sum_s (-z^2/2)^s / (s! (2n+3)(2n+5)...(2n+2s+1));
// otherwise Miller's backward recurrence f_{n-1} = (2n+1)/z f_n - f_{n+1}, normalised by whichever
// of j_0 = sin z / z and j_1 = sin z/z^2 - cos z/z is larger in modulus.
__device__ inline void sph_j(int nmax, c64 z, c64 *out) {
    double az = cabsd(z);
    if (az < 1.0) {
        c64 z2h = -0.5 * (z * z);
        c64 zn = {1.0, 0.0};
        double df = 1.0;  // (2n+1)!!
        for (int n = 0; n <= nmax; ++n) {
            if (n > 0) { zn = zn * z; df *= (2.0 * n + 1.0); }
            c64 term = {1.0, 0.0}, sum = {1.0, 0.0};
            for (int s = 1; s < 40; ++s) {
                term = cdiv(term * z2h, c64{(double)s * (2.0 * n + 2.0 * s + 1.0), 0.0});
                sum += term;
                if (abs2(term) < 1e-36 * abs2(sum)) break;
            }
            out[n] = (1.0 / df) * (zn * sum);
        }
        return;
    }
    int nstart = nmax + 16 + (int)(az);
    c64 fp1 = {0.0, 0.0}, f = {1e-30, 0.0};  // f = f_{n}, fp1 = f_{n+1}, n = nstart
    c64 zinv = cdiv(c64{1.0, 0.0}, z);
    for (int n = nstart; n >= 1; --n) {
        c64 fm1 = ((2.0 * n + 1.0) * (zinv * f)) - fp1;
        fp1 = f;
        f = fm1;                               // now f = f_{n-1}
        if (n - 1 <= nmax) out[n - 1] = f;
        if (abs2(f) > 1e200) {                 // rescale the recurrence and everything stored
            const double sc = 1e-100;
            f = sc * f;
            fp1 = sc * fp1;
            for (int q = n - 1; q <= nmax; ++q)
                if (q >= 0) out[q] = sc * out[q];
        }
    }
    c64 f0, f1;
    f0 = out[0];
    f1 = nmax >= 1 ? out[1] : fp1;
    // sin z, cos z for complex z
    double sr, cr;
    sincos(z.re, &sr, &cr);
    double sh = sinh(z.im), ch = cosh(z.im);
    c64 sinz = {sr * ch, cr * sh}, cosz = {cr * ch, -sr * sh};
    c64 j0 = sinz * zinv;
    c64 j1 = sinz * zinv * zinv - cosz * zinv;
    c64 scale = abs2(j0) >= abs2(j1) ? cdiv(j0, f0) : cdiv(j1, f1);
    for (int n = 0; n <= nmax; ++n) out[n] = out[n] * scale;
}

// spherical Hankel h_n^(1)(z), n = 0..nmax, by upward recurrence from
// h_0 = -i e^{iz}/z, h_1 = -e^{iz}(z + i)/z^2.
__device__ inline void sph_h1(int nmax, c64 z, c64 *out) {
    c64 eiz = cexpd(c64{-z.im, z.re});
    c64 zinv = cdiv(c64{1.0, 0.0}, z);
    out[0] = c64{0.0, -1.0} * eiz * zinv;
    if (nmax >= 1) out[1] = -(eiz * (z + c64{0.0, 1.0}) * zinv * zinv);
    for (int n = 1; n < nmax; ++n) out[n + 1] = ((2.0 * n + 1.0) * (zinv * out[n])) - out[n - 1];
}

// R_n^m (regular, j_n) or S_n^m (singular, h_n) at r for n = 0..nmax: out[nm_index(n,m)].
// work: needs (nmax+1) complex radial values and (nmax+1)(nmax+2)/2 Legendre values.
template <bool SINGULAR>
__device__ inline void wave_functions(int nmax, c64 k, const double r[3], c64 *out, c64 *rad, double *Pb) {
    double rr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double ct = rr > 0 ? r[2] / rr : 1.0;
    double phi = (r[0] == 0.0 && r[1] == 0.0) ? 0.0 : atan2(r[1], r[0]);
    c64 z = k * rr;
    if (SINGULAR) sph_h1(nmax, z, rad);
    else {
        if (rr == 0.0) { rad[0] = {1.0, 0.0}; for (int n = 1; n <= nmax; ++n) rad[n] = {0.0, 0.0}; }
        else sph_j(nmax, z, rad);
    }
    legendre_bar(nmax, ct, Pb);
    for (int m = 0; m <= nmax; ++m) {
        double sp, cp;
        sincos(m * phi, &sp, &cp);
        double sgn = (m & 1) ? -1.0 : 1.0;  // (-1)^m, the same for +m and -m
        for (int n = m; n <= nmax; ++n) {
            double a = sgn * Pb[n * (n + 1) / 2 + m];
            c64 v = rad[n] * a;
            out[nm_index(n, m)] = v * c64{cp, sp};
            if (m > 0) out[nm_index(n, -m)] = v * c64{cp, -sp};
        }
    }
}

// gradient of R_n^m for n = 0..nmax-1 from R up to degree nmax (ladder relations that follow from
// the plane-wave representation R_n^m(r) = (4 pi i^n)^{-1} int exp(i k s.r) Y_n^m(s) dOmega_s):
//   d_z R_n^m        = k [ a_{n-1}^m R_{n-1}^m - a_n^m R_{n+1}^m ]
//   (d_x + i d_y) R_n^m = k sgn(m)  [ b2(n,m) R_{n-1}^{m+1} + b1(n,m) R_{n+1}^{m+1} ]
//   (d_x - i d_y) R_n^m = k sgn(-m) [ b2(n,-m) R_{n-1}^{m-1} + b1(n,-m) R_{n+1}^{m-1} ]
//   a_n^m = sqrt((n+1+m)(n+1-m)/((2n+1)(2n+3))),  b1(n,m) = sqrt((n+m+1)(n+m+2)/((2n+1)(2n+3))),
//   b2(n,m) = sqrt((n-m)(n-m-1)/((2n-1)(2n+1))),  sgn(m) = +1 for m >= 0 and -1 for m < 0.
__device__ __forceinline__ c64 Rget(const c64 *R, int nmax, int n, int m) {
    if (n < 0 || n > nmax || m < -n || m > n) return c64{0.0, 0.0};
    return R[nm_index(n, m)];
}
__device__ inline void grad_regular(int p, c64 k, const c64 *R /* up to degree p */, int n, int m, c64 g[3]) {
    auto a = [](int nn, int mm) -> double {
        if (nn < 0) return 0.0;
        return sqrt((double)(nn + 1 + mm) * (nn + 1 - mm) / ((2.0 * nn + 1.0) * (2.0 * nn + 3.0)));
    };
    auto b1 = [](int nn, int mm) -> double {
        return sqrt((double)(nn + mm + 1) * (nn + mm + 2) / ((2.0 * nn + 1.0) * (2.0 * nn + 3.0)));
    };
    auto b2 = [](int nn, int mm) -> double {
        if (nn < 1) return 0.0;
        double v = (double)(nn - mm) * (nn - mm - 1);
        return v <= 0 ? 0.0 : sqrt(v / ((2.0 * nn - 1.0) * (2.0 * nn + 1.0)));
    };
    c64 dz = k * (a(n - 1, m) * Rget(R, p, n - 1, m) - a(n, m) * Rget(R, p, n + 1, m));
    double sp = m >= 0 ? 1.0 : -1.0, sm = m <= 0 ? 1.0 : -1.0;
    c64 dp = (sp * k) * (b2(n, m) * Rget(R, p, n - 1, m + 1) + b1(n, m) * Rget(R, p, n + 1, m + 1));
    c64 dm = (sm * k) * (b2(n, -m) * Rget(R, p, n - 1, m - 1) + b1(n, -m) * Rget(R, p, n + 1, m - 1));
    g[0] = 0.5 * (dp + dm);
    c64 d = dp - dm;  // (dp - dm) / (2i)
    g[1] = c64{0.5 * d.im, -0.5 * d.re};
    g[2] = dz;
}
