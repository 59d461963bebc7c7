"""Mie series for a homogeneous sphere under a plane wave (Bohren & Huffman, the textbook the paper
cites for its sphere checks in Section 3.2 and Appendix D).

TEST INFRASTRUCTURE ONLY: used by the oracle's own pins and by the tests; no product code
imports it.

Conventions: time factor exp(-i omega t) as in Section 2.1; background relative permittivity 1
and permeability 1 (wavenumber k), sphere of radius ``a`` centred at the origin with relative
permittivity ``eps_in`` and permeability 1; incident field E_inc = x exp(i k z).  Fields are
expanded in the vector spherical harmonics M_{o1n}, M_{e1n}, N_{o1n}, N_{e1n} of Bohren &
Huffman Eq. (4.50), with the angular functions pi_n = P_n^1/sin(theta), tau_n = dP_n^1/dtheta.
"""
from __future__ import annotations

import numpy as np
from scipy.special import spherical_jn, spherical_yn


def _psi(n, z):
    return z * spherical_jn(n, z)


def _dpsi(n, z):
    return spherical_jn(n, z) + z * spherical_jn(n, z, derivative=True)


def _h1(n, z):
    return spherical_jn(n, z) + 1j * spherical_yn(n, z)


def _dh1(n, z):
    return spherical_jn(n, z, derivative=True) + 1j * spherical_yn(n, z, derivative=True)


def _xi(n, z):
    return z * _h1(n, z)


def _dxi(n, z):
    return _h1(n, z) + z * _dh1(n, z)


def default_nmax(x):
    return int(np.ceil(abs(x) + 4.05 * abs(x) ** (1.0 / 3.0) + 8))


def coefficients(eps_in, x, nmax=None):
    """Scattering (a_n, b_n) and internal (c_n, d_n) coefficients, n = 1..nmax, for size
    parameter x = k a and relative index m = sqrt(eps_in) (principal root, Im m >= 0)."""
    if nmax is None:
        nmax = default_nmax(x)
    m = np.sqrt(complex(eps_in))
    if m.imag < 0:
        m = -m
    n = np.arange(1, nmax + 1)
    mx = m * x
    px, dpx = _psi(n, x), _dpsi(n, x)
    pm, dpm = _psi(n, mx), _dpsi(n, mx)
    xx, dxx = _xi(n, x), _dxi(n, x)
    a = (m * pm * dpx - px * dpm) / (m * pm * dxx - xx * dpm)
    b = (pm * dpx - m * px * dpm) / (pm * dxx - m * xx * dpm)
    c = (m * px * dxx - m * xx * dpx) / (pm * dxx - m * xx * dpm)
    d = (m * px * dxx - m * xx * dpx) / (m * pm * dxx - xx * dpm)
    return a, b, c, d


def ibc_coefficients(eta, x, nmax=None):
    """Scattering coefficients (a_n, b_n), n = 1..nmax, of a sphere whose surface obeys the
    impedance condition of Eq. (2.24), n x E = Z n x (n x H), with eta = Z / Z_background.
    From E_t = Z (r x H) at r = a with the total exterior field of Bohren & Huffman Eqs. (4.37),
    (4.45): the theta and phi components give, per degree n,
        b_n = (psi_n - i eta psi'_n) / (xi_n - i eta xi'_n),
        a_n = (psi'_n + i eta psi_n) / (xi'_n + i eta xi_n)     (argument x = k a).
    eta = 0 is the perfect conductor (a_n = psi'_n/xi'_n, b_n = psi_n/xi_n); eta = 1/m is the
    large-|m| limit of the coefficients in ``coefficients``."""
    if nmax is None:
        nmax = default_nmax(x)
    n = np.arange(1, nmax + 1)
    px, dpx = _psi(n, x), _dpsi(n, x)
    xx, dxx = _xi(n, x), _dxi(n, x)
    a = (dpx + 1j * eta * px) / (dxx + 1j * eta * xx)
    b = (px - 1j * eta * dpx) / (xx - 1j * eta * dxx)
    return a, b


def _scattering(eps_in, x, nmax, impedance):
    if impedance is None:
        a, b, _, _ = coefficients(eps_in, x, nmax)
        return a, b
    return ibc_coefficients(impedance, x, nmax)


def _angular(nmax, mu):
    """pi_n, tau_n (n = 1..nmax) at mu = cos(theta); shapes [nmax, P]."""
    P = mu.shape[0]
    pi = np.zeros((nmax + 1, P))
    tau = np.zeros((nmax + 1, P))
    pi[1] = 1.0
    tau[1] = mu
    for n in range(2, nmax + 1):
        pi[n] = (2 * n - 1) / (n - 1) * mu * pi[n - 1] - n / (n - 1) * pi[n - 2]
        tau[n] = n * mu * pi[n] - (n + 1) * pi[n - 1]
    return pi[1:], tau[1:]


def _vsh(nmax, rho, theta, phi, kind):
    """Spherical components (r, theta, phi) of M_o1n, M_e1n, N_o1n, N_e1n, shape [4, nmax, 3, P];
    kind 1 uses j_n, kind 3 uses h_n^(1)."""
    n = np.arange(1, nmax + 1)[:, None]
    if kind == 1:
        z = spherical_jn(n, rho[None, :])
        dz = z + rho[None, :] * spherical_jn(n, rho[None, :], derivative=True)   # [rho z_n]'
    else:
        z = _h1(n, rho[None, :])
        dz = z + rho[None, :] * _dh1(n, rho[None, :])
    pi, tau = _angular(nmax, np.cos(theta))
    st, cp, sp = np.sin(theta)[None, :], np.cos(phi)[None, :], np.sin(phi)[None, :]
    zr = z / rho[None, :]
    dzr = dz / rho[None, :]
    zero = np.zeros_like(z)
    Mo = np.stack([zero, cp * pi * z, -sp * tau * z], axis=1)
    Me = np.stack([zero, -sp * pi * z, -cp * tau * z], axis=1)
    No = np.stack([sp * n * (n + 1) * st * pi * zr, sp * tau * dzr, cp * pi * dzr], axis=1)
    Ne = np.stack([cp * n * (n + 1) * st * pi * zr, cp * tau * dzr, -sp * pi * dzr], axis=1)
    return np.stack([Mo, Me, No, Ne])


def _to_cartesian(Fs, theta, phi):
    """Fs [..., 3(r,theta,phi), P] -> [..., P, 3(x,y,z)]"""
    st, ct, sp, cp = np.sin(theta), np.cos(theta), np.sin(phi), np.cos(phi)
    er = np.stack([st * cp, st * sp, ct], -1)
    et = np.stack([ct * cp, ct * sp, -st], -1)
    ep = np.stack([-sp, cp, np.zeros_like(sp)], -1)
    Fr, Ft, Fp = Fs[..., 0, :], Fs[..., 1, :], Fs[..., 2, :]
    return Fr[..., None] * er + Ft[..., None] * et + Fp[..., None] * ep


def _spherical(points):
    r = np.linalg.norm(points, axis=1)
    theta = np.arccos(np.clip(points[:, 2] / r, -1.0, 1.0))
    phi = np.arctan2(points[:, 1], points[:, 0])
    return r, theta, phi


def fields(points, k, a, eps_in, region="outside", nmax=None, impedance=None):
    """Electric field E and curl E at ``points`` [P,3] (must lie in ``region``: 'outside' gives the
    total exterior field E_inc + E_sca, 'inside' the internal field).  Returns (E, curlE),
    each [P,3] complex.  With ``impedance`` = eta the sphere obeys Eq. (2.24) with Z = eta
    times the background impedance (``eps_in`` unused; 'outside' only)."""
    x = k * a
    if nmax is None:
        nmax = default_nmax(x) + 4
    if impedance is not None:
        assert region == "outside"
        an, bn = ibc_coefficients(impedance, x, nmax)
    else:
        an, bn, cn, dn = coefficients(eps_in, x, nmax)
    n = np.arange(1, nmax + 1)
    En = (1j ** n) * (2 * n + 1) / (n * (n + 1))
    r, theta, phi = _spherical(np.asarray(points, dtype=np.float64))
    if region == "outside":
        kk = k
        V = _vsh(nmax, kk * r, theta, phi, 3)
        Mo, Me, No, Ne = V
        cE = En[:, None, None]
        Es = (cE * (1j * an[:, None, None] * Ne - bn[:, None, None] * Mo)).sum(0)
        Cs = (cE * (1j * an[:, None, None] * kk * Me - bn[:, None, None] * kk * No)).sum(0)
        E = _to_cartesian(Es, theta, phi)
        C = _to_cartesian(Cs, theta, phi)
        ph = np.exp(1j * k * points[:, 2])
        E[:, 0] += ph
        C[:, 1] += 1j * k * ph
        return E, C
    m = np.sqrt(complex(eps_in))
    if m.imag < 0:
        m = -m
    kk = m * k
    V = _vsh(nmax, kk * r, theta, phi, 1)
    Mo, Me, No, Ne = V
    cE = En[:, None, None]
    Ei = (cE * (cn[:, None, None] * Mo - 1j * dn[:, None, None] * Ne)).sum(0)
    Ci = (cE * (cn[:, None, None] * kk * No - 1j * dn[:, None, None] * kk * Me)).sum(0)
    return _to_cartesian(Ei, theta, phi), _to_cartesian(Ci, theta, phi)


def surface_unknowns(points, normals, k, a, eps_in, nmax=None, impedance=None):
    """The BEM unknowns of Eq. (2.12) from the Mie series at surface points: Phi = E_0 (total
    exterior field) and Psi = n x curl E_0 with the scatterer's outward normal n.  [P,6]."""
    E, C = fields(points, k, a, eps_in, "outside", nmax, impedance)
    Psi = np.cross(normals, C)
    return np.concatenate([E, Psi], axis=1)


def cross_sections(k, a, eps_in, nmax=None, impedance=None):
    """(C_ext, C_sca, C_abs) from the Mie coefficients (Bohren & Huffman Eqs. 4.61-4.62); with
    ``impedance`` = eta those of the impedance sphere (``ibc_coefficients``)."""
    x = k * a
    if nmax is None:
        nmax = default_nmax(x)
    an, bn = _scattering(eps_in, x, nmax, impedance)
    n = np.arange(1, len(an) + 1)
    cext = 2 * np.pi / k ** 2 * np.sum((2 * n + 1) * (an + bn).real)
    csca = 2 * np.pi / k ** 2 * np.sum((2 * n + 1) * (abs(an) ** 2 + abs(bn) ** 2))
    return cext, csca, cext - csca


def radiation_pressure(k, a, eps_in, nmax=None):
    """Radiation-pressure cross section C_pr = C_ext - <cos theta> C_sca of the sphere, with the
    asymmetry term from the Mie coefficients (Bohren & Huffman Eq. 4.74):
    <cos theta> C_sca = (4 pi / k^2) sum_n [ n (n+2)/(n+1) Re(a_n a*_{n+1} + b_n b*_{n+1})
                                             + (2n+1)/(n (n+1)) Re(a_n b*_n) ].
    The time-averaged force on the sphere in a unit plane wave in vacuum is C_pr / 2 along d."""
    x = k * a
    an, bn, _, _ = coefficients(eps_in, x, nmax)
    n = np.arange(1, len(an) + 1)
    cext, csca, _ = cross_sections(k, a, eps_in, nmax)
    t1 = n[:-1] * (n[:-1] + 2) / (n[:-1] + 1) * (an[:-1] * np.conj(an[1:]) + bn[:-1] * np.conj(bn[1:])).real
    t2 = (2 * n + 1) / (n * (n + 1)) * (an * np.conj(bn)).real
    gcsca = 4 * np.pi / k ** 2 * (np.sum(t1) + np.sum(t2))
    return cext - gcsca


def asymmetry_by_quadrature(k, a, eps_in, n_theta=400, nmax=None):
    """<cos theta> C_sca by quadrature of the amplitude functions S1, S2 (Bohren & Huffman
    Eqs. 4.74 in integral form): (pi / k^2) int (|S1|^2 + |S2|^2) cos theta sin theta dtheta, an
    evaluation independent of the closed form in radiation_pressure."""
    x = k * a
    an, bn, _, _ = coefficients(eps_in, x, nmax)
    nm = len(an)
    n = np.arange(1, nm + 1)
    mu, w = np.polynomial.legendre.leggauss(n_theta)
    pi_n, tau_n = _angular(nm, mu)                     # [nmax, n_theta]
    f = ((2 * n + 1) / (n * (n + 1)))[:, None]
    S1 = np.sum(f * (an[:, None] * pi_n + bn[:, None] * tau_n), axis=0)
    S2 = np.sum(f * (an[:, None] * tau_n + bn[:, None] * pi_n), axis=0)
    return np.pi / k ** 2 * float(np.sum(w * (abs(S1) ** 2 + abs(S2) ** 2) * mu))

