"""Pins of the oracle's magnetic field and of the optical-force formulas (CPU).

- H = curl E / (i k0 mu_0) from the curl of the representation formula must equal the central
  finite-difference curl of the oracle's electric near field.
- The Mie asymmetry term of the radiation pressure in closed form (Bohren & Huffman 4.74) must
  equal its quadrature from the amplitude functions S1, S2.
- The Maxwell-stress force on a sphere around the scatterer (near fields) and the far-zone
  momentum balance (C_ext d - int |F|^2 u) / 2 are independent evaluations of the same force;
  for the solved sphere they must agree, and approach the Mie radiation pressure C_pr / 2.
"""
import numpy as np
import pytest

import fmbem_inputs as fi
import oracle
from oracle import mie


def _sphere_quadrature(n_theta, n_phi):
    mu, wmu = np.polynomial.legendre.leggauss(n_theta)
    ph = 2 * np.pi * np.arange(n_phi) / n_phi
    MU, PH = np.meshgrid(mu, ph, indexing="ij")
    ST = np.sqrt(1 - MU ** 2)
    nq = np.stack([ST * np.cos(PH), ST * np.sin(PH), MU], -1).reshape(-1, 3)
    wq = (wmu[:, None] * np.full(n_phi, 2 * np.pi / n_phi)[None, :]).ravel()
    return nq, wq


def force_stress(o, x, d, e, center, radius, n_theta=24, n_phi=48):
    nq, wq = _sphere_quadrature(n_theta, n_phi)
    pts = np.asarray(center)[None, :] + radius * nq
    E = o.near_field(x, pts, d, e)
    H = o.near_field_h(x, pts, d, e)
    en = np.sum(np.conj(E) * nq, 1)
    hn = np.sum(np.conj(H) * nq, 1)
    u = np.sum(abs(E) ** 2 + abs(H) ** 2, 1)
    tn = 0.5 * np.real(E * en[:, None] + H * hn[:, None] - 0.5 * u[:, None] * nq)
    return np.sum((wq * radius ** 2)[:, None] * tn, 0)


def force_farfield(o, x, d, e, n_theta=24, n_phi=48):
    k = o.k[0].real
    rq, wq = _sphere_quadrature(n_theta, n_phi)
    F = o.far_field(x, np.concatenate([np.atleast_2d(d), rq]))
    cext = 4 * np.pi / k * np.imag(np.vdot(e, F[0]))
    return 0.5 * (cext * np.asarray(d) - np.sum((wq * np.sum(abs(F[1:]) ** 2, 1))[:, None] * rq, 0))


def test_magnetic_field_is_the_curl_of_the_electric_field():
    V, F, D = fi.icosphere(2)
    o = oracle.Oracle(V, F, D, [1.0, -4 + 0.3j], [1.0, 1.0], 1.3)
    x = fi.random_complex((o.N, 6), seed=3)
    d = np.array([0.3, -0.2, 0.9])
    d /= np.linalg.norm(d)
    e = np.cross(d, [1.0, 0, 0]).astype(np.complex128)
    e /= np.linalg.norm(e)
    pts = np.array([[1.6, 0.2, -0.3], [0.1, -2.2, 0.7], [-1.0, 1.0, 1.5]])
    H = o.near_field_h(x, pts, d, e)
    h = 1e-4
    for p, Hp in zip(pts, H):
        J = np.zeros((3, 3), dtype=np.complex128)  # J[j][k] = d E_k / d r_j
        for j in range(3):
            dp = np.zeros(3)
            dp[j] = h
            J[j] = (o.near_field(x, p + dp, d, e)[0] - o.near_field(x, p - dp, d, e)[0]) / (2 * h)
        curl = np.array([J[1, 2] - J[2, 1], J[2, 0] - J[0, 2], J[0, 1] - J[1, 0]])
        np.testing.assert_allclose(Hp * (1j * o.k0 * 1.0), curl, rtol=1e-6, atol=1e-8 * abs(curl).max())


@pytest.mark.parametrize("eps", [2.25, -8.5 + 0.3j, 1.77])
@pytest.mark.parametrize("k", [0.5, 1.0, 3.0])
def test_mie_asymmetry_closed_form_matches_quadrature(eps, k):
    cext, csca, _ = mie.cross_sections(k, 1.0, eps)
    g_closed = cext - mie.radiation_pressure(k, 1.0, eps)
    assert abs(g_closed - mie.asymmetry_by_quadrature(k, 1.0, eps)) < 1e-10 * max(abs(g_closed), 1e-3)


def test_stress_tensor_of_exact_mie_fields_is_the_radiation_pressure():
    """The stress-tensor integral of the exact Mie fields over a sphere of radius 2a equals the
    radiation pressure C_pr / 2 along d (pins the stress formula, its units, and C_pr)."""
    k0, eps, R = 1.0, 2.25, 2.0
    nq, wq = _sphere_quadrature(24, 48)
    E, C = mie.fields(R * nq, k0, 1.0, eps, "outside")
    H = C / (1j * k0)
    en, hn = np.sum(np.conj(E) * nq, 1), np.sum(np.conj(H) * nq, 1)
    u = np.sum(abs(E) ** 2 + abs(H) ** 2, 1)
    Fz = np.sum((wq * R ** 2)[:, None] * 0.5 * np.real(E * en[:, None] + H * hn[:, None] - 0.5 * u[:, None] * nq), 0)
    assert abs(Fz[2] - mie.radiation_pressure(k0, 1.0, eps) / 2) < 1e-8
    assert np.linalg.norm(Fz[:2]) < 1e-10


def test_forces_of_the_representation_formula_converge_to_mie():
    """With the exact Mie surface data as the unknowns, the fields of the representation formula
    (E and H = curl E / (i k0)) give a stress-tensor force equal to the far-zone momentum balance
    (two independent evaluations), converging to C_pr / 2 as the mesh is refined."""
    k0, eps = 1.0, 2.25
    cpr2 = mie.radiation_pressure(k0, 1.0, eps) / 2
    d = np.array([0.0, 0.0, 1.0])
    e = np.array([1.0, 0.0, 0.0], dtype=np.complex128)
    errs = []
    for sub in (2, 3):
        V, F, D = fi.icosphere(sub)
        o = oracle.Oracle(V, F, D, [1.0, eps], [1.0, 1.0], k0)
        xm = mie.surface_unknowns(o.s, o.n, k0, 1.0, eps)
        Fs = force_stress(o, xm, d, e, np.zeros(3), 2.0)
        Ff = force_farfield(o, xm, d, e)
        assert np.linalg.norm(Fs - Ff) < 1e-5 * np.linalg.norm(Ff)
        errs.append(abs(Fs[2] - cpr2) / cpr2)
    print("relative errors", errs)
    assert errs[1] < 0.5 * errs[0] and errs[1] < 0.01
