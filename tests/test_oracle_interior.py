"""Pins for the oracle's fields inside the scatterers (representation formula of the scatterer
domains, Appendix A; the relation behind Eq. 2.5 at points inside Omega_j).

None of these re-types the oracle's formulas:
  * from the exact Mie surface data of a sphere, the interior E and H converge to the Mie
    internal field, and the same sum at exterior points (the null-field integral) vanishes;
  * from the exact surface data of an interior plane wave of k_j (with mu_j != 1 and two
    scatterers), the plane wave and its H = k_j d x e / (k0 mu_j) are reproduced;
  * H is the curl of E / (i k0 mu_j) by central differences;
  * the field of a solved system converges to the Mie internal field."""
import numpy as np
import pytest

import fmbem_inputs as fi
import oracle
from oracle import mie


def _rate(errs):
    return [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]


def _points(rng, n, r0, r1):
    P = rng.normal(size=(n, 3))
    rad = r0 + (r1 - r0) * rng.random((n, 1))
    return P * rad / np.linalg.norm(P, axis=1, keepdims=True)


@pytest.mark.parametrize("eps,k0", [(2.25, 1.0), (-8.5 + 0.3j, 0.5)])
def test_exact_mie_data_give_the_internal_field(eps, k0):
    rng = np.random.default_rng(0)
    P = _points(rng, 30, 0.0, 0.6)
    Q = _points(rng, 30, 1.6, 2.0)
    Em, Cm = mie.fields(P, k0, 1.0, eps, "inside")
    Hm = Cm / (1j * k0)
    eE, eH, null = [], [], []
    for sub in (2, 3, 4):
        V, F, D = fi.icosphere(sub)
        o = oracle.Oracle(V, F, D, [1.0, eps], [1.0, 1.0], k0)
        xm = mie.surface_unknowns(o.s, o.n, k0, 1.0, eps)
        E, H = o.interior_field(xm, P, 1, magnetic=True)
        eE.append(np.linalg.norm(E - Em) / np.linalg.norm(Em))
        eH.append(np.linalg.norm(H - Hm) / np.linalg.norm(Hm))
        null.append(np.linalg.norm(o.interior_field(xm, Q, 1)) / np.linalg.norm(Em))
    assert all(q > 3 for q in _rate(eE)) and eE[-1] < 2e-3, eE
    assert all(q > 3 for q in _rate(eH)) and eH[-1] < 2e-3, eH
    assert null[-1] < 1e-4, null


def test_interior_plane_wave_with_mu_and_two_scatterers():
    """Scatterer j carries the plane wave E_j = e exp(i k_j d.r) (k_j = k0 sqrt(eps_j mu_j)); its
    surface data follow from Eqs. (2.6)-(2.7): Phi = E_0 with T_j E_0 = E_j, Psi = n x curl E_j /
    gamma_j.  The other scatterer's data are zero."""
    m1 = fi.icosphere(3, 0.5, (-0.8, 0.0, 0.0), domain=1)
    m2 = fi.icosphere(3, 0.4, (0.7, 0.1, 0.0), domain=2)
    V, F, D = fi.merge_meshes(m1, m2)
    eps, mu, k0 = [1.0, 3.0 + 0.2j, -2.0 + 0.5j], [1.0, 1.7, 1.0], 1.2
    o = oracle.Oracle(V, F, D, eps, mu, k0)
    d = np.array([0.36, 0.48, 0.8])
    e = np.array([0.8, 0.0, -0.36], dtype=np.complex128)
    e -= d * np.dot(d, e)
    for j, ctr, rad in ((1, (-0.8, 0.0, 0.0), 0.5), (2, (0.7, 0.1, 0.0), 0.4)):
        kj = o.k[j]
        sel = o.dom == j
        Ej = e[None] * np.exp(1j * kj * (o.s @ d))[:, None]
        Cj = 1j * kj * np.cross(d, e)[None] * np.exp(1j * kj * (o.s @ d))[:, None]
        n = o.n
        x = np.zeros((o.N, 6), dtype=np.complex128)
        ratio = (eps[j] - eps[0]) / eps[0]
        x[sel, :3] = (Ej + ratio * n * np.sum(n * Ej, 1, keepdims=True))[sel]
        x[sel, 3:] = (np.cross(n, Cj) / (mu[j] / mu[0]))[sel]
        P = np.asarray(ctr) + _points(np.random.default_rng(j), 20, 0.0, 0.5 * rad)
        E, H = o.interior_field(x, P, j, magnetic=True)
        ph = np.exp(1j * kj * (P @ d))[:, None]
        Ee = e[None] * ph
        He = (kj / (k0 * mu[j])) * np.cross(d, e)[None] * ph
        assert np.linalg.norm(E - Ee) / np.linalg.norm(Ee) < 0.02
        assert np.linalg.norm(H - He) / np.linalg.norm(He) < 0.02


def test_h_is_the_curl_of_e():
    V, F, D = fi.icosphere(2)
    eps, mu, k0 = [1.0, 2.0 + 0.3j], [1.0, 1.4], 1.1
    o = oracle.Oracle(V, F, D, eps, mu, k0)
    rng = np.random.default_rng(5)
    x = rng.normal(size=(o.N, 6)) + 1j * rng.normal(size=(o.N, 6))
    P = _points(rng, 5, 0.1, 0.5)
    _, H = o.interior_field(x, P, 1, magnetic=True)
    h = 1e-5
    J = np.zeros((len(P), 3, 3), dtype=np.complex128)   # J[p, i, a] = dE_i / dr_a
    for a in range(3):
        dp = np.zeros(3)
        dp[a] = h
        J[:, :, a] = (o.interior_field(x, P + dp, 1) - o.interior_field(x, P - dp, 1)) / (2 * h)
    curl = np.stack([J[:, 2, 1] - J[:, 1, 2], J[:, 0, 2] - J[:, 2, 0], J[:, 1, 0] - J[:, 0, 1]], 1)
    np.testing.assert_allclose(H, curl / (1j * k0 * mu[1]), rtol=1e-6, atol=1e-8 * np.abs(H).max())


def test_solved_system_converges_to_the_internal_field():
    eps, k0 = 2.25, 1.0
    rng = np.random.default_rng(1)
    P = _points(rng, 30, 0.0, 0.6)
    Em, _ = mie.fields(P, k0, 1.0, eps, "inside")
    errs = []
    for sub in (2, 3, 4):
        V, F, D = fi.icosphere(sub)
        o = oracle.Oracle(V, F, D, [1.0, eps], [1.0, 1.0], k0)
        x, its, res, conv = o.gmres(o.plane_wave_rhs([0, 0, 1.0], [1.0, 0, 0]), tol=1e-10)
        errs.append(np.linalg.norm(o.interior_field(x[0], P, 1) - Em) / np.linalg.norm(Em))
    assert all(q > 1.6 for q in _rate(errs)), errs
    assert errs[-1] < 0.03, errs
