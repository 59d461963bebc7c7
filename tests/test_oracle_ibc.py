"""Pins for the oracle's impedance-boundary-condition variant (Section 2.3, Eqs. 2.24-2.25).

None of these re-types the oracle's formulas:
  * the Mie series of the impedance sphere (oracle/mie.py, derived from Eq. 2.24 and the vector
    spherical harmonics of Bohren & Huffman) satisfies n x E = Z n x (n x H) on the sphere with
    H from the curl of the series itself, and tends to the penetrable sphere's series as |m|
    grows with Z = 1/m (the regime in which the condition holds for a good conductor);
  * the Eq. (2.25) operator is the background equation of Eq. (2.12) with n0 x curl E_0 replaced
    through Eq. (2.24), which is how the paper obtains it;
  * the exact impedance-sphere fields leave a residual that vanishes at first order under mesh
    refinement, and the solved surface field, near field and cross sections converge to the series;
  * a passive surface (Re Z > 0) absorbs, and the absorbed power closes the energy balance."""
import numpy as np
import pytest

import fmbem_inputs as fi
import oracle
from oracle import mie


def _rate(errs):
    return [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]


@pytest.mark.parametrize("eta", [0.0, 0.3 - 0.2j, 0.00707 * (1 - 1j), 0.006 - 0.343j])
def test_mie_impedance_sphere_satisfies_eq_2_24(eta):
    rng = np.random.default_rng(1)
    k, a = 1.3, 1.0
    P = rng.normal(size=(40, 3))
    P *= a / np.linalg.norm(P, axis=1, keepdims=True)
    E, C = mie.fields(P, k, a, None, "outside", impedance=eta)
    H = C / (1j * k)
    n = P / a
    lhs = np.cross(n, E)
    rhs = eta * np.cross(n, np.cross(n, H))
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(E) < 1e-12


def test_mie_impedance_sphere_is_the_large_index_limit():
    d = []
    for eps in (1 + 1e2j, 1 + 1e3j, 1 + 1e4j):
        cp = np.array(mie.cross_sections(1.0, 1.0, eps))
        ci = np.array(mie.cross_sections(1.0, 1.0, None, impedance=1 / np.sqrt(eps)))
        d.append(np.max(np.abs(cp - ci) / np.abs(cp)))
    assert all(q > 5 for q in _rate(d)), d
    assert d[-1] < 3e-5


def test_operator_is_the_background_equation_with_eq_2_24():
    V, F, D = fi.icosphere(2)
    o = oracle.Oracle(V, F, D, [1.0, 1 + 1e4j], [1.0, 1.0], 1.0)
    rng = np.random.default_rng(2)
    E = rng.normal(size=(2, o.N, 3)) + 1j * rng.normal(size=(2, o.N, 3))
    y = o.ibc_matvec(E)
    y6 = o.matvec(o.ibc_unknowns(E))
    assert np.linalg.norm(y - y6[..., :3]) / np.linalg.norm(y) < 1e-13
    # Psi is tangential and scales with zeta = i k0 / Z
    P = o.ibc_psi(E)
    assert np.max(np.abs(np.sum(P * o.n[None], -1))) < 1e-12 * np.max(np.abs(P))
    assert abs(o.ibc_zeta()[1] - 1j / np.sqrt(1 / (1 + 1e4j))) < 1e-9


@pytest.fixture(scope="module")
def ibc_study():
    """Lossy impedance sphere, eta = 1/sqrt(2.25 + 1i), k0 a = 1, vertex nodes on icospheres 2-4."""
    eps, k0 = 2.25 + 1j, 1.0
    eta = 1 / np.sqrt(eps)
    th = np.linspace(0, 2 * np.pi, 37)[:-1]
    pts = np.concatenate([np.stack([2 * np.sin(th), 0 * th, 2 * np.cos(th)], 1),
                          np.stack([0 * th, 2 * np.sin(th), 2 * np.cos(th)], 1)])
    Em, _ = mie.fields(pts, k0, 1.0, None, "outside", impedance=eta)
    out = []
    for sub in (2, 3, 4):
        V, F, D = fi.icosphere(sub)
        o = oracle.Oracle(V, F, D, [1.0, eps], [1.0, 1.0], k0)
        b = o.plane_wave_rhs([0, 0, 1.0], [1.0, 0, 0])[:, :, :3]
        xm = mie.surface_unknowns(o.s, o.n, k0, 1.0, None, impedance=eta)
        res = np.linalg.norm(o.ibc_matvec(xm[:, :3]) - b[0]) / np.linalg.norm(b[0])
        x, rr = o.ibc_solve(b)
        assert rr[0] < 1e-9
        x6 = o.ibc_unknowns(x[0])
        ePhi = np.linalg.norm(x[0] - xm[:, :3]) / np.linalg.norm(xm[:, :3])
        eNF = np.linalg.norm(o.near_field(x6, pts, [0, 0, 1.0], [1.0, 0, 0]) - Em) / np.linalg.norm(Em)
        cs = o.cross_sections(x6, [0, 0, 1.0], [1.0, 0, 0])
        out.append(dict(res=res, ePhi=ePhi, eNF=eNF, cs=cs))
    return out, mie.cross_sections(k0, 1.0, None, impedance=eta)


def test_exact_fields_leave_a_first_order_residual(ibc_study):
    r = [s["res"] for s in ibc_study[0]]
    assert all(q > 1.8 for q in _rate(r)), r
    assert r[-1] < 0.06


def test_solution_converges_to_the_series(ibc_study):
    e = [s["ePhi"] for s in ibc_study[0]]
    nf = [s["eNF"] for s in ibc_study[0]]
    assert all(q > 1.6 for q in _rate(e)), e
    assert all(q > 1.6 for q in _rate(nf)), nf
    assert e[-1] < 0.3 and nf[-1] < 0.12


def test_cross_sections_and_absorption(ibc_study):
    study, (cext_m, csca_m, cabs_m) = ibc_study
    dext = [abs(s["cs"][0] - cext_m) / cext_m for s in study]
    assert all(q > 1.6 for q in _rate(dext)), dext
    assert dext[-1] < 0.15
    for s in study:
        cext, csca, cabs = s["cs"]
        assert cabs > 0
    bal = [abs(s["cs"][0] - s["cs"][1] - s["cs"][2]) / s["cs"][0] for s in study]
    assert bal[-1] < 0.02, bal
