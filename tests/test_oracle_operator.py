"""Pins for the oracle's dense Nystrom operator, preconditioner and GMRES (Eqs. 2.9-2.13, 3.1-3.2).

None of these re-types the oracle's formulas.  They check what the mathematics fixes:
  * Exact Maxwell fields satisfy the boundary integral equations (2.5), so applying the
    discrete operator to the exact surface values leaves a residual that vanishes under mesh
    refinement (first order for the one-point rule): the incident field in the transparent
    limit (both row groups), a field radiating from inside the scatterer (background rows, no
    incident field), and a plane wave of the interior wavenumber (scatterer rows, with the
    boundary conditions (2.6)-(2.7) giving Phi and Psi).
  * The solved surface field, the near field on a circle of radius 2a (the paper's Fig. 4
    check) and the cross sections converge to the Mie series.
  * Energy conservation (optical theorem), transversality of the far field, reciprocity.
  * GMRES reproduces a dense direct solve; the preconditioner lowers the iteration count."""
import numpy as np
import pytest

import fmbem_inputs as fi
import oracle
from oracle import mie


def _residual_rows(o, x, b=None):
    y = o.matvec(x)
    if b is not None:
        y = y - b
    return y


def _rate(errs):
    return [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]


def test_wavenumber_branch():
    V, F, D = fi.icosphere(1)
    o = oracle.Oracle(V, F, D, [1.0, -8.5 + 0.3j], [1.0, 1.0], 0.5)
    k = o.k[1]
    assert k.imag > 0 and abs(k * k - 0.25 * (-8.5 + 0.3j)) < 1e-14
    o = oracle.Oracle(V, F, D, [1.0, -10 + 0.4j], [1.0, 1.0], 1.5)
    assert o.k[1].imag > 0 and abs(o.k[1] - (0.0949 + 4.7444j)) < 1e-3


@pytest.mark.parametrize("mode,subs", [("vertex", (2, 3, 4)), ("centroid", (1, 2, 3))])
def test_transparent_limit_residual_converges(mode, subs):
    errs = []
    for sub in subs:
        V, F, D = fi.icosphere(sub)
        o = oracle.Oracle(V, F, D, [1.0, 1.0], [1.0, 1.0], 1.0, mode=mode)
        d = np.array([0.3, -0.2, 0.9])
        d /= np.linalg.norm(d)
        e = np.cross(d, [1.0, 0, 0])
        e /= np.linalg.norm(e)
        ph = np.exp(1j * o.s @ d)
        E = e[None, :] * ph[:, None]
        C = 1j * np.cross(d, e)[None, :] * ph[:, None]
        x = np.concatenate([E, np.cross(o.n, C)], 1)
        b = o.plane_wave_rhs(d, e)[0]
        r = _residual_rows(o, x, b)
        errs.append(np.linalg.norm(r) / np.linalg.norm(b))
    assert all(q > 1.3 for q in _rate(errs)), errs
    assert errs[-1] < 0.035


def _dipole_field(points, k, c, center):
    """E = curl(c g), g = exp(ikr)/r around ``center``: an exact radiating Maxwell field."""
    r = points - center
    R = np.linalg.norm(r, axis=1)
    u = r / R[:, None]
    g = np.exp(1j * k * R) / R
    g1 = (1j * k - 1 / R) * g
    g2 = ((1j * k - 1 / R) ** 2 + 1 / R ** 2) * g
    E = g1[:, None] * np.cross(u, c[None, :])
    cu = u @ c
    # curl E = (c.grad) grad g + k^2 g c
    C = g2[:, None] * cu[:, None] * u + (g1 / R)[:, None] * (c[None, :] - cu[:, None] * u) + (k * k * g)[:, None] * c
    return E, C


def test_background_rows_vanish_for_radiating_field():
    errs = []
    for sub in (2, 3, 4):
        V, F, D = fi.icosphere(sub)
        o = oracle.Oracle(V, F, D, [1.0, 2.25], [1.0, 1.0], 1.3)
        E, C = _dipole_field(o.s, 1.3, np.array([0.2, -0.7, 0.5]), np.array([0.1, 0.2, -0.15]))
        x = np.concatenate([E, np.cross(o.n, C)], 1)
        y = o.matvec(x)
        errs.append(np.linalg.norm(y[:, :3]) / np.linalg.norm(E))
    assert all(q > 1.5 for q in _rate(errs)), errs
    assert errs[-1] < 0.03


@pytest.mark.parametrize("eps,mu,k0", [(2.25, 1.0, 1.0), (-8.5 + 0.3j, 1.0, 0.5), (2.0 + 0.1j, 1.4, 0.8)])
def test_scatterer_rows_vanish_for_interior_field(eps, mu, k0):
    errs = []
    for sub in (2, 3, 4):
        V, F, D = fi.icosphere(sub)
        o = oracle.Oracle(V, F, D, [1.0, eps], [1.0, mu], k0)
        kj = o.k[1]
        d = np.array([0.4, 0.5, -0.7])
        d /= np.linalg.norm(d)
        e = np.cross(d, [0, 0, 1.0])
        e /= np.linalg.norm(e)
        ph = np.exp(1j * kj * (o.s @ d))
        Ej = e[None, :] * ph[:, None]
        Cj = 1j * kj * np.cross(d, e)[None, :] * ph[:, None]
        n = o.n
        # boundary conditions (2.6)-(2.7): E_j = T E_0, n x curl E_j = gamma n x curl E_0
        t = (1.0 - eps) / eps
        Ej_n = np.sum(Ej * n, 1)
        E0 = Ej - (t / (1 + t)) * Ej_n[:, None] * n
        Psi = np.cross(n, Cj) / (mu / 1.0)
        y = o.matvec(np.concatenate([E0, Psi], 1))
        errs.append(np.linalg.norm(y[:, 3:]) / np.linalg.norm(Ej))
    assert all(q > 1.5 for q in _rate(errs)), errs
    assert errs[-1] < 0.03


@pytest.fixture(scope="module")
def mie_study():
    th = np.linspace(0, 2 * np.pi, 73)[:-1]
    pts = np.concatenate([np.stack([2 * np.sin(th), 0 * th, 2 * np.cos(th)], 1),
                          np.stack([0 * th, 2 * np.sin(th), 2 * np.cos(th)], 1)])
    Em, _ = mie.fields(pts, 1.0, 1.0, 2.25, "outside")
    out = []
    for sub in (2, 3, 4):
        V, F, D = fi.icosphere(sub)
        o = oracle.Oracle(V, F, D, [1.0, 2.25], [1.0, 1.0], 1.0)
        b = o.plane_wave_rhs([0, 0, 1.0], [1.0, 0, 0])
        x, its, res, conv = o.gmres(b, tol=1e-10)
        assert conv[0] and res[0] <= 1e-10
        xm = mie.surface_unknowns(o.s, o.n, 1.0, 1.0, 2.25)
        ePhi = np.linalg.norm(x[0, :, :3] - xm[:, :3]) / np.linalg.norm(xm[:, :3])
        Enf = o.near_field(x[0], pts, [0, 0, 1.0], [1.0, 0, 0])
        eNF = np.linalg.norm(Enf - Em) / np.linalg.norm(Em)
        cs = o.cross_sections(x[0], [0, 0, 1.0], [1.0, 0, 0])
        rh = np.random.default_rng(0).normal(size=(50, 3))
        rh /= np.linalg.norm(rh, axis=1, keepdims=True)
        Ff = o.far_field(x[0], rh)
        trans = np.linalg.norm(np.sum(Ff * rh, 1)) / np.linalg.norm(Ff)
        out.append(dict(ePhi=ePhi, eNF=eNF, cs=cs, trans=trans))
    return out


def test_mie_surface_field_converges(mie_study):
    e = [s["ePhi"] for s in mie_study]
    assert all(q > 1.6 for q in _rate(e)), e
    assert e[-1] < 0.025


def test_mie_near_field_converges(mie_study):
    """Fig. 4 of the paper: near field on circles of radius 2a in the xoz and yoz planes."""
    e = [s["eNF"] for s in mie_study]
    assert all(q > 1.8 for q in _rate(e)), e
    assert e[-1] < 0.01


def test_cross_sections_and_optical_theorem(mie_study):
    cext_m, csca_m, _ = mie.cross_sections(1.0, 1.0, 2.25)
    dsca = [abs(s["cs"][1] - csca_m) / csca_m for s in mie_study]
    cons = [abs(s["cs"][0] - s["cs"][1] - s["cs"][2]) / s["cs"][0] for s in mie_study]
    cabs = [abs(s["cs"][2]) / s["cs"][0] for s in mie_study]
    assert dsca[-1] < 0.03
    assert all(q > 1.5 for q in _rate(cons)) and cons[-1] < 0.005, cons
    assert all(q > 1.5 for q in _rate(cabs)), cabs           # lossless sphere: C_abs -> 0


def test_far_field_transverse(mie_study):
    t = [s["trans"] for s in mie_study]
    assert all(q > 1.5 for q in _rate(t)), t


def test_lossy_sphere_absorbs_and_converges():
    """Plasmonic sphere (eps = -8.5+0.3i, k0 a = 0.5): positive absorption, energy balance, and
    first-order convergence of the near field and of C_sca towards the Mie series."""
    eps, k0 = -8.5 + 0.3j, 0.5
    th = np.linspace(0, 2 * np.pi, 37)[:-1]
    pts = np.stack([2 * np.sin(th), 0 * th, 2 * np.cos(th)], 1)
    Em, _ = mie.fields(pts, k0, 1.0, eps, "outside")
    mext, msca, mabs = mie.cross_sections(k0, 1.0, eps)
    enf, esca, cons = [], [], []
    for sub in (2, 3):
        V, F, D = fi.icosphere(sub)
        o = oracle.Oracle(V, F, D, [1.0, eps], [1.0, 1.0], k0)
        b = o.plane_wave_rhs([0, 0, 1.0], [1.0, 0, 0])
        x, its, res, conv = o.gmres(b, tol=1e-9)
        assert conv[0]
        cext, csca, cabs = o.cross_sections(x[0], [0, 0, 1.0], [1.0, 0, 0])
        assert cabs > 0 and csca > 0
        cons.append(abs(cext - csca - cabs) / cext)
        E = o.near_field(x[0], pts, [0, 0, 1.0], [1.0, 0, 0])
        enf.append(np.linalg.norm(E - Em) / np.linalg.norm(Em))
        esca.append(abs(csca - msca) / msca)
    assert enf[0] / enf[1] > 1.6 and esca[0] / esca[1] > 1.4, (enf, esca)
    assert cons[1] < cons[0] and cons[1] < 0.03, cons


def test_reciprocity():
    errs = []
    di = np.array([0.2, 0.3, 0.93]); di /= np.linalg.norm(di)
    ds = np.array([-0.6, 0.5, 0.2]); ds /= np.linalg.norm(ds)
    ei = np.cross(di, [1.0, 0, 0]); ei /= np.linalg.norm(ei)
    es = np.cross(ds, [0, 1.0, 0]); es /= np.linalg.norm(es)
    for sub in (2, 3):
        V, F, D = fi.spheroid(1.0, 1.6, sub)
        o = oracle.Oracle(V, F, D, [1.0, 2.0 + 0.2j], [1.0, 1.0], 1.2)
        b = np.concatenate([o.plane_wave_rhs(di, ei), o.plane_wave_rhs(-ds, es)])
        x, its, res, conv = o.gmres(b, tol=1e-10)
        A = es @ o.far_field(x[0], ds)[0]
        B = ei @ o.far_field(x[1], -di)[0]
        errs.append(abs(A - B) / abs(A))
    assert errs[-1] < 0.02 and errs[1] < errs[0], errs


def test_gmres_matches_dense_solve():
    V, F, D = fi.icosphere(1)
    o = oracle.Oracle(V, F, D, [1.0, -3 + 0.5j], [1.0, 1.2], 1.1)
    n6 = 6 * o.N
    Id = np.eye(n6, dtype=np.complex128).reshape(n6, o.N, 6)
    A = o.matvec(Id).reshape(n6, n6).T
    b = o.plane_wave_rhs([0, 0.6, 0.8], [1.0, 0, 0])
    xd = np.linalg.solve(A, b.reshape(-1))
    for pre in (True, False):
        x, its, res, conv = o.gmres(b, tol=1e-12, restart=30, precond=pre)
        assert conv[0]
        assert np.linalg.norm(x.reshape(-1) - xd) < 1e-9 * np.linalg.norm(xd)
    # the preconditioner blocks are the diagonal 6x6 blocks of A (A_self, Eq. 3.2)
    M = o.precond_blocks()
    for a in (0, 5, 17):
        np.testing.assert_allclose(A[6 * a:6 * a + 6, 6 * a:6 * a + 6], M[a], atol=1e-13)
    z = o.precond_apply(b)
    np.testing.assert_allclose(np.einsum("nij,nj->ni", M, z[0]), b[0], atol=1e-12)


def test_preconditioner_reduces_iterations():
    """Fig. 3 of the paper: eps = 1.33^2, ka = 1.67 inside the sphere."""
    V, F, D = fi.icosphere(3)
    o = oracle.Oracle(V, F, D, [1.0, 1.33 ** 2], [1.0, 1.0], 1.67 / 1.33)
    b = o.plane_wave_rhs([0, 0, 1.0], [1.0, 0, 0])
    _, it_p, _, cp = o.gmres(b, tol=1e-6, restart=50, max_iter=400, precond=True)
    _, it_n, _, cn = o.gmres(b, tol=1e-6, restart=50, max_iter=400, precond=False)
    assert cp[0]
    assert it_p[0] < it_n[0]


def test_rows_subset_and_multi_rhs_consistent():
    V, F, D = fi.icosphere(2)
    o = oracle.Oracle(V, F, D, [1.0, -8.5 + 0.3j], [1.0, 1.0], 0.5)
    x = fi.random_complex((3, o.N, 6), seed=1)
    y = o.matvec(x)
    for r in range(3):
        np.testing.assert_allclose(o.matvec(x[r]), y[r], rtol=0, atol=1e-12)
    rows = fi.sample_rows(o.N, 20, seed=2)
    np.testing.assert_allclose(o.matvec_rows(x, rows), y[:, rows], rtol=0, atol=1e-12)


def test_two_scatterers_rows_see_their_own_nodes():
    """With two disjoint spheres, a plane wave of sphere 1's interior wavenumber placed on
    sphere 1 satisfies sphere 1's rows whatever sphere 2 carries (its nodes are not sources of
    domain 1); the transparent limit of both converges like the single sphere."""
    m1 = fi.icosphere(3, 0.6, (-0.8, 0, 0), domain=1)
    m2 = fi.icosphere(2, 0.4, (0.7, 0.1, 0), domain=2)
    V, F, D = fi.merge_meshes(m1, m2)
    o = oracle.Oracle(V, F, D, [1.0, 2.25, -4 + 0.3j], [1.0, 1.0, 1.0], 1.0)
    on1 = o.dom == 1
    kj = o.k[1]
    d = np.array([0.0, 0.6, 0.8])
    e = np.array([1.0, 0, 0])
    ph = np.exp(1j * kj * (o.s @ d))
    Ej = e[None, :] * ph[:, None]
    Cj = 1j * kj * np.cross(d, e)[None, :] * ph[:, None]
    t = (1.0 - 2.25) / 2.25
    E0 = Ej - (t / (1 + t)) * np.sum(Ej * o.n, 1)[:, None] * o.n
    x = np.concatenate([E0, np.cross(o.n, Cj)], 1)
    x[~on1] = fi.random_complex((int((~on1).sum()), 6), seed=4)
    y = o.matvec(x)
    r1 = np.linalg.norm(y[on1, 3:]) / np.linalg.norm(Ej[on1])
    assert r1 < 0.03


@pytest.mark.parametrize("case_", ["sphere_vertex", "sphere_centroid", "two_scatterers"])
def test_transpose_bilinear_identity(case_):
    """<y, A x> = <A^T y, x> (bilinear, no conjugation) for random x, y: the transposed product is
    pinned to the forward operator, which the other pins tie to the paper and to Mie."""
    if case_ == "two_scatterers":
        mesh = fi.merge_meshes(fi.icosphere(2, 0.6, (-0.8, 0, 0), domain=1), fi.icosphere(2, 0.4, (0.7, 0.1, 0.05), domain=2))
        o = oracle.Oracle(*mesh, [1.0, 2.25, -4 + 0.3j], [1.0, 1.3, 1.0], 1.2)
    else:
        mode = "vertex" if case_ == "sphere_vertex" else "centroid"
        o = oracle.Oracle(*fi.icosphere(2), [1.0, -8.5 + 0.3j], [1.0, 1.0], 0.7, mode=mode)
    x = fi.random_complex((2, o.N, 6), seed=31)
    y = fi.random_complex((2, o.N, 6), seed=32)
    lhs = np.sum(y * o.matvec(x))
    rhs = np.sum(o.matvec_transpose(y) * x)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_transpose_matches_explicit_matrix():
    """On a 42-node mesh, A assembled column by column from the forward product, transposed with
    numpy, applied to a random vector, equals the oracle's transposed product; the rows variant
    returns the same entries."""
    o = oracle.Oracle(*fi.icosphere(1), [1.0, 2.25], [1.0, 1.3], 1.0)
    n = 6 * o.N
    A = np.empty((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1.0
        A[:, j] = o.matvec(e.reshape(o.N, 6)).reshape(n)
    x = fi.random_complex((o.N, 6), seed=33)
    yt = o.matvec_transpose(x).reshape(n)
    np.testing.assert_allclose(yt, A.T @ x.reshape(n), rtol=0, atol=1e-13 * np.abs(yt).max())
    rows = np.array([0, 7, 41])
    np.testing.assert_array_equal(o.matvec_transpose_rows(x, rows), o.matvec_transpose(x)[rows])
