"""Pins for the oracle's near-singular correction (the option near_singular_radius; off, i.e. the
paper's one-point rule of Eq. (2.8) for every pair, at radius 0).

With a radius rho > 0, a source node beta within R < rho sqrt(w_beta) of the target contributes
the integral of the Eq. (2.12) kernel over its patch (density and normal held constant) instead
of the one-point term; each flat piece of the patch is split into 4^L triangles integrated with
the centroid rule.  None of these tests re-types that arithmetic:
  * the patch pieces cover exactly the node weight (a far-away point sees w / (4 pi R));
  * the subdivision rule converges, at second order in the piece size, to an adaptive
    quadrature (scipy) of the same integrals over pieces built here from the patch's
    definition, for complex wavenumbers, vertex and centroid nodes;
  * in the operator, only rows with near-singular sources change, and a single Psi entry moves
    them by exactly the monopole integrals (sign, domain wavenumber, gamma_j of Eq. 2.13);
  * the corrected operator still satisfies the boundary equations for exact Maxwell fields to
    first order, and for centroid nodes (whose neighbours sit closest to the patches) the
    correction lowers that consistency residual at every mesh size;
  * its transpose satisfies the bilinear identity with the forward product."""
import numpy as np
import pytest

import fmbem_inputs as fi
import oracle

integrate = pytest.importorskip("scipy.integrate")

KC = 1.5 * np.sqrt(-10 + 0.4j)  # interior wavenumber of the silver-like torus (Im k > 0)


def _pieces(V, F, b, mode):
    """The flat pieces of node b's patch, from the definition: the triangle itself (centroid
    nodes) or, in every triangle incident to vertex b, the two halves (b, mid, centroid) of its
    barycentric dual-cell quadrilateral (vertex nodes)."""
    if mode == "centroid":
        return [V[F[b]]]
    out = []
    for t in np.nonzero((F == b).any(1))[0]:
        tri = list(F[t])
        a = tri.index(b)
        A, B, C = V[tri[a]], V[tri[(a + 1) % 3]], V[tri[(a + 2) % 3]]
        G = (A + B + C) / 3
        out += [np.array([A, (A + B) / 2, G]), np.array([A, G, (A + C) / 2])]
    return out


def _adaptive(pieces, pt, k):
    """int g and int grad' g over the pieces by adaptive 2-D quadrature (scipy dblquad)."""
    vals = np.zeros(8)
    for P in pieces:
        e1, e2 = P[1] - P[0], P[2] - P[0]
        jac = np.linalg.norm(np.cross(e1, e2))

        def f(v, u, i):
            r = P[0] + u * e1 + v * e2 - pt
            R = np.linalg.norm(r)
            g = np.exp(1j * k * R) / (4 * np.pi * R)
            q = g if i < 2 else g * (1j * k - 1 / R) / R * r[(i - 2) // 2]
            return jac * (q.real if i % 2 == 0 else q.imag)
        for i in range(8):
            vals[i] += integrate.dblquad(f, 0, 1, 0, lambda u: 1 - u, args=(i,), epsabs=1e-13, epsrel=1e-11)[0]
    return complex(vals[0], vals[1]), vals[2::2] + 1j * vals[3::2]


@pytest.mark.parametrize("mode", ["vertex", "centroid"])
def test_patch_pieces_cover_the_node_weight(mode):
    V, F, D = fi.spheroid(1.0, 2.0, 2)
    o = oracle.Oracle(V, F, D, [1.0, 2.25], [1.0, 1.0], 1.0, mode=mode)
    for b in range(0, o.N, 7):
        far = o.s[b] + 1e7 * o.n[b]
        for L in (0, 2, 4):
            G, _ = o.patch_integral(b, far, 0.0, levels=L)
            assert abs(G * 4 * np.pi * 1e7 / o.w[b] - 1) < 1e-6, (b, L)


@pytest.mark.parametrize("mode", ["vertex", "centroid"])
def test_patch_integral_converges_to_adaptive_quadrature(mode):
    V, F, D = fi.icosphere(1)
    o = oracle.Oracle(V, F, D, [1.0, 2.25], [1.0, 1.0], 1.0, mode=mode)
    b = 5
    d = np.linalg.norm(o.s - o.s[b], axis=1)
    d[b] = np.inf
    a = int(np.argmin(d))  # the nearest node: the most singular neighbour pair
    for k in (1.0, KC):
        Gr, Ar = _adaptive(_pieces(V, F, b, mode), o.s[a], k)
        scale = abs(Gr) + np.linalg.norm(Ar)
        errs = []
        for L in (2, 3, 4, 5):
            G, A = o.patch_integral(b, o.s[a], k, levels=L)
            errs.append((abs(G - Gr) + np.linalg.norm(A - Ar)) / scale)
        ratios = [errs[i] / errs[i + 1] for i in range(3)]
        assert errs[1] < 1e-2 and errs[-1] < 1e-3, (k, errs)
        assert all(3.0 < q < 5.5 for q in ratios), (k, errs, ratios)


def test_single_psi_entry_moves_rows_by_the_monopole_integrals():
    V, F, D = fi.icosphere(1)
    eps, mu, k0 = [1.0, -10 + 0.4j], [1.0, 1.7], 1.5
    rho = 1.5
    o0 = oracle.Oracle(V, F, D, eps, mu, k0)
    o1 = oracle.Oracle(V, F, D, eps, mu, k0, near_singular_radius=rho, near_singular_levels=4)
    b = 11
    x = np.zeros((o0.N, 6), dtype=np.complex128)
    x[b, 3] = 1.0  # Psi_x of node b
    dy = o1.matvec(x) - o0.matvec(x)
    R = np.linalg.norm(o0.s - o0.s[b], axis=1)
    near = (R < rho * np.sqrt(o0.w[b])) & (R > 0)
    assert near.sum() >= 3
    assert np.all(dy[~near] == 0)
    gam = mu[1] / mu[0]
    for a in np.nonzero(near)[0]:
        for side, k, fac in ((0, o0.k[0], -1.0), (1, o0.k[1], gam)):
            Gr, _ = _adaptive(_pieces(V, F, b, "vertex"), o0.s[a], k)
            g1 = o0.w[b] * np.exp(1j * k * R[a]) / (4 * np.pi * R[a])
            want = fac * (Gr - g1)
            got = dy[a, 3 * side]
            assert abs(got - want) < 2e-3 * abs(want), (a, side, got, want)
            assert np.all(np.abs(dy[a, 3 * side + 1:3 * side + 3]) == 0)


@pytest.mark.parametrize("mode,subs", [("vertex", (2, 3, 4)), ("centroid", (1, 2, 3))])
def test_corrected_operator_keeps_exact_fields_consistent(mode, subs):
    """Transparent limit (eps_j = eps_0): E = E_inc and Psi = n x curl E_inc solve the equations
    exactly, so the discrete residual must vanish at first order with the correction too."""
    res = {0.0: [], 2.5: []}
    for sub in subs:
        V, F, D = fi.icosphere(sub)
        for rho in res:
            o = oracle.Oracle(V, F, D, [1.0, 1.0], [1.0, 1.0], 1.0, mode=mode, near_singular_radius=rho)
            d = np.array([0.3, -0.2, 0.9])
            d /= np.linalg.norm(d)
            e = np.cross(d, [1.0, 0, 0])
            e /= np.linalg.norm(e)
            ph = np.exp(1j * o.s @ d)
            x = np.concatenate([e[None, :] * ph[:, None], np.cross(o.n, 1j * np.cross(d, e)[None, :] * ph[:, None])], 1)
            b = o.plane_wave_rhs(d, e)[0]
            res[rho].append(np.linalg.norm(o.matvec(x) - b) / np.linalg.norm(b))
    r = res[2.5]
    assert all(r[i] / r[i + 1] > 1.3 for i in range(len(r) - 1)), r
    if mode == "centroid":
        assert all(c < 0.8 * p for c, p in zip(res[2.5], res[0.0])), res


def test_corrected_transpose_bilinear_identity():
    V, F, D = fi.icosphere(2)
    o = oracle.Oracle(V, F, D, [1.0, -8.5 + 0.3j], [1.0, 1.3], 0.5, near_singular_radius=2.0)
    x = fi.random_complex((2, o.N, 6), seed=3)
    y = fi.random_complex((2, o.N, 6), seed=4)
    lhs = np.sum(y * o.matvec(x))
    rhs = np.sum(o.matvec_transpose(y) * x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("eps,mu,k0", [(2.0 + 0.1j, 1.4, 0.8), (-8.5 + 0.3j, 1.0, 0.5)])
def test_corrected_scatterer_rows_vanish_for_interior_field(eps, mu, k0):
    """A plane wave of the interior wavenumber with the boundary conditions (2.6)-(2.7) solves the
    scatterer equations: with centroid nodes and the correction, the residual of the scatterer
    rows vanishes at first order and stays below the one-point rule's (T_j, gamma_j and k_j all
    enter the corrected pairs)."""
    res = {0.0: [], 2.5: []}
    for sub in (1, 2, 3):
        V, F, D = fi.icosphere(sub)
        for rho in res:
            o = oracle.Oracle(V, F, D, [1.0, eps], [1.0, mu], k0, mode="centroid", near_singular_radius=rho)
            kj = o.k[1]
            d = np.array([0.4, 0.5, -0.7])
            d /= np.linalg.norm(d)
            e = np.cross(d, [0, 0, 1.0])
            e /= np.linalg.norm(e)
            ph = np.exp(1j * kj * (o.s @ d))
            Ej = e[None, :] * ph[:, None]
            Cj = 1j * kj * np.cross(d, e)[None, :] * ph[:, None]
            t = (1.0 - eps) / eps
            E0 = Ej - (t / (1 + t)) * np.sum(Ej * o.n, 1)[:, None] * o.n
            y = o.matvec(np.concatenate([E0, np.cross(o.n, Cj) / mu], 1))
            res[rho].append(np.linalg.norm(y[:, 3:]) / np.linalg.norm(Ej))
    r = res[2.5]
    assert all(r[i] / r[i + 1] > 1.6 for i in range(len(r) - 1)), r
    assert all(c < 0.8 * p for c, p in zip(res[2.5], res[0.0])), res
