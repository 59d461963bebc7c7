"""Pins for the oracle's self-patch integrals (Appendix B, Eqs. B.2-B.9).

The closed forms are checked against brute-force numerical quadrature in polar coordinates
about O (adaptive in the angle, with the radial integral done exactly), against the disk limit
(int dA/rho = 2 pi a for a disk of radius a about its centre) and against symmetry (a centrally
symmetric polygon has int r/r dA = CPV int r/r^3 dA = 0)."""
import numpy as np
import pytest
from scipy import integrate

import oracle


def _frame(normal):
    n = normal / np.linalg.norm(normal)
    a = np.array([1.0, 0, 0]) if abs(n[0]) < 0.9 else np.array([0, 1.0, 0])
    e1 = np.cross(n, a)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    return n, e1, e2


def _brute(poly2d):
    """Polar quadrature about the origin of a star-shaped polygon given in 2-D (CCW)."""
    P = np.asarray(poly2d)
    ang = np.arctan2(P[:, 1], P[:, 0])

    def rmax(phi):
        d = np.array([np.cos(phi), np.sin(phi)])
        best = np.inf
        for i in range(len(P)):
            a, b = P[i], P[(i + 1) % len(P)]
            e = b - a
            M = np.array([d, -e]).T
            det = np.linalg.det(M)
            if abs(det) < 1e-15:
                continue
            t, s = np.linalg.solve(M, a)
            if t > 0 and -1e-12 <= s <= 1 + 1e-12:
                best = min(best, t)
        return best

    pts = sorted(np.mod(ang, 2 * np.pi))
    opts = dict(points=pts, limit=500, epsabs=1e-13, epsrel=1e-12)
    I1 = integrate.quad(lambda p: rmax(p), 0, 2 * np.pi, **opts)[0]
    S = integrate.quad(lambda p: 0.5 * rmax(p) ** 2, 0, 2 * np.pi, **opts)[0]
    V1 = [integrate.quad(lambda p: 0.5 * rmax(p) ** 2 * np.cos(p), 0, 2 * np.pi, **opts)[0],
          integrate.quad(lambda p: 0.5 * rmax(p) ** 2 * np.sin(p), 0, 2 * np.pi, **opts)[0]]
    # CPV int rhohat/rho^2 dA = int rhohat ln(rmax) dphi (the ln of the excluded radius
    # integrates to zero over the full circle)
    V3 = [integrate.quad(lambda p: np.log(rmax(p)) * np.cos(p), 0, 2 * np.pi, **opts)[0],
          integrate.quad(lambda p: np.log(rmax(p)) * np.sin(p), 0, 2 * np.pi, **opts)[0]]
    return I1, S, np.array(V1), np.array(V3)


def _random_star_polygon(rng, nv):
    ang = np.sort(rng.uniform(0, 2 * np.pi, nv))
    # keep angular gaps below pi so that the origin is strictly inside
    while np.max(np.diff(np.concatenate([ang, [ang[0] + 2 * np.pi]]))) > 0.9 * np.pi:
        ang = np.sort(rng.uniform(0, 2 * np.pi, nv))
    r = rng.uniform(0.3, 1.5, nv)
    return np.stack([r * np.cos(ang), r * np.sin(ang)], 1)


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4])
def test_polygon_integrals_match_brute_force(seed):
    rng = np.random.default_rng(seed)
    poly = _random_star_polygon(rng, int(rng.integers(3, 9)))
    n, e1, e2 = _frame(rng.normal(size=3))
    pts3 = poly[:, :1] * e1 + poly[:, 1:] * e2
    I1, S, V1, V3 = oracle.polygon_integrals(pts3, n)
    bI1, bS, bV1, bV3 = _brute(poly)
    assert abs(I1 - bI1) < 1e-10 * max(1, abs(bI1))
    assert abs(S - bS) < 1e-10
    np.testing.assert_allclose([V1 @ e1, V1 @ e2], bV1, atol=1e-10)
    np.testing.assert_allclose([V3 @ e1, V3 @ e2], bV3, atol=1e-9)
    # the vectors lie in the plane of the polygon
    assert abs(V1 @ n) < 1e-12 and abs(V3 @ n) < 1e-12


def test_disk_limit_and_symmetry():
    a = 0.7
    for m in (64, 512, 4096):
        th = 2 * np.pi * np.arange(m) / m
        pts = np.stack([a * np.cos(th), a * np.sin(th), 0 * th], 1)
        I1, S, V1, V3 = oracle.polygon_integrals(pts, np.array([0, 0, 1.0]))
        # inscribed regular m-gon: exact I1 = m a cos(pi/m) * 2 asinh(tan(pi/m))
        exact = m * a * np.cos(np.pi / m) * 2 * np.arcsinh(np.tan(np.pi / m))
        assert abs(I1 - exact) < 1e-12
        assert abs(S - 0.5 * m * a * a * np.sin(2 * np.pi / m)) < 1e-12
        assert np.linalg.norm(V1) < 1e-12 and np.linalg.norm(V3) < 1e-10
    assert abs(I1 - 2 * np.pi * a) < 1e-5


def test_centroid_self_patch_matches_brute_force():
    import fmbem_inputs as fi
    V, F, D = fi.icosphere(1)
    o = oracle.Oracle(V, F, D, [1.0, 2.25], [1.0, 1.0], 1.0, mode="centroid")
    for t in (0, 7, 33):
        A, B, C = V[F[t]]
        n, e1, e2 = o.n[t], None, None
        n, e1, e2 = _frame(n)
        O = o.s[t]
        poly = np.array([[(P - O) @ e1, (P - O) @ e2] for P in (A, B, C)])
        bI1, bS, bV1, bV3 = _brute(poly)
        assert abs(o.I1[t] - bI1) < 1e-10
        assert abs(o.S[t] - bS) < 1e-12
        assert abs(o.S[t] - o.w[t]) < 1e-12          # the patch of a centroid node is its triangle
        np.testing.assert_allclose([o.V3[t] @ e1, o.V3[t] @ e2], bV3, atol=1e-9)


def test_vertex_dual_cells_tile_the_mesh():
    """Vertex weights are one third of the incident areas, so they sum to the mesh area; the
    projected dual cells are planar polygons of about the same area; symmetric cells have
    vanishing first moments."""
    import fmbem_inputs as fi
    V, F, D = fi.icosphere(3)
    o = oracle.Oracle(V, F, D, [1.0, 2.25], [1.0, 1.0], 1.0)
    A, B, C = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(B - A, C - A), axis=1).sum()
    assert abs(o.w.sum() - area) < 1e-12 * area
    assert np.all(o.S <= o.w * (1 + 1e-12))
    assert abs(o.S.sum() / area - 1) < 1e-2      # projection onto the tangent planes shrinks by O(h^2)
    # normals: unit, outward on the sphere
    assert np.allclose(np.linalg.norm(o.n, axis=1), 1)
    assert np.all(np.einsum("ij,ij->i", o.n, o.s) > 0.99)
    # the 12 five-fold vertices of the icosahedron keep their 5-fold symmetry under midpoint
    # refinement, so their dual cells give V1 = V3 = 0; the other vertices do not
    np.testing.assert_allclose(o.V1[:12], 0, atol=1e-14)
    np.testing.assert_allclose(o.V3[:12], 0, atol=1e-12)
    assert np.max(np.linalg.norm(o.V3[12:], axis=1)) > 1e-3
