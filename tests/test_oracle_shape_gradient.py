"""Pins for the dense reference of the extinction gradient with respect to vertex positions
(oracle/shape_gradient.py): the adjoint formula against central differences of full dense
solves, and translation invariance (moving every vertex together leaves C_ext unchanged, so the
gradient sums to zero over all vertices)."""
import numpy as np

import fmbem_inputs as fi
from oracle import shape_gradient as sg


def _wave():
    d = np.array([0.36, 0.48, 0.8])
    e = np.array([0.8, 0.0, -0.36], dtype=np.complex128)
    return d, e - d * np.dot(d, e)


def test_adjoint_gradient_matches_full_solves_and_is_translation_invariant():
    V, F, D = fi.icosphere(1)
    eps, mu, k0 = [1.0, 2.25 + 0.1j], [1.0, 1.0], 1.0
    d, e = _wave()
    c, g = sg.extinction_vertex_gradient(V, F, D, eps, mu, k0, d, e)
    assert abs(c - sg.extinction(V, F, D, eps, mu, k0, d, e)) < 1e-12 * abs(c)
    h = 1e-6
    for v, cc in ((0, 0), (5, 2), (17, 1), (33, 0)):
        Vp, Vm = V.copy(), V.copy()
        Vp[v, cc] += h
        Vm[v, cc] -= h
        fd = (sg.extinction(Vp, F, D, eps, mu, k0, d, e) - sg.extinction(Vm, F, D, eps, mu, k0, d, e)) / (2 * h)
        assert abs(g[v, cc] - fd) < 1e-7 * np.abs(g).max(), (v, cc, g[v, cc], fd)
    assert np.abs(g.sum(0)).max() < 1e-7 * np.abs(g).max()


def test_two_scatterers_with_mu():
    m1 = fi.icosphere(1, 0.5, (-0.7, 0.0, 0.0), domain=1)
    m2 = fi.icosphere(1, 0.4, (0.6, 0.1, 0.0), domain=2)
    V, F, D = fi.merge_meshes(m1, m2)
    eps, mu, k0 = [1.0, 3.0 + 0.2j, -2.0 + 0.5j], [1.0, 1.7, 1.0], 1.2
    d, e = _wave()
    c, g = sg.extinction_vertex_gradient(V, F, D, eps, mu, k0, d, e)
    h = 1e-6
    for v, cc in ((3, 1), (50, 2)):
        Vp, Vm = V.copy(), V.copy()
        Vp[v, cc] += h
        Vm[v, cc] -= h
        fd = (sg.extinction(Vp, F, D, eps, mu, k0, d, e) - sg.extinction(Vm, F, D, eps, mu, k0, d, e)) / (2 * h)
        assert abs(g[v, cc] - fd) < 1e-7 * np.abs(g).max(), (v, cc, g[v, cc], fd)
    assert np.abs(g.sum(0)).max() < 1e-7 * np.abs(g).max()


def test_force_gradient_matches_full_solves():
    """The Maxwell-stress force on the smaller of two spheres: its dense adjoint vertex gradient
    against central differences of the force from full dense solves, for vertices of both
    spheres."""
    m1 = fi.icosphere(1, 0.5, (-0.6, 0.0, 0.0), domain=1)
    m2 = fi.icosphere(1, 0.3, (0.5, 0.1, 0.0), domain=2)
    V, F, D = fi.merge_meshes(m1, m2)
    eps, mu, k0 = [1.0, 2.25 + 0.1j, -4.0 + 0.5j], [1.0, 1.0, 1.0], 1.5
    d = np.array([0.6, 0.0, 0.8])
    e = np.array([0.8, 0.0, -0.6], dtype=np.complex128)
    ctr, rad = np.array([0.5, 0.1, 0.0]), 0.42
    Fo, g = sg.force_vertex_gradient(V, F, D, eps, mu, k0, d, e, ctr, rad)
    assert np.allclose(Fo, sg.force(V, F, D, eps, mu, k0, d, e, ctr, rad), rtol=1e-12, atol=1e-15)
    h = 1e-6
    for v, cc in ((50, 0), (60, 2), (3, 1)):
        Vp, Vm = V.copy(), V.copy()
        Vp[v, cc] += h
        Vm[v, cc] -= h
        fd = (sg.force(Vp, F, D, eps, mu, k0, d, e, ctr, rad) - sg.force(Vm, F, D, eps, mu, k0, d, e, ctr, rad)) / (2 * h)
        assert np.abs(g[:, v, cc] - fd).max() < 1e-7 * np.abs(g).max(), (v, cc, g[:, v, cc], fd)
