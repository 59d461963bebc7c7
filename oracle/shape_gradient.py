"""Dense reference for the gradient of the extinction cross section with respect to the mesh
vertex positions (vertex nodes), by the adjoint method of the discrete system of Eq. (2.9).

TEST INFRASTRUCTURE ONLY: used by the tests; no product code imports it.

For one plane wave (d, e), C_ext = Im f with f = (4 pi / k) conj(e) . F(d) (optical theorem, F the
far-field amplitude of the representation formula, Appendix A).  With A(V) x = b(V) and
f = L(V)^T x (complex bilinear), the adjoint lambda, A^T lambda = L, gives for every vertex
coordinate theta

    df/dtheta = d/dtheta [ L(V)^T x + lambda^T b(V) - lambda^T A(V) x ]   at fixed x and lambda,

and the derivative of the bracket is taken here as the central difference of the oracle's own
dense quantities rebuilt on the perturbed mesh (node positions, weights, normals and self
patches all follow the vertices).  Everything is dense FP64 and O(N^2) per coordinate, meant for
meshes of a few hundred nodes."""
from __future__ import annotations

import numpy as np

from . import Oracle


def _functional_value(o, x, d, e):
    """f = (4 pi / k) conj(e) . F(d) of the solution x [N, 6] on the oracle o's geometry."""
    k = o.k[0].real
    return 4 * np.pi / k * np.dot(np.conj(e), o.far_field(x, np.asarray(d)[None])[0])


def _functional_coefficients(o, d, e):
    """L [N, 6] with f(x) = sum L * x, from the far field of unit vectors (f is linear in x)."""
    L = np.zeros((o.N, 6), dtype=np.complex128)
    for b in range(o.N):
        for q in range(6):
            u = np.zeros((o.N, 6), dtype=np.complex128)
            u[b, q] = 1.0
            L[b, q] = _functional_value(o, u, d, e)
    return L


def dense_matrix(o):
    """A [6N, 6N] from the oracle's matvec of the identity."""
    n = 6 * o.N
    return o.matvec(np.eye(n, dtype=np.complex128).reshape(n, o.N, 6)).reshape(n, n).T


def extinction_vertex_gradient(V, F, D, eps, mu, k0, d, e, h=1e-6, return_state=False):
    """(C_ext, dC_ext/dV [nv, 3]) for the plane wave (d, e) by the dense adjoint formula above;
    with return_state also the dense solution x and adjoint lambda ([N, 6] each)."""
    V = np.asarray(V, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    e = np.asarray(e, dtype=np.complex128)
    o = Oracle(V, F, D, eps, mu, k0)
    A = dense_matrix(o)
    b = o.plane_wave_rhs(d, e)[0].reshape(-1)
    x = np.linalg.solve(A, b).reshape(o.N, 6)
    L = _functional_coefficients(o, d, e)
    lam = np.linalg.solve(A.T, L.reshape(-1)).reshape(o.N, 6)
    cext = float(np.imag(np.sum(L * x)))

    def G(Vp):
        op = Oracle(Vp, F, D, eps, mu, k0)
        bp = op.plane_wave_rhs(d, e)[0]
        return _functional_value(op, x, d, e) + np.sum(lam * bp) - np.sum(lam * op.matvec(x))

    grad = np.zeros_like(V)
    for v in range(len(V)):
        for c in range(3):
            Vp, Vm = V.copy(), V.copy()
            Vp[v, c] += h
            Vm[v, c] -= h
            grad[v, c] = np.imag((G(Vp) - G(Vm)) / (2 * h))
    if return_state:
        return cext, grad, x, lam
    return cext, grad


def extinction(V, F, D, eps, mu, k0, d, e):
    """C_ext of a dense solve on the mesh (V, F, D)."""
    o = Oracle(np.asarray(V, dtype=np.float64), F, D, eps, mu, k0)
    A = dense_matrix(o)
    x = np.linalg.solve(A, o.plane_wave_rhs(d, e)[0].reshape(-1)).reshape(o.N, 6)
    return float(np.imag(_functional_value(o, x, d, e)))
