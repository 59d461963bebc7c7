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


# ------------------------------------------------------------------ optical force (App. D)
def _sphere(center, radius, n_theta, n_phi):
    mu, wmu = np.polynomial.legendre.leggauss(n_theta)
    ph = 2 * np.pi * np.arange(n_phi) / n_phi
    MU, PH = np.meshgrid(mu, ph, indexing="ij")
    ST = np.sqrt(1 - MU ** 2)
    nq = np.stack([ST * np.cos(PH), ST * np.sin(PH), MU], -1).reshape(-1, 3)
    wq = (wmu[:, None] * np.full(n_phi, 2 * np.pi / n_phi)[None, :]).ravel() * radius ** 2
    return np.asarray(center, dtype=np.float64)[None] + radius * nq, nq, wq


def stress_force(o, x, d, e, center, radius, n_theta=12, n_phi=24):
    """Time-averaged Maxwell-stress force on the particles inside the sphere (center, radius):
    the surface integral of T n, T = 1/2 Re[E E* + H H* - 1/2 (|E|^2 + |H|^2) I] (vacuum
    background), with the oracle's total E and H on the sphere."""
    pts, nq, wq = _sphere(center, radius, n_theta, n_phi)
    E = o.near_field(x, pts, d, e)
    H = o.near_field_h(x, pts, d, e)
    en, hn = np.sum(np.conj(E) * nq, 1), np.sum(np.conj(H) * nq, 1)
    u = np.sum(abs(E) ** 2 + abs(H) ** 2, 1)
    return np.sum(wq[:, None] * 0.5 * np.real(E * en[:, None] + H * hn[:, None] - 0.5 * u[:, None] * nq), 0)


def force_vertex_gradient(V, F, D, eps, mu, k0, d, e, center, radius, n_theta=12, n_phi=24, h=1e-6,
                          return_state=False):
    """(F [3], dF/dV [3, nv, 3]) of the Maxwell-stress force by the dense adjoint formula (with
    return_state also x, lambda [3, N, 6], the stress points and the coefficients cE, cH).

    F_i is a real quadratic form of the fields on the stress sphere, so dF_i = 2 Re(sum_p cE_p . dE_p
    + cH_p . dH_p) with the holomorphic (Wirtinger) coefficients cE, cH of F_i at the current
    fields; with the fields' linear dependence on x, N_i(V)^T x = sum_p cE_p . E_sca(r_p) +
    cH_p . H_sca(r_p), and A^T lambda_i = N_i:
        dF_i/dtheta = 2 Re d/dtheta [ N_i^T x + lambda_i^T b - lambda_i^T A x ]  (x, lambda fixed)."""
    V = np.asarray(V, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    e = np.asarray(e, dtype=np.complex128)
    zero = np.zeros(3, dtype=np.complex128)
    o = Oracle(V, F, D, eps, mu, k0)
    A = dense_matrix(o)
    b = o.plane_wave_rhs(d, e)[0].reshape(-1)
    x = np.linalg.solve(A, b).reshape(o.N, 6)
    pts, nq, wq = _sphere(center, radius, n_theta, n_phi)
    E = o.near_field(x, pts, d, e)
    H = o.near_field_h(x, pts, d, e)
    en, hn = np.sum(np.conj(E) * nq, 1), np.sum(np.conj(H) * nq, 1)
    u = np.sum(abs(E) ** 2 + abs(H) ** 2, 1)
    force = np.sum(wq[:, None] * 0.5 * np.real(E * en[:, None] + H * hn[:, None] - 0.5 * u[:, None] * nq), 0)
    eye = np.eye(3)

    def wirtinger(Fv, fn):  # [3 (component i), P, 3]: d F_i / d F_j at point p
        return 0.25 * wq[None, :, None] * (eye[:, None, :] * fn[None, :, None] + np.conj(Fv).T[:, :, None] * nq[None]
                                           - nq.T[:, :, None] * np.conj(Fv)[None])

    cE, cH = wirtinger(E, en), wirtinger(H, hn)

    def functional(op, xx, i):  # sum_p cE . E_sca + cH . H_sca of the solution xx on op's geometry
        Es = op.near_field(xx, pts, d, zero)
        Hs = op.near_field_h(xx, pts, d, zero)
        return np.sum(cE[i] * Es) + np.sum(cH[i] * Hs)

    # N_i from the functional of unit vectors (it is linear in x), then the adjoints
    lam = []
    for i in range(3):
        Ni = np.zeros((o.N, 6), dtype=np.complex128)
        for bnode in range(o.N):
            for q in range(6):
                unit = np.zeros((o.N, 6), dtype=np.complex128)
                unit[bnode, q] = 1.0
                Ni[bnode, q] = functional(o, unit, i)
        lam.append(np.linalg.solve(A.T, Ni.reshape(-1)).reshape(o.N, 6))

    grad = np.zeros((3, len(V), 3))
    for v in range(len(V)):
        for c in range(3):
            Gs = []
            for sgn in (1, -1):
                Vx = V.copy()
                Vx[v, c] += sgn * h
                op = Oracle(Vx, F, D, eps, mu, k0)
                bx = op.plane_wave_rhs(d, e)[0]
                Ax = op.matvec(x)
                Gs.append([functional(op, x, i) + np.sum(lam[i] * bx) - np.sum(lam[i] * Ax) for i in range(3)])
            for i in range(3):
                grad[i, v, c] = 2 * np.real((Gs[0][i] - Gs[1][i]) / (2 * h))
    if return_state:  # the dense solution, adjoints [3, N, 6], stress points and coefficients
        return force, grad, x, np.stack(lam), pts, cE, cH
    return force, grad


def force(V, F, D, eps, mu, k0, d, e, center, radius, n_theta=12, n_phi=24):
    """Maxwell-stress force of a dense solve on the mesh (V, F, D)."""
    o = Oracle(np.asarray(V, dtype=np.float64), F, D, eps, mu, k0)
    A = dense_matrix(o)
    x = np.linalg.solve(A, o.plane_wave_rhs(d, e)[0].reshape(-1)).reshape(o.N, 6)
    return stress_force(o, x, d, e, center, radius, n_theta, n_phi)
