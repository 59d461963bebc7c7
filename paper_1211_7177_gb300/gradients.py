"""Adjoint gradients of the extinction cross section and of the optical force with respect to
the permittivities, and of the extinction with respect to the mesh vertex positions.

The extinction of a plane wave (d, e) is the imaginary part of a linear functional of the
solution, C_ext = Im f(x) with f(x) = (4 pi / k0) conj(e) . F(d) (optical theorem, F the far-field
amplitude of Section 4).  With A x = b and b independent of the permittivities, the adjoint
method gives for any parameter p of A

    df/dp = -lambda^T (dA/dp) x,   A^T lambda = L,   f(x) = L^T x,

so one forward solve and one adjoint solve serve every parameter.  A depends holomorphically on
eps_j (through k_j = k0 sqrt(eps_j mu_j), the jump T_j and the self blocks of Appendix B), so
(dA/deps_j) x is the complex derivative, taken by the library as the central difference of two FMM
products on operators with eps_j +- h (same mesh and tree, fmbem_eps_sensitivity); then

    dC/dRe(eps_j) = Im(df/deps_j),   dC/dIm(eps_j) = Re(df/deps_j).

Every solve, product, functional, reduction and far-field evaluation runs in the library's CUDA
kernels; this module only sequences the calls.
"""
from __future__ import annotations

import numpy as np

from . import FMBEM, FMBEMError


def extinction(handle, x, dirs, pols):
    """C_ext [n_rhs] of the solutions x [n_rhs, N, 6] (CUDA) of the plane waves (dirs, pols), by
    the optical theorem on the device (fmbem_cross_sections)."""
    return handle.cross_sections(x, dirs, pols, n_theta=2, n_phi=2)[0]


def extinction_eps_gradient(V, F, D, eps, mu, k0, dirs, pols, j, tol=1e-10, h=None, **options):
    """(C_ext, dC_ext/dRe(eps_j), dC_ext/dIm(eps_j)), each [n_rhs], for the plane waves
    (dirs[r], pols[r]) on the mesh (V, F, D) with permittivities eps and permeabilities mu
    (index 0 the background), by one forward and one adjoint GMRES solve to tol and the library's
    sensitivity lambda^T (dA/deps_j) x (fmbem_eps_sensitivity; h is its central-difference step,
    default 1e-5 max(1, |eps_j|))."""
    eps = [complex(e) for e in eps]
    if not 1 <= j < len(eps):
        raise ValueError("j must index a scatterer (1..J)")
    g = FMBEM(V, F, D, eps, mu, k0, **options)
    dirs = np.atleast_2d(np.asarray(dirs, dtype=np.float64))
    pols = np.atleast_2d(np.asarray(pols, dtype=np.complex128))
    x, _, _, st = g.solve(g.plane_wave_rhs(dirs, pols), tol=tol)
    if st != 0:
        raise FMBEMError(st, "forward solve did not converge")
    L = g.far_field_functional(dirs, 4 * np.pi / g.kb.real * np.conj(pols))
    cext = extinction(g, x, dirs, pols)
    lam, _, _, st = g.adjoint_solve(L, tol=tol)
    if st != 0:
        raise FMBEMError(st, "adjoint solve did not converge")
    df = -g.eps_sensitivity(j, x, lam, step=h)  # d f / d eps_j (holomorphic)
    return cext, df.imag, df.real


def extinction_vertex_gradient(V, F, D, eps, mu, k0, dirs, pols, tol=1e-10, **options):
    """(C_ext [n_rhs], dC_ext/dV [n_rhs, nv, 3]) for the plane waves (dirs[r], pols[r]) on the mesh
    (V, F, D) (vertex nodes): one forward and one adjoint GMRES solve through the FMM, then the
    vertex derivative of L^T x + lambda^T b - lambda^T A x at fixed x and lambda
    (fmbem_shape_gradient), whose imaginary part is the extinction's."""
    g = FMBEM(V, F, D, eps, mu, k0, **options)
    dirs = np.atleast_2d(np.asarray(dirs, dtype=np.float64))
    pols = np.atleast_2d(np.asarray(pols, dtype=np.complex128))
    x, _, _, st = g.solve(g.plane_wave_rhs(dirs, pols), tol=tol)
    if st != 0:
        raise FMBEMError(st, "forward solve did not converge")
    coef = 4 * np.pi / g.kb.real * np.conj(pols)
    L = g.far_field_functional(dirs, coef)
    cext = extinction(g, x, dirs, pols)
    lam, _, _, st = g.adjoint_solve(L, tol=tol)
    if st != 0:
        raise FMBEMError(st, "adjoint solve did not converge")
    grad = g.shape_gradient(x, lam, dirs, pols, dirs, coef)
    return cext, grad.imag


def _force_adjoint(g, d, e, center, radius, n_theta, n_phi, tol):
    """Forward solve, the Maxwell-stress force on the sphere (center, radius), the Wirtinger
    coefficients cE, cH [3, P, 3] of its components at the sphere points pts, their near-field
    functionals L [3, N, 6] (all from fmbem_force_stress_functional) and the adjoints lambda."""
    g._vacuum_background()
    x, _, _, st = g.solve(g.plane_wave_rhs(d, e), tol=tol)
    if st != 0:
        raise FMBEMError(st, "forward solve did not converge")
    force, pts, cE, cH, L = g.force_stress_functional(x, d, e, center, radius, n_theta, n_phi)
    lam, _, _, st = g.adjoint_solve(L, tol=tol)
    if st != 0:
        raise FMBEMError(st, "adjoint solve did not converge")
    return x, force, pts, cE, cH, lam


def force_eps_gradient(V, F, D, eps, mu, k0, d, e, j, center, radius, n_theta=24, n_phi=48, tol=1e-10, h=None,
                       **options):
    """(F [3], dF/dRe(eps_j) [3], dF/dIm(eps_j) [3]): the time-averaged Maxwell-stress force on the
    particles inside the sphere (center, radius) in the unit plane wave (d, e) (vacuum
    background), and its derivatives, by one forward solve, three adjoint solves (one per force
    component) and the operator derivative of extinction_eps_gradient.

    The force is a real quadratic form of the solution, F_i = sum_p w_p (T(E, H) n)_i, so
    dF_i = 2 Re(L_i^T dx) with L_i the holomorphic (Wirtinger) derivative: for the point p,
    dF_i/dE_j = w_p / 4 [delta_ij (conj(E).n) + conj(E_i) n_j - n_i conj(E_j)] (and likewise for
    H), mapped to the unknowns by fmbem_force_stress_functional.  With A^T lambda_i = L_i and
    s_i = lambda_i^T (dA/deps_j) x (fmbem_eps_sensitivity): dF_i/dRe(eps_j) = -2 Re(s_i),
    dF_i/dIm(eps_j) = 2 Im(s_i)."""
    eps = [complex(v) for v in eps]
    if not 1 <= j < len(eps):
        raise ValueError("j must index a scatterer (1..J)")
    g = FMBEM(V, F, D, eps, mu, k0, **options)
    d = np.asarray(d, dtype=np.float64).reshape(1, 3)
    e = np.asarray(e, dtype=np.complex128).reshape(1, 3)
    x, force, _, _, _, lam = _force_adjoint(g, d, e, center, radius, n_theta, n_phi, tol)
    sv = g.eps_sensitivity(j, x.expand(3, -1, -1).contiguous(), lam, step=h)  # s_i = lambda_i^T (dA/deps_j) x
    return force, -2 * sv.real, 2 * sv.imag


def force_vertex_gradient(V, F, D, eps, mu, k0, d, e, center, radius, n_theta=24, n_phi=48, tol=1e-10, **options):
    """(F [3], dF/dV [3, nv, 3]): the Maxwell-stress force of force_eps_gradient and its gradient
    with respect to the mesh vertex positions (vertex nodes; the stress sphere stays fixed), by
    one forward and three adjoint solves: dF_i/dV = 2 Re d/dV [N_i^T x + lambda_i^T b -
    lambda_i^T A x] at fixed x and lambda_i, N_i the near-field functional of F_i's Wirtinger
    coefficients (fmbem_shape_gradient_near)."""
    g = FMBEM(V, F, D, eps, mu, k0, **options)
    d = np.asarray(d, dtype=np.float64).reshape(1, 3)
    e = np.asarray(e, dtype=np.complex128).reshape(1, 3)
    x, force, pts, cE, cH, lam = _force_adjoint(g, d, e, center, radius, n_theta, n_phi, tol)
    x3 = x.expand(3, -1, -1).contiguous()
    out = g.shape_gradient_near(x3, lam, np.repeat(d, 3, 0), np.repeat(e, 3, 0), pts, cE, cH)
    return force, 2 * out.real
