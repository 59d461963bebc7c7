"""FP64 CPU oracle of the Nystrom EFIE boundary-element operator (arXiv 1211.7177).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg import this package.  The product library (``paper_1211_7177_gb300``) never
imports, links or runs anything here, and this package never imports the product.

``fmbem_oracle.c`` holds the arithmetic (plain C, double precision, OpenMP over target nodes):
the dense one-point Nystrom operator of Eqs. (2.9)-(2.12) with the analytic self-patch terms of
Appendix B, the block-diagonal preconditioner of Eq. (3.2), right-preconditioned GMRES of
Eq. (3.1), plane-wave right-hand sides and the far-field amplitude of the representation
formula (Appendix A).  This module compiles it with gcc on first use and wraps it with ctypes;
the cross sections below are short numpy reductions of the oracle's own outputs.

Readings taken where the paper is silent (each listed in the design notes):
vertex nodes use one third of the incident triangle areas and the area-weighted normal, and
their self patch is the barycentric dual cell projected on the tangent plane; T_j multiplies the
1/2 jump term of the scatterer equations; eps_0, mu_0 are the background's relative values;
k = k0 sqrt(eps mu) takes the root with Im k >= 0; the background equation uses n0 = -n and
n0 x curl E = -Psi.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmbem_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (no GPU needed).  Returns its path."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, dbl, i32 = ctypes.c_int64, ctypes.c_double, ctypes.c_int
            lib.oracle_create.restype = P
            lib.oracle_create.argtypes = [i32, i64, P, i64, P, P, i32, P, P, dbl, ctypes.c_char_p, i32]
            lib.oracle_destroy.argtypes = [P]
            lib.oracle_num_nodes.restype = i64
            lib.oracle_num_nodes.argtypes = [P]
            lib.oracle_geometry.argtypes = [P] * 9
            lib.oracle_wavenumbers.argtypes = [P, P]
            lib.oracle_precond_blocks.argtypes = [P, P]
            lib.oracle_matvec.argtypes = [P, i64, P, P]
            lib.oracle_matvec_rows.argtypes = [P, i64, i64, P, P, P]
            lib.oracle_matvec_transpose.argtypes = [P, i64, P, P]
            lib.oracle_matvec_transpose_rows.argtypes = [P, i64, i64, P, P, P]
            lib.oracle_precond_apply.argtypes = [P, i64, P, P]
            lib.oracle_plane_wave_rhs.argtypes = [P, i64, P, P, P]
            lib.oracle_gmres.restype = i32
            lib.oracle_gmres.argtypes = [P, P, P, dbl, i32, i32, i32, P, P]
            lib.oracle_far_field.argtypes = [P, P, i64, P, P]
            lib.oracle_near_field.argtypes = [P, P, i64, P, P, P, P]
            lib.oracle_near_field_h.argtypes = [P, P, i64, P, P, P, P]
            lib.oracle_polygon_integrals.argtypes = [i32, P, P, P]
            lib.oracle_ibc_matvec.argtypes = [P, i64, P, P]
            lib.oracle_interior_field.argtypes = [P, P, i64, P, P, P, P]
            lib.oracle_ibc_precond_blocks.argtypes = [P, P]
            lib.oracle_ibc_psi.argtypes = [P, i64, P, P]
            lib.oracle_ibc_zeta.argtypes = [P, P]
            lib.oracle_set_near_singular.argtypes = [P, dbl, i32]
            lib.oracle_patch_integral.argtypes = [P, i64, P, dbl, dbl, i32, P]
            lib.oracle_num_threads.restype = i32
            _lib = lib
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def polygon_integrals(pts, normal):
    """Appendix B integrals over a planar polygon given by its vertices relative to the
    evaluation point O (counter-clockwise about ``normal``): returns
    (I1 = int dA/rho, S = area, V1 = int r/r dA, V3 = CPV int r/r^3 dA)."""
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    nrm = np.ascontiguousarray(normal, dtype=np.float64)
    out = np.zeros(8)
    _load().oracle_polygon_integrals(len(pts), _ptr(pts), _ptr(nrm), _ptr(out))
    return out[0], out[1], out[2:5].copy(), out[5:8].copy()


class Oracle:
    """Dense FP64 Nystrom operator for one mesh and one set of media.

    ``eps``/``mu``: relative permittivity/permeability of the background (index 0) and of
    scatterers 1..J; ``k0``: vacuum wavenumber; ``mode``: 'vertex' or 'centroid' nodes."""

    def __init__(self, V, F, D, eps, mu, k0, mode="vertex", near_singular_radius=0.0, near_singular_levels=3):
        lib = _load()
        self.V = np.ascontiguousarray(V, dtype=np.float64)
        self.F = np.ascontiguousarray(F, dtype=np.int32)
        self.D = np.ascontiguousarray(D, dtype=np.int32)
        self.J = int(self.D.max())
        self.eps = np.ascontiguousarray(np.asarray(eps, dtype=np.complex128))
        self.mu = np.ascontiguousarray(np.asarray(mu, dtype=np.complex128))
        assert len(self.eps) == self.J + 1 and len(self.mu) == self.J + 1
        self.k0 = float(k0)
        self.mode = mode
        err = ctypes.create_string_buffer(256)
        h = lib.oracle_create(0 if mode == "vertex" else 1, len(self.V), _ptr(self.V), len(self.F), _ptr(self.F),
                              _ptr(self.D), self.J, _ptr(self.eps), _ptr(self.mu), self.k0, err, 256)
        if not h:
            raise ValueError("invalid mesh: " + err.value.decode())
        self._h = ctypes.c_void_p(h)
        self._lib = lib
        N = int(lib.oracle_num_nodes(self._h))
        self.N = N
        self.s = np.zeros((N, 3))
        self.n = np.zeros((N, 3))
        self.w = np.zeros(N)
        self.dom = np.zeros(N, dtype=np.int32)
        self.I1 = np.zeros(N)
        self.S = np.zeros(N)
        self.V1 = np.zeros((N, 3))
        self.V3 = np.zeros((N, 3))
        lib.oracle_geometry(self._h, _ptr(self.s), _ptr(self.n), _ptr(self.w), _ptr(self.dom), _ptr(self.I1),
                            _ptr(self.S), _ptr(self.V1), _ptr(self.V3))
        k = np.zeros(self.J + 1, dtype=np.complex128)
        lib.oracle_wavenumbers(self._h, _ptr(k))
        self.k = k
        # near-singular correction (off at radius 0, the paper's operator): a source node within
        # R < radius * sqrt(w) of the target contributes the integral of the kernel over its patch
        # (4^levels sub-triangles per flat piece, centroid rule) instead of the one-point term
        self.near_singular_radius = float(near_singular_radius)
        self.near_singular_levels = int(near_singular_levels)
        lib.oracle_set_near_singular(self._h, self.near_singular_radius, self.near_singular_levels)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None:
            self._lib.oracle_destroy(h)
            self._h = None

    def _vec(self, x):
        x = np.ascontiguousarray(x, dtype=np.complex128)
        if x.ndim == 2:
            x = x[None]
        assert x.shape[1:] == (self.N, 6), x.shape
        return x

    def matvec(self, x):
        """y = A x; x [n_rhs, N, 6] (or [N, 6]) complex128."""
        squeeze = np.ndim(x) == 2
        x = self._vec(x)
        y = np.empty_like(x)
        self._lib.oracle_matvec(self._h, x.shape[0], _ptr(x), _ptr(y))
        return y[0] if squeeze else y

    def patch_integral(self, b, point, k, levels=None):
        """(int g dA', int grad' g dA' [3]) over node b's patch seen from ``point`` with wavenumber
        k, by the subdivision rule of the near-singular correction (``levels`` defaults to the
        instance's)."""
        L = self.near_singular_levels if levels is None else int(levels)
        pt = np.ascontiguousarray(point, dtype=np.float64)
        out = np.zeros(8)
        k = complex(k)
        self._lib.oracle_patch_integral(self._h, int(b), _ptr(pt), k.real, k.imag, L, _ptr(out))
        return complex(out[0], out[1]), out[2::2] + 1j * out[3::2]

    def matvec_rows(self, x, rows):
        """Rows of A x for the node indices ``rows``: [n_rhs, len(rows), 6]."""
        squeeze = np.ndim(x) == 2
        x = self._vec(x)
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        y = np.empty((x.shape[0], len(rows), 6), dtype=np.complex128)
        self._lib.oracle_matvec_rows(self._h, x.shape[0], len(rows), _ptr(rows), _ptr(x), _ptr(y))
        return y[0] if squeeze else y

    def matvec_transpose(self, x):
        """y = A^T x (bilinear transpose); x [n_rhs, N, 6] (or [N, 6]) complex128."""
        squeeze = np.ndim(x) == 2
        x = self._vec(x)
        y = np.empty_like(x)
        self._lib.oracle_matvec_transpose(self._h, x.shape[0], _ptr(x), _ptr(y))
        return y[0] if squeeze else y

    def matvec_transpose_rows(self, x, rows):
        """Entries of A^T x for the node indices ``rows``: [n_rhs, len(rows), 6]."""
        squeeze = np.ndim(x) == 2
        x = self._vec(x)
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        y = np.empty((x.shape[0], len(rows), 6), dtype=np.complex128)
        self._lib.oracle_matvec_transpose_rows(self._h, x.shape[0], len(rows), _ptr(rows), _ptr(x), _ptr(y))
        return y[0] if squeeze else y

    def precond_blocks(self):
        M = np.zeros((self.N, 6, 6), dtype=np.complex128)
        self._lib.oracle_precond_blocks(self._h, _ptr(M))
        return M

    def precond_apply(self, v):
        squeeze = np.ndim(v) == 2
        v = self._vec(v)
        z = np.empty_like(v)
        self._lib.oracle_precond_apply(self._h, v.shape[0], _ptr(v), _ptr(z))
        return z[0] if squeeze else z

    def plane_wave_rhs(self, dirs, pols):
        dirs = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
        pols = np.ascontiguousarray(np.atleast_2d(pols), dtype=np.complex128)
        b = np.empty((len(dirs), self.N, 6), dtype=np.complex128)
        self._lib.oracle_plane_wave_rhs(self._h, len(dirs), _ptr(dirs), _ptr(pols), _ptr(b))
        return b

    def gmres(self, b, tol=1e-6, restart=50, max_iter=1000, precond=True, x0=None):
        """Right-preconditioned GMRES(restart) for each right-hand side.
        Returns (x [n_rhs,N,6], iters [n_rhs], relres [n_rhs], converged [n_rhs])."""
        b = self._vec(b)
        x = np.zeros_like(b) if x0 is None else self._vec(x0).copy()
        its, res, conv = [], [], []
        for r in range(b.shape[0]):
            xi = np.ascontiguousarray(x[r])
            it = ctypes.c_int(0)
            rr = ctypes.c_double(0)
            st = self._lib.oracle_gmres(self._h, _ptr(np.ascontiguousarray(b[r])), _ptr(xi), tol, restart, max_iter,
                                        1 if precond else 0, ctypes.byref(it), ctypes.byref(rr))
            x[r] = xi
            its.append(it.value)
            res.append(rr.value)
            conv.append(st == 0)
        return x, np.array(its), np.array(res), np.array(conv)

    def far_field(self, x, rhat):
        """Far-field amplitude F(rhat) (E_sca ~ exp(i k r)/r F) of one solution x [N,6]."""
        x = np.ascontiguousarray(x, dtype=np.complex128)
        assert x.shape == (self.N, 6)
        rhat = np.ascontiguousarray(np.atleast_2d(rhat), dtype=np.float64)
        F = np.empty((len(rhat), 3), dtype=np.complex128)
        self._lib.oracle_far_field(self._h, _ptr(x), len(rhat), _ptr(rhat), _ptr(F))
        return F

    def near_field(self, x, points, d, e):
        """Total electric field at exterior points [P,3] from the representation formula
        (Appendix A) for one solution x [N,6] excited by the plane wave (d, e)."""
        x = np.ascontiguousarray(x, dtype=np.complex128)
        pts = np.ascontiguousarray(np.atleast_2d(points), dtype=np.float64)
        d = np.ascontiguousarray(d, dtype=np.float64)
        e = np.ascontiguousarray(e, dtype=np.complex128)
        E = np.empty((len(pts), 3), dtype=np.complex128)
        self._lib.oracle_near_field(self._h, _ptr(x), len(pts), _ptr(pts), _ptr(d), _ptr(e), _ptr(E))
        return E

    def near_field_h(self, x, points, d, e):
        """Total magnetic field H = curl E / (i k0 mu_0) at exterior points [P,3] (the curl of
        the representation formula of near_field) for one solution x [N,6] of the plane wave
        (d, e)."""
        x = np.ascontiguousarray(x, dtype=np.complex128)
        pts = np.ascontiguousarray(np.atleast_2d(points), dtype=np.float64)
        d = np.ascontiguousarray(d, dtype=np.float64)
        e = np.ascontiguousarray(e, dtype=np.complex128)
        H = np.empty((len(pts), 3), dtype=np.complex128)
        self._lib.oracle_near_field_h(self._h, _ptr(x), len(pts), _ptr(pts), _ptr(d), _ptr(e), _ptr(H))
        return H

    def interior_field(self, x, points, domain, magnetic=False):
        """Fields inside the scatterers from the representation formula of each point's domain
        (``domain`` [P] scatterer ids): E [P,3], and with magnetic=True (E, H), H = curl E /
        (i k0 mu_j).  At a point outside its domain the same sum is the null-field integral."""
        x = np.ascontiguousarray(x, dtype=np.complex128)
        assert x.shape == (self.N, 6)
        pts = np.ascontiguousarray(np.atleast_2d(points), dtype=np.float64)
        dom = np.ascontiguousarray(np.broadcast_to(np.asarray(domain, dtype=np.int32), (len(pts),)))
        E = np.empty((len(pts), 3), dtype=np.complex128)
        H = np.empty((len(pts), 3), dtype=np.complex128) if magnetic else None
        self._lib.oracle_interior_field(self._h, _ptr(x), len(pts), _ptr(pts), _ptr(dom), _ptr(E),
                                        _ptr(H) if H is not None else None)
        return (E, H) if magnetic else E

    def cross_sections(self, x, d, e, n_theta=48, n_phi=96):
        """(C_ext, C_sca, C_abs) of one solution x for the incident plane wave (d, e), |e| = 1.
        C_ext by the optical theorem (4 pi / k) Im[e* . F(d)]; C_sca as the integral of |F|^2 over
        the unit sphere (Gauss-Legendre in cos(theta) x trapezoid in phi); C_abs as the inward
        flux of the time-averaged Poynting vector through the surface, Eq. (4.2), written with
        n x curl E = Psi:  -(1/k) sum_a w_a Im(Phi_a . conj(Psi_a))."""
        k = self.k[0]
        assert abs(k.imag) == 0.0
        k = k.real
        d = np.asarray(d, dtype=np.float64)
        e = np.asarray(e, dtype=np.complex128)
        Fd = self.far_field(x, d[None])[0]
        cext = 4 * np.pi / k * np.imag(np.vdot(e, Fd))
        mu, wmu = np.polynomial.legendre.leggauss(n_theta)
        ph = 2 * np.pi * np.arange(n_phi) / n_phi
        MU, PH = np.meshgrid(mu, ph, indexing="ij")
        ST = np.sqrt(1 - MU ** 2)
        rh = np.stack([ST * np.cos(PH), ST * np.sin(PH), MU], -1).reshape(-1, 3)
        F = self.far_field(x, rh)
        wq = (wmu[:, None] * np.full(n_phi, 2 * np.pi / n_phi)[None, :]).ravel()
        csca = float(np.sum(wq * np.sum(np.abs(F) ** 2, axis=1)))
        cabs = -1.0 / k * float(np.sum(self.w * np.imag(np.sum(x[:, :3] * np.conj(x[:, 3:]), axis=1))))
        return float(cext), csca, cabs

    # ---------------------------------------------------------------- impedance boundary condition
    # Section 2.3: scatterers modelled by Eq. (2.24) instead of their interior equations; the
    # system is Eq. (2.25) in E_0 alone, vectors [n_rhs, N, 3].  Z_j = sqrt(mu_j / eps_j) of each
    # scatterer's medium (principal root), zeta_j = i k0 mu_0 / Z_j.

    def ibc_zeta(self):
        """zeta_j = i k0 mu_0 / Z_j per scatterer, [J+1] (entry 0 unused)."""
        z = np.zeros(self.J + 1, dtype=np.complex128)
        self._lib.oracle_ibc_zeta(self._h, _ptr(z))
        return z

    def _vec3(self, x):
        x = np.ascontiguousarray(x, dtype=np.complex128)
        if x.ndim == 2:
            x = x[None]
        assert x.shape[1:] == (self.N, 3), x.shape
        return x

    def ibc_matvec(self, x):
        """y = A_IBC x, the operator of Eq. (2.25); x [n_rhs, N, 3] (or [N, 3])."""
        squeeze = np.ndim(x) == 2
        x = self._vec3(x)
        y = np.empty_like(x)
        self._lib.oracle_ibc_matvec(self._h, x.shape[0], _ptr(x), _ptr(y))
        return y[0] if squeeze else y

    def ibc_precond_blocks(self):
        """The 3x3 self blocks of Eq. (2.25), [N, 3, 3]."""
        M = np.zeros((self.N, 3, 3), dtype=np.complex128)
        self._lib.oracle_ibc_precond_blocks(self._h, _ptr(M))
        return M

    def ibc_psi(self, E):
        """Psi = n x curl E_0 implied by Eq. (2.24) for surface fields E [n_rhs, N, 3] (or [N, 3])."""
        squeeze = np.ndim(E) == 2
        E = self._vec3(E)
        P = np.empty_like(E)
        self._lib.oracle_ibc_psi(self._h, E.shape[0], _ptr(E), _ptr(P))
        return P[0] if squeeze else P

    def ibc_unknowns(self, E):
        """The 6-vector (Phi, Psi) of Eq. (2.12) for an impedance solution E [.., N, 3], so that
        the far field, near field and cross sections above apply to it."""
        return np.concatenate([np.asarray(E), self.ibc_psi(E)], axis=-1)

    def ibc_solve(self, b, tol=1e-10, restart=200, max_iter=2000):
        """Solve Eq. (2.25) A_IBC x = b for each right-hand side b [n_rhs, N, 3] by right-
        preconditioned GMRES (scipy's GMRES on A M^-1 with M the 3x3 self blocks; the residual it
        measures is the true residual).  Returns (x, relres [n_rhs])."""
        from scipy.sparse.linalg import LinearOperator, gmres
        b = self._vec3(b)
        Minv = np.linalg.inv(self.ibc_precond_blocks())
        n = 3 * self.N

        def apply(u):
            z = np.einsum("aij,aj->ai", Minv, u.reshape(self.N, 3))
            return self.ibc_matvec(z).reshape(n)

        op = LinearOperator((n, n), matvec=apply, dtype=np.complex128)
        xs, res = [], []
        for r in range(b.shape[0]):
            u, info = gmres(op, b[r].reshape(n), rtol=tol, atol=0.0, restart=restart, maxiter=max_iter)
            x = np.einsum("aij,aj->ai", Minv, u.reshape(self.N, 3))
            rr = np.linalg.norm(self.ibc_matvec(x) - b[r]) / np.linalg.norm(b[r])
            xs.append(x)
            res.append(rr)
        return np.stack(xs), np.array(res)
