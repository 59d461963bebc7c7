"""A stand-in for the library handle on the CPU: a small dense system A(V, eps) x = b(V) on the
vertex positions V (one node per vertex), a far-field-like functional L(V), and near fields
E, H linear in x through a smooth kernel of the distance to each node.  Its methods mirror the
handle's, and the shape gradients are central differences of L^T x + lambda^T b - lambda^T A x
(or its near-field analogue) at fixed x and lambda, so that the autograd wrappers' adjoint
assembly can be checked against central differences of their own forward values."""
import numpy as np
import torch


class FakeHandle:
    def __init__(self, V, F, D, eps, mu, k0, **options):
        self.V = np.asarray(V, dtype=np.float64)
        self.eps = [complex(e) for e in eps]
        self.N = len(self.V)
        self.kb = complex(k0)

    def _A(self, V):
        n = 6 * self.N
        i = np.arange(n)
        node = i // 6
        P = V[node]
        A = 0.2 * np.exp(1j * (P @ P.T)) / n + np.diag(3.0 + 0.5 * np.sin(P[:, 0] + 2 * P[:, 1]) + 0j)
        A += np.diag(np.where(i % 6 >= 3, self.eps[1], 1.0) * (1 + 0.1 * P[:, 2]))
        return A

    def _b(self, V, dirs, pols):
        ph = np.exp(1j * (dirs @ V.T))                          # [n, N]
        b = np.zeros((len(dirs), self.N, 6), dtype=np.complex128)
        b[:, :, :3] = ph[:, :, None] * pols[:, None, :]
        return b

    def _L(self, V, dirs, coef):
        ph = np.exp(-1j * (dirs @ V.T))
        L = np.zeros((len(dirs), self.N, 6), dtype=np.complex128)
        L[:, :, :3] = ph[:, :, None] * coef[:, None, :]
        L[:, :, 3:] = 0.3 * ph[:, :, None] * np.cos(V)[None] * coef[:, None, :]
        return L

    def plane_wave_rhs(self, dirs, pols):
        self._dirs, self._pols = dirs, pols
        return torch.from_numpy(self._b(self.V, dirs, pols))

    def solve(self, b, tol=1e-10, **kw):
        A = self._A(self.V)
        x = np.stack([np.linalg.solve(A, bb.reshape(-1)).reshape(self.N, 6) for bb in b.numpy()])
        return torch.from_numpy(x), None, None, 0

    def adjoint_solve(self, L, tol=1e-10, **kw):
        A = self._A(self.V)
        lam = np.stack([np.linalg.solve(A.T, ll.reshape(-1)).reshape(self.N, 6) for ll in L.numpy()])
        return torch.from_numpy(lam), None, None, 0

    def matvec(self, x, **kw):
        A = self._A(self.V)
        return torch.from_numpy(np.stack([(A @ xx.reshape(-1)).reshape(self.N, 6) for xx in x.numpy()]))

    def far_field_functional(self, dirs, coef):
        self._coef = coef
        return torch.from_numpy(self._L(self.V, dirs, coef))

    def shape_gradient(self, x, lam, dirs, pols, rhat, coef):
        x, lam = x.numpy(), lam.numpy()
        h = 1e-6
        out = np.zeros((len(dirs), self.N, 3), dtype=np.complex128)

        def G(V):
            A = self._A(V)
            Ax = np.stack([(A @ xx.reshape(-1)).reshape(self.N, 6) for xx in x])
            return (np.sum(self._L(V, rhat, coef) * x, axis=(1, 2)) + np.sum(lam * self._b(V, dirs, pols), axis=(1, 2))
                    - np.sum(lam * Ax, axis=(1, 2)))

        for v in range(self.N):
            for c in range(3):
                Vp, Vm = self.V.copy(), self.V.copy()
                Vp[v, c] += h
                Vm[v, c] -= h
                out[:, v, c] = (G(Vp) - G(Vm)) / (2 * h)
        return out

    # ---- near fields: E = E_inc + sum_b K(r, s_b) (Phi_b + 0.2 Psi_b), H = H_inc + sum_b 0.5 K Psi_b
    def _vacuum_background(self):
        pass

    @staticmethod
    def _K(P, V):
        R = np.linalg.norm(P[:, None, :] - V[None, :, :], axis=-1)
        return np.exp(1j * R) / R                                   # [P, N]

    def near_field(self, x, pts, dirs=None, pols=None, magnetic=False, **kw):
        x = x.numpy()
        K = self._K(np.asarray(pts), self.V)
        E = np.einsum("pb,rbq->rpq", K, x[:, :, :3] + 0.2 * x[:, :, 3:])
        H = np.einsum("pb,rbq->rpq", K, 0.5 * x[:, :, 3:])
        if dirs is not None:
            d, e = np.atleast_2d(dirs), np.atleast_2d(pols)
            ph = np.exp(1j * (np.asarray(pts) @ d.T)).T               # [n, P]
            E = E + ph[:, :, None] * e[:, None, :]
            H = H + ph[:, :, None] * np.cross(d, e)[:, None, :]
        return (E, H) if magnetic else E

    def _N(self, V, pts, cE, cH):
        K = self._K(np.asarray(pts), V)
        N = np.zeros((cE.shape[0], self.N, 6), dtype=np.complex128)
        N[:, :, :3] = np.einsum("pb,fpq->fbq", K, cE)
        N[:, :, 3:] = np.einsum("pb,fpq->fbq", K, 0.2 * cE + 0.5 * cH)
        return N

    def near_field_functional(self, pts, cE, cH=None):
        return torch.from_numpy(self._N(self.V, pts, cE, cH))

    def shape_gradient_near(self, x, lam, dirs, pols, pts, cE, cH=None):
        x, lam = x.numpy(), lam.numpy()
        h = 1e-6
        out = np.zeros((x.shape[0], self.N, 3), dtype=np.complex128)

        def G(V):
            A = self._A(V)
            Ax = np.stack([(A @ xx.reshape(-1)).reshape(self.N, 6) for xx in x])
            return (np.sum(self._N(V, pts, cE, cH) * x, axis=(1, 2)) + np.sum(lam * self._b(V, dirs, pols), axis=(1, 2))
                    - np.sum(lam * Ax, axis=(1, 2)))

        for v in range(self.N):
            for c in range(3):
                Vp, Vm = self.V.copy(), self.V.copy()
                Vp[v, c] += h
                Vm[v, c] -= h
                out[:, v, c] = (G(Vp) - G(Vm)) / (2 * h)
        return out

    # ---- the library's reductions, restated on the stand-in system
    def cross_sections(self, x, dirs, pols, n_theta=2, n_phi=2):
        """C_ext = Im(L^T x) with L the far-field-like functional of (dirs, 4 pi / k conj(pols))."""
        dirs, pols = np.atleast_2d(dirs), np.atleast_2d(pols)
        L = self._L(self.V, dirs, 4 * np.pi / self.kb.real * np.conj(pols))
        cext = np.sum(L * x.numpy(), axis=(1, 2)).imag
        return cext, np.zeros_like(cext), np.zeros_like(cext)

    def eps_sensitivity(self, j, x, lam, step=None):
        """lambda^T (dA/deps_j) x by the central difference of the stand-in operator."""
        h = 1e-5 if step is None else step
        e0 = self.eps[j]
        self.eps[j] = e0 + h
        Ap = self._A(self.V)
        self.eps[j] = e0 - h
        Am = self._A(self.V)
        self.eps[j] = e0
        dA = (Ap - Am) / (2 * h)
        x, lam = x.numpy(), lam.numpy()
        return np.array([np.sum(ll.reshape(-1) * (dA @ xx.reshape(-1))) for xx, ll in zip(x, lam)])

    def force_stress_functional(self, x, d, e, center, radius, n_theta=24, n_phi=48):
        """Stress-type force of the stand-in fields on a sphere and the functionals of its
        components' Wirtinger coefficients (the quantities fmbem_force_stress_functional returns)."""
        mu, wmu = np.polynomial.legendre.leggauss(n_theta)
        ph = 2 * np.pi * np.arange(n_phi) / n_phi
        MU, PH = np.meshgrid(mu, ph, indexing="ij")
        ST = np.sqrt(1 - MU ** 2)
        nq = np.stack([ST * np.cos(PH), ST * np.sin(PH), MU], -1).reshape(-1, 3)
        wq = (wmu[:, None] * np.full(n_phi, 2 * np.pi / n_phi)[None, :]).ravel() * radius ** 2
        pts = np.asarray(center, dtype=np.float64)[None, :] + radius * nq
        E, H = self.near_field(x, pts, d, e, magnetic=True)
        E, H = E[0], H[0]
        en, hn = np.sum(np.conj(E) * nq, 1), np.sum(np.conj(H) * nq, 1)
        u = np.sum(np.abs(E) ** 2 + np.abs(H) ** 2, 1)
        force = np.sum(wq[:, None] * 0.5 * np.real(E * en[:, None] + H * hn[:, None] - 0.5 * u[:, None] * nq), 0)
        eye = np.eye(3)

        def wirtinger(Fv, fn):
            c = (eye[:, None, :] * fn[None, :, None] + np.conj(Fv).T[:, :, None] * nq[None, :, :]
                 - nq.T[:, :, None] * np.conj(Fv)[None, :, :])
            return 0.25 * wq[None, :, None] * c

        cE, cH = wirtinger(E, en), wirtinger(H, hn)
        return force, pts, cE, cH, self.near_field_functional(pts, cE, cH)
