"""Plumbing of autograd.extinction on the CPU, with a stand-in for the library handle: a small
dense system A(V, eps) x = b(V) with a functional f = L(V)^T x, whose methods mirror the handle's
(solve, adjoint_solve, matvec, far_field_functional, plane_wave_rhs, and shape_gradient as the
central difference of L^T x + lambda^T b - lambda^T A x at fixed x and lambda).  The autograd
function's gradients with respect to the vertex positions and the permittivities must then equal
central differences of its own forward value: this checks the adjoint assembly (signs, Re / Im,
PyTorch's complex convention, the weighting by the incoming gradient) independently of the GPU
kernels, which the GPU tests check against the dense oracle."""
import numpy as np
import pytest
import torch

import paper_1211_7177_gb300 as fm
from paper_1211_7177_gb300 import autograd


class _FakeHandle:
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


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(fm, "FMBEM", _FakeHandle)


def test_extinction_gradients_match_central_differences(fake):
    rng = np.random.default_rng(3)
    V0 = rng.normal(size=(4, 3)) * 0.5
    dirs = np.array([[0.0, 0.6, 0.8], [1.0, 0.0, 0.0]])
    pols = np.array([[1.0, 0.0, 0.0], [0.0, 0.6j, 0.8]], dtype=np.complex128)
    eps0 = np.array([1.0, 2.0 + 0.3j])
    wts = torch.tensor([0.7, -1.3], dtype=torch.float64)
    args = (None, None, [1.0, 1.0], 1.0, dirs, pols)

    def loss(V, eps):
        return torch.sum(wts * autograd.extinction(V, eps, *args))

    V = torch.tensor(V0, requires_grad=True)
    eps = torch.tensor(eps0, dtype=torch.complex128, requires_grad=True)
    loss(V, eps).backward()
    h = 1e-6
    with torch.no_grad():
        for v, c in ((0, 0), (2, 1), (3, 2)):
            Vp, Vm = V0.copy(), V0.copy()
            Vp[v, c] += h
            Vm[v, c] -= h
            fd = (loss(torch.tensor(Vp), torch.tensor(eps0)) - loss(torch.tensor(Vm), torch.tensor(eps0))) / (2 * h)
            assert abs(V.grad[v, c].item() - fd.item()) < 1e-6 * max(1.0, abs(fd.item())), (v, c)
        for dz in (h, 1j * h):
            ep, em = eps0.copy(), eps0.copy()
            ep[1] += dz
            em[1] -= dz
            fd = (loss(torch.tensor(V0), torch.tensor(ep)) - loss(torch.tensor(V0), torch.tensor(em))) / (2 * h)
            got = eps.grad[1].real if dz == h else eps.grad[1].imag
            assert abs(got.item() - fd.item()) < 1e-6 * max(1.0, abs(fd.item())), dz
