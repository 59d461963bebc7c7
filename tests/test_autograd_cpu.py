"""Plumbing of the adjoint gradients (autograd.extinction, autograd.force and the functions of
gradients.py) on the CPU, with a stand-in for the library handle: a small
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
from fake_handle import FakeHandle
from paper_1211_7177_gb300 import autograd


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(fm, "FMBEM", FakeHandle)


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
    # the background permittivity is held fixed: its entry is NaN, never a silent zero
    assert torch.isnan(eps.grad[0].real) and torch.isnan(eps.grad[0].imag)
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


def test_force_gradients_match_central_differences(fake):
    """The same check for autograd.force: the stress force (a real quadratic form of the fields on
    the stress sphere), its vertex gradient through shape_gradient_near and its permittivity
    gradient, each component weighted by the incoming gradient."""
    rng = np.random.default_rng(5)
    V0 = rng.normal(size=(4, 3)) * 0.5
    d = np.array([0.0, 0.6, 0.8])
    e = np.array([1.0, 0.0, 0.0], dtype=np.complex128)
    eps0 = np.array([1.0, 2.0 + 0.3j])
    wts = torch.tensor([0.4, -1.1, 0.9], dtype=torch.float64)
    args = (None, None, [1.0, 1.0], 1.0, d, e, np.zeros(3), 3.0, 6, 12)

    def loss(V, eps):
        return torch.sum(wts * autograd.force(V, eps, *args))

    V = torch.tensor(V0, requires_grad=True)
    eps = torch.tensor(eps0, dtype=torch.complex128, requires_grad=True)
    loss(V, eps).backward()
    # the background permittivity is held fixed: its entry is NaN, never a silent zero
    assert torch.isnan(eps.grad[0].real) and torch.isnan(eps.grad[0].imag)
    h = 1e-6
    with torch.no_grad():
        for v, c in ((0, 2), (1, 0), (3, 1)):
            Vp, Vm = V0.copy(), V0.copy()
            Vp[v, c] += h
            Vm[v, c] -= h
            fd = (loss(torch.tensor(Vp), torch.tensor(eps0)) - loss(torch.tensor(Vm), torch.tensor(eps0))) / (2 * h)
            assert abs(V.grad[v, c].item() - fd.item()) < 1e-6 * max(1.0, abs(fd.item())), (v, c, V.grad[v, c], fd)
        for dz in (h, 1j * h):
            ep, em = eps0.copy(), eps0.copy()
            ep[1] += dz
            em[1] -= dz
            fd = (loss(torch.tensor(V0), torch.tensor(ep)) - loss(torch.tensor(V0), torch.tensor(em))) / (2 * h)
            got = eps.grad[1].real if dz == h else eps.grad[1].imag
            assert abs(got.item() - fd.item()) < 1e-6 * max(1.0, abs(fd.item())), (dz, got, fd)


def test_gradient_functions_match_central_differences(fake):
    """gradients.extinction_vertex_gradient / extinction_eps_gradient / force_vertex_gradient /
    force_eps_gradient with the stand-in handle, against central differences of the extinction
    and of the force recomputed from scratch on displaced inputs."""
    from paper_1211_7177_gb300 import gradients as gr
    rng = np.random.default_rng(7)
    V0 = rng.normal(size=(4, 3)) * 0.5
    d = np.array([0.0, 0.6, 0.8])
    e = np.array([1.0, 0.0, 0.0], dtype=np.complex128)
    eps0 = [1.0, 2.0 + 0.3j]
    mu = [1.0, 1.0]
    h = 1e-6

    def cext(V, eps):
        return gr.extinction_vertex_gradient(V, None, None, eps, mu, 1.0, d[None], e[None])[0][0]

    def force(V, eps):
        return gr.force_vertex_gradient(V, None, None, eps, mu, 1.0, d, e, np.zeros(3), 3.0, 6, 12)[0]

    _, gV = gr.extinction_vertex_gradient(V0, None, None, eps0, mu, 1.0, d[None], e[None])
    _, gRe, gIm = gr.extinction_eps_gradient(V0, None, None, eps0, mu, 1.0, d[None], e[None], j=1)
    _, fV = gr.force_vertex_gradient(V0, None, None, eps0, mu, 1.0, d, e, np.zeros(3), 3.0, 6, 12)
    _, fRe, fIm = gr.force_eps_gradient(V0, None, None, eps0, mu, 1.0, d, e, 1, np.zeros(3), 3.0, 6, 12)
    for v, c in ((0, 1), (2, 2)):
        Vp, Vm = V0.copy(), V0.copy()
        Vp[v, c] += h
        Vm[v, c] -= h
        assert abs(gV[0, v, c] - (cext(Vp, eps0) - cext(Vm, eps0)) / (2 * h)) < 1e-6
        assert np.abs(fV[:, v, c] - (force(Vp, eps0) - force(Vm, eps0)) / (2 * h)).max() < 1e-6
    for dz, gc, gf in ((h, gRe[0], fRe), (1j * h, gIm[0], fIm)):
        ep, em = list(eps0), list(eps0)
        ep[1] += dz
        em[1] -= dz
        assert abs(gc - (cext(V0, ep) - cext(V0, em)) / (2 * h)) < 1e-6
        assert np.abs(gf - (force(V0, ep) - force(V0, em)) / (2 * h)).max() < 1e-6
