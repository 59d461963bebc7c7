"""The adjoint-gradient building blocks on the device and the torch.autograd functions over them.

- fmbem_cross_sections (far fields, quadrature and absorption reduced on the device) against the
  far-field amplitudes integrated here with the same rule;
- fmbem_force_stress against the stress tensor integrated here from fmbem_near_field's fields;
- fmbem_force_stress_functional: its force equals fmbem_force_stress's, and its functionals
  predict the force's change under a small change of the solution (dF_i = 2 Re L_i^T dx);
- fmbem_eps_sensitivity against the central difference of two handles' products;
- autograd.extinction and autograd.force: .backward() gives the gradients of the gradient
  functions (themselves pinned to the dense oracle and to central differences of GPU solves in
  test_gpu_parity.py), and NaN for the background permittivity."""
import numpy as np
import pytest

import fmbem_inputs as fi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1211_7177_gb300 as fm  # noqa: E402
from paper_1211_7177_gb300 import autograd, gradients  # noqa: E402


def sphere_rule(nt, nphi):
    mu, wmu = np.polynomial.legendre.leggauss(nt)
    ph = 2 * np.pi * np.arange(nphi) / nphi
    MU, PH = np.meshgrid(mu, ph, indexing="ij")
    ST = np.sqrt(1 - MU ** 2)
    q = np.stack([ST * np.cos(PH), ST * np.sin(PH), MU], -1).reshape(-1, 3)
    w = (wmu[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).ravel()
    return q, w


@pytest.fixture(scope="module")
def two_spheres():
    """Two dielectric spheres a = 0.5 (eps 2.25 and -2 + 0.5i), 162 nodes each, k0 = 1, and the
    solutions of two plane waves."""
    V, F, D = fi.merge_meshes(fi.icosphere(2, 0.5, (-0.7, 0, 0)), fi.icosphere(2, 0.5, (0.7, 0, 0), domain=2))
    eps, mu, k0 = [1.0, 2.25, -2 + 0.5j], [1.0, 1.0, 1.0], 1.0
    g = fm.FMBEM(V, F, D, eps, mu, k0, p=10)
    dirs = np.array([[0.0, 0.0, 1.0], [0.6, 0.0, 0.8]])
    pols = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]], dtype=np.complex128)
    x, _, _, st = g.solve(g.plane_wave_rhs(dirs, pols), tol=1e-10)
    assert st == 0
    yield (V, F, D, eps, mu, k0), g, x, dirs, pols
    g.close()


def test_cross_sections_on_the_device(two_spheres):
    _, g, x, dirs, pols = two_spheres
    cext, csca, cabs = g.cross_sections(x, dirs, pols, n_theta=24, n_phi=48)
    q, w = sphere_rule(24, 48)
    F = g.far_field(x, np.concatenate([dirs, q]))
    for r in range(2):
        e_ref = 4 * np.pi / g.kb.real * np.imag(np.vdot(pols[r], F[r, r]))
        s_ref = np.sum(w * np.sum(np.abs(F[r, 2:]) ** 2, axis=1))
        a_ref = -fm.fmbem_absorption(g.h, x)[r] / g.kb.real
        assert abs(cext[r] - e_ref) < 1e-12 * abs(e_ref)
        assert abs(csca[r] - s_ref) < 1e-12 * abs(s_ref)
        assert abs(cabs[r] - a_ref) < 1e-12 * abs(a_ref)
        # energy balance of the discrete solution (optical theorem), to discretisation error
        assert abs(cext[r] - csca[r] - cabs[r]) < 0.05 * abs(cext[r])


def test_stress_force_and_its_functional_on_the_device(two_spheres):
    _, g, x, dirs, pols = two_spheres
    c, rad = np.array([0.7, 0.0, 0.0]), 0.65
    Fd = g.force_stress(x, dirs, pols, c, rad, n_theta=16, n_phi=32)
    q, w = sphere_rule(16, 32)
    pts = c + rad * q
    E, H = g.near_field(x, pts, dirs, pols, magnetic=True)
    for r in range(2):
        en = np.sum(np.conj(E[r]) * q, 1)
        hn = np.sum(np.conj(H[r]) * q, 1)
        u = np.sum(np.abs(E[r]) ** 2 + np.abs(H[r]) ** 2, 1)
        ref = np.sum((w * rad ** 2)[:, None] * 0.5 * np.real(E[r] * en[:, None] + H[r] * hn[:, None] - 0.5 * u[:, None] * q), 0)
        assert np.allclose(Fd[r], ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())
    x0 = x[:1].contiguous()
    force, pts2, cE, cH, L = g.force_stress_functional(x0, dirs[0], pols[0], c, rad, n_theta=16, n_phi=32)
    assert np.allclose(force, Fd[0], rtol=1e-12, atol=1e-15)
    key = lambda a: a[np.lexsort(np.round(a, 9).T[::-1])]  # the same point set (node order may differ)
    assert np.allclose(key(pts2), key(pts))
    # first-order change of the force under a small change of the solution
    dx = 1e-6 * torch.from_numpy(fi.random_complex((1, g.N, 6), seed=3)).cuda()
    Fp = g.force_stress(x0 + dx, dirs[:1], pols[:1], c, rad, n_theta=16, n_phi=32)[0]
    Fm = g.force_stress(x0 - dx, dirs[:1], pols[:1], c, rad, n_theta=16, n_phi=32)[0]
    pred = 2 * torch.sum(L * dx, dim=(1, 2)).real.cpu().numpy()
    assert np.allclose((Fp - Fm) / 2, pred, rtol=1e-5, atol=1e-6 * np.abs(pred).max())


def test_eps_sensitivity_matches_two_handles(two_spheres):
    (V, F, D, eps, mu, k0), g, x, dirs, pols = two_spheres
    lam = torch.from_numpy(fi.random_complex((2, g.N, 6), seed=5)).cuda()
    for j in (1, 2):
        h = 1e-5 * max(1.0, abs(eps[j]))
        s = g.eps_sensitivity(j, x, lam, step=h)
        ep, em = list(eps), list(eps)
        ep[j] += h
        em[j] -= h
        gp, gm = fm.FMBEM(V, F, D, ep, mu, k0, p=10), fm.FMBEM(V, F, D, em, mu, k0, p=10)
        ref = torch.sum(lam * (gp.matvec(x) - gm.matvec(x)) / (2 * h), dim=(1, 2)).cpu().numpy()
        assert np.allclose(s, ref, rtol=1e-9), (j, s, ref)
        gp.close()
        gm.close()


def test_autograd_extinction_and_force_match_the_gradient_functions():
    """autograd.extinction / autograd.force .backward() against gradients.* on a 162-node sphere."""
    V, F, D = fi.icosphere(2)
    eps, mu, k0 = [1.0, 2.5 + 0.2j], [1.0, 1.0], 1.2
    d, e = np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0], dtype=np.complex128)
    opts = dict(p=10)
    Vt = torch.tensor(V, dtype=torch.float64, requires_grad=True)
    et = torch.tensor(np.asarray(eps, dtype=np.complex128), requires_grad=True)
    c = autograd.extinction(Vt, et, F, D, mu, k0, d, e, **opts)
    c.sum().backward()
    c_ref, gV = gradients.extinction_vertex_gradient(V, F, D, eps, mu, k0, d[None], e[None], **opts)
    _, dre, dim = gradients.extinction_eps_gradient(V, F, D, eps, mu, k0, d[None], e[None], j=1, **opts)
    assert abs(c.item() - c_ref[0]) < 1e-9 * abs(c_ref[0])
    assert np.allclose(Vt.grad.numpy(), gV[0], rtol=1e-6, atol=1e-8 * np.abs(gV).max())
    assert abs(et.grad[1].real.item() - dre[0]) < 1e-6 * abs(dre[0]) and abs(et.grad[1].imag.item() - dim[0]) < 1e-6 * abs(dim[0])
    assert torch.isnan(et.grad[0].real)
    # force on the sphere inside a sphere of radius 1.5 (z component)
    Vt = torch.tensor(V, dtype=torch.float64, requires_grad=True)
    et = torch.tensor(np.asarray(eps, dtype=np.complex128), requires_grad=True)
    f = autograd.force(Vt, et, F, D, mu, k0, d, e, [0, 0, 0], 1.5, **opts)
    f[2].backward()
    f_ref, gF = gradients.force_vertex_gradient(V, F, D, eps, mu, k0, d, e, [0, 0, 0], 1.5, **opts)
    _, fre, fim = gradients.force_eps_gradient(V, F, D, eps, mu, k0, d, e, 1, [0, 0, 0], 1.5, **opts)
    assert np.allclose(f.detach().numpy(), f_ref, rtol=1e-9, atol=1e-12)
    assert np.allclose(Vt.grad.numpy(), gF[2], rtol=1e-6, atol=1e-8 * np.abs(gF[2]).max())
    assert abs(et.grad[1].real.item() - fre[2]) < 1e-6 * abs(fre[2]) + 1e-12
    assert abs(et.grad[1].imag.item() - fim[2]) < 1e-6 * abs(fim[2]) + 1e-12
    assert torch.isnan(et.grad[0].real)
