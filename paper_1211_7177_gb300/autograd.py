"""Differentiable wrappers of the FMM-BEM product and solve, and of the extinction cross section
as a function of the vertex positions and permittivities, for torch.autograd.

The operator A (Eq. 2.9) is fixed by the handle; these functions are differentiable with respect
to their vector argument.  PyTorch's convention for complex tensors makes the gradient of a real
loss L with respect to a complex input z the vector g with dL = Re(sum conj(g) dz), so

  y = A x:      grad_x = A^H grad_y = conj(A^T conj(grad_y))      (fmbem_adjoint_matvec)
  x = A^-1 b:   grad_b = A^-H grad_x = conj(A^-T conj(grad_x))    (fmbem_adjoint_solve)

Every product and solve runs in the library's CUDA kernels.
"""
from __future__ import annotations

import torch

from . import FMBEMError, FP64


class _Matvec(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, handle, precision):
        ctx.handle, ctx.precision = handle, precision
        return handle.matvec(x.detach().contiguous(), precision=precision)

    @staticmethod
    def backward(ctx, gy):
        gx = ctx.handle.adjoint_matvec(gy.conj().contiguous(), precision=ctx.precision).conj()
        return gx, None, None


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, handle, tol, max_iter):
        x, _, _, st = handle.solve(b.detach().contiguous(), tol=tol, max_iter=max_iter)
        if st != 0:
            raise FMBEMError(st, "forward solve did not converge")
        ctx.handle, ctx.tol, ctx.max_iter = handle, tol, max_iter
        return x

    @staticmethod
    def backward(ctx, gx):
        lam, _, _, st = ctx.handle.adjoint_solve(gx.conj().contiguous(), tol=ctx.tol, max_iter=ctx.max_iter)
        if st != 0:
            raise FMBEMError(st, "adjoint solve did not converge")
        return lam.conj(), None, None, None


def matvec(handle, x, precision=FP64):
    """y = A x, differentiable in x (x: complex128 CUDA tensor [n_rhs, N, 6])."""
    return _Matvec.apply(x, handle, precision)


def solve(handle, b, tol=1e-8, max_iter=1000):
    """x = A^-1 b by GMRES, differentiable in b; the backward pass is one adjoint solve."""
    return _Solve.apply(b, handle, tol, max_iter)


class _Extinction(torch.autograd.Function):
    """C_ext [n_rhs] of the plane waves (dirs, pols) on the mesh with vertex positions V and
    permittivities eps; differentiable in V (through fmbem_shape_gradient) and in eps (through
    the operator's central difference in each eps_j, as gradients.extinction_eps_gradient)."""

    @staticmethod
    def forward(ctx, V, eps, F, D, mu, k0, dirs, pols, options):
        import numpy as np

        from . import FMBEM
        Vn = V.detach().cpu().numpy().astype(np.float64)
        en = [complex(v) for v in eps.detach().cpu().numpy()]
        g = FMBEM(Vn, F, D, en, mu, k0, **options)
        x, _, _, st = g.solve(g.plane_wave_rhs(dirs, pols), tol=1e-10)
        if st != 0:
            raise FMBEMError(st, "forward solve did not converge")
        coef = 4 * np.pi / g.kb.real * np.conj(pols)
        L = g.far_field_functional(dirs, coef)
        cext = g.cross_sections(x, dirs, pols, n_theta=2, n_phi=2)[0]
        ctx.state = (g, x, L, coef, Vn, en, F, D, mu, k0, dirs, pols, options)
        ctx.devices = (V.device, eps.device)
        return torch.as_tensor(np.asarray(cext, dtype=np.float64), device=V.device)

    @staticmethod
    def backward(ctx, go):
        import numpy as np

        from . import FMBEM
        g, x, L, coef, Vn, en, F, D, mu, k0, dirs, pols, options = ctx.state
        lam, _, _, st = g.adjoint_solve(L, tol=1e-10)
        if st != 0:
            raise FMBEMError(st, "adjoint solve did not converge")
        w = go.detach().cpu().numpy().astype(np.float64)  # dLoss/dC_ext[r]
        gV = geps = None
        if ctx.needs_input_grad[0]:
            dV = g.shape_gradient(x, lam, dirs, pols, dirs, coef).imag  # [n_rhs, nv, 3]
            gV = torch.from_numpy(np.einsum("r,rvc->vc", w, dV)).to(ctx.devices[0])
        if ctx.needs_input_grad[1]:
            # eps_0 (the background) is held fixed: it also enters the incident field and the
            # optical theorem's prefactor, which this adjoint does not differentiate, so its entry
            # is NaN rather than a silent zero
            ge = np.zeros(len(en), dtype=np.complex128)
            ge[0] = complex(np.nan, np.nan)
            for j in range(1, len(en)):
                df = -g.eps_sensitivity(j, x, lam)  # d f / d eps_j (holomorphic), fmbem_eps_sensitivity
                # C = Im f: dC/dRe = Im df, dC/dIm = Re df; the complex gradient is dRe + i dIm
                ge[j] = np.sum(w * (df.imag + 1j * df.real))
            geps = torch.from_numpy(ge).to(ctx.devices[1])
        return gV, geps, None, None, None, None, None, None, None


def extinction(V, eps, F, D, mu, k0, dirs, pols, **options):
    """C_ext [n_rhs] (float64 tensor) of the plane waves (dirs[r], pols[r]) on the mesh (V, F, D),
    differentiable in V (float64 tensor [nv, 3], vertex nodes) and eps (complex128 tensor [J+1]):
    one forward and one adjoint GMRES solve serve both gradients.  Under PyTorch's convention the
    gradient of a real loss with respect to eps_j is dL/dRe(eps_j) + i dL/dIm(eps_j).  Only the
    scatterers' permittivities eps[1:] are differentiated: the background eps[0] is held fixed and
    its gradient entry is NaN (slice eps[1:] into a leaf tensor to optimise the scatterers)."""
    import numpy as np
    dirs = np.atleast_2d(np.asarray(dirs, dtype=np.float64))
    pols = np.atleast_2d(np.asarray(pols, dtype=np.complex128))
    return _Extinction.apply(V, eps, F, D, mu, k0, dirs, pols, options)


class _Force(torch.autograd.Function):
    """Maxwell-stress force [3] on the particles inside the sphere (center, radius) in the plane
    wave (d, e) (vacuum background); differentiable in the vertex positions V (fmbem_shape_
    gradient_near) and the permittivities eps (operator central differences), each force
    component's gradient being 2 Re of its Wirtinger functional's (see gradients.py)."""

    @staticmethod
    def forward(ctx, V, eps, F, D, mu, k0, d, e, center, radius, n_theta, n_phi, options):
        import numpy as np

        from . import FMBEM
        from .gradients import _force_adjoint
        Vn = V.detach().cpu().numpy().astype(np.float64)
        en = [complex(v) for v in eps.detach().cpu().numpy()]
        g = FMBEM(Vn, F, D, en, mu, k0, **options)
        x, force, pts, cE, cH, lam = _force_adjoint(g, d, e, center, radius, n_theta, n_phi, 1e-10)
        ctx.state = (g, x, pts, cE, cH, lam, Vn, en, F, D, mu, k0, d, e, options)
        ctx.devices = (V.device, eps.device)
        return torch.as_tensor(np.asarray(force, dtype=np.float64), device=V.device)

    @staticmethod
    def backward(ctx, go):
        import numpy as np

        from . import FMBEM
        g, x, pts, cE, cH, lam, Vn, en, F, D, mu, k0, d, e, options = ctx.state
        w = go.detach().cpu().numpy().astype(np.float64)  # dLoss/dF_i
        gV = geps = None
        if ctx.needs_input_grad[0]:
            x3 = x.expand(3, -1, -1).contiguous()
            out = g.shape_gradient_near(x3, lam, np.repeat(d, 3, 0), np.repeat(e, 3, 0), pts, cE, cH)
            gV = torch.from_numpy(np.einsum("i,ivc->vc", w, 2 * out.real)).to(ctx.devices[0])
        if ctx.needs_input_grad[1]:
            ge = np.zeros(len(en), dtype=np.complex128)
            ge[0] = complex(np.nan, np.nan)  # eps_0 held fixed (see _Extinction.backward)
            x3 = x.expand(3, -1, -1).contiguous()
            for j in range(1, len(en)):
                sv = g.eps_sensitivity(j, x3, lam)  # s_i = lambda_i^T (dA/deps_j) x, fmbem_eps_sensitivity
                ge[j] = np.sum(w * (-2 * sv.real + 1j * 2 * sv.imag))  # dF_i/dRe + i dF_i/dIm
            geps = torch.from_numpy(ge).to(ctx.devices[1])
        return gV, geps, None, None, None, None, None, None, None, None, None, None, None


def force(V, eps, F, D, mu, k0, d, e, center, radius, n_theta=24, n_phi=48, **options):
    """The Maxwell-stress force [3] (float64 tensor) of gradients.force_eps_gradient, differentiable
    in V (float64 tensor [nv, 3], vertex nodes; the stress sphere stays fixed) and eps (complex128
    tensor [J+1]): one forward and three adjoint solves serve both gradients.  As for extinction,
    the background eps[0] is held fixed and its gradient entry is NaN."""
    import numpy as np
    d = np.asarray(d, dtype=np.float64).reshape(1, 3)
    e = np.asarray(e, dtype=np.complex128).reshape(1, 3)
    return _Force.apply(V, eps, F, D, mu, k0, d, e, np.asarray(center, dtype=np.float64), float(radius), n_theta,
                        n_phi, options)
