"""Differentiable wrappers of the FMM-BEM product and solve for torch.autograd.

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
