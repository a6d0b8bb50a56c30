"""torch.autograd.Function around the solver: x = D[U]^-1 b, differentiable
in the links U and the source b.

Backward, for the gradient g of a real loss with respect to x:
  lambda = D^-dag g = gamma5 D^-1 gamma5 g   (qcd_solve_adjoint, same solver)
  dL/db  = lambda
  dL/dU  = gradient of -Re<lambda, D[U] x>   (qcd_force: hopping outer
           products and clover-leaf insertions)
in torch's convention for complex tensors (dL/dRe + i dL/dIm).  Only x is
kept from the forward pass; every step runs in the CUDA library.
"""
from __future__ import annotations

import torch

from . import qcd


class CloverSolve(torch.autograd.Function):
    @staticmethod
    def forward(fctx, U, b, qctx, kappa, csw, tol, levels):
        qctx.gauge_load(U)
        qctx.clover_build(kappa, csw)
        x = torch.empty_like(b)
        info = qctx.solve(b.contiguous(), x, tol=tol, precision_levels=levels)
        fctx.qctx, fctx.kappa, fctx.csw, fctx.tol, fctx.levels = qctx, kappa, csw, tol, levels
        fctx.info = info
        fctx.save_for_backward(U, x)
        return x

    @staticmethod
    def backward(fctx, g):
        U, x = fctx.saved_tensors
        qctx = fctx.qctx
        # the context must hold this U's fields (another forward may have
        # loaded different links in between)
        if getattr(qctx, "_loaded_tag", None) != _tag(U, fctx.kappa, fctx.csw):
            qctx.gauge_load(U)
            qctx.clover_build(fctx.kappa, fctx.csw)
            qctx._loaded_tag = _tag(U, fctx.kappa, fctx.csw)
        g = g.contiguous()
        lam = torch.empty_like(g)
        qctx.solve_adjoint(g, lam, tol=fctx.tol, precision_levels=fctx.levels)
        grad_U = None
        if fctx.needs_input_grad[0]:
            grad_U = torch.empty_like(U)
            qctx.force(U, x, lam, grad_U)
        grad_b = lam if fctx.needs_input_grad[1] else None
        return grad_U, grad_b, None, None, None, None, None


def clover_solve(U: torch.Tensor, b: torch.Tensor, qctx: "qcd.Context", kappa: float, csw: float,
                 tol: float = 1e-12, levels: int = 2) -> torch.Tensor:
    """x = D[U]^-1 b on qctx's lattice (U [V,4,3,3], b [V,4,3], complex128 on
    the GPU), differentiable in U and b."""
    x = CloverSolve.apply(U, b, qctx, kappa, csw, tol, levels)
    qctx._loaded_tag = _tag(U, kappa, csw)
    return x


def _tag(U, kappa, csw):
    return (U.data_ptr(), U._version, float(kappa), float(csw))
