"""torch.autograd.Function for J(kappa) = u^T K(kappa) v.

Forward and backward both call the library's matrix-free adjoint
(iga_integrate_backward): the forward asks for J only, the backward recomputes
g = dJ/dkappa from the basis tables (no element matrix and no g is stored
between the two; only kappa, u, v and the plan are kept).  Gradients with
respect to u and v are not provided (they would be K v and K^T u).
"""
from __future__ import annotations

import torch


class IgaBilinear(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kappa, u, v, plan, jac=None):
        if kappa.dtype != torch.float64:
            raise TypeError("kappa must be float64 (one value per quadrature point)")
        J = torch.empty(1, dtype=torch.float64, device=kappa.device)
        plan.backward(kappa.contiguous(), u.contiguous(), v.contiguous(), grad=None, J=J, jac=jac)
        ctx.save_for_backward(kappa, u, v)
        ctx.plan = plan
        ctx.jac = jac
        return J[0]

    @staticmethod
    def backward(ctx, gJ):
        kappa, u, v = ctx.saved_tensors
        g = torch.empty(kappa.numel(), dtype=u.dtype, device=kappa.device)
        ctx.plan.backward(kappa.contiguous(), u.contiguous(), v.contiguous(), grad=g, J=None,
                          jac=ctx.jac)
        return gJ * g.to(torch.float64).view_as(kappa), None, None, None, None


def iga_bilinear(kappa, u, v, plan, jac=None):
    """J = u^T K(kappa) v, differentiable with respect to kappa."""
    return IgaBilinear.apply(kappa, u, v, plan, jac)
