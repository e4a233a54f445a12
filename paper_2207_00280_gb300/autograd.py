"""torch.autograd.Functions over the library's matrix-free kernels.

IgaBilinear: J(kappa, u, v) = u^T K(kappa) v.  The forward asks the adjoint
kernel (iga_integrate_backward) for J only; the backward recomputes
g = dJ/dkappa from the basis tables (no element matrix and no g is stored
between the two) and, when u or v need gradients, applies the operator:
dJ/du = K(kappa) v and dJ/dv = K(kappa)^T u = K(kappa) u (iga_apply).

IgaApply: y = alpha K(kappa) x + beta M(rho) x.  Both operators are symmetric,
so dL/dx = alpha K g_y + beta M g_y (one more iga_apply), and since y is linear
in kappa, dL/dkappa_q = alpha * (dJ/dkappa_q of J = g_y^T K(kappa) x), the
adjoint kernel with u = g_y, v = x.  rho is not differentiated.

IgaIntegrate: (K_e, M_e) = element matrices of every element (iga_integrate).
Both are linear in the coefficients, so the backward maps the upstream
gradients dL/dK_e and dL/dM_e to dL/dkappa and dL/drho at every quadrature
point with one call of the reverse sum-factorization kernel
(iga_integrate_grad); nothing is saved between the two passes.
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
        plan, jac = ctx.plan, ctx.jac
        gk = gu = gv = None
        kc = kappa.detach().contiguous()
        if ctx.needs_input_grad[0]:
            g = torch.empty(kappa.numel(), dtype=u.dtype, device=kappa.device)
            plan.backward(kc, u.detach().contiguous(), v.detach().contiguous(), grad=g, J=None,
                          jac=jac)
            gk = gJ * g.to(torch.float64).view_as(kappa)
        if ctx.needs_input_grad[1]:
            gu = gJ.to(u.dtype) * plan.apply(v.detach().contiguous(), kappa=kc, jac=jac)
        if ctx.needs_input_grad[2]:
            gv = gJ.to(v.dtype) * plan.apply(u.detach().contiguous(), kappa=kc, jac=jac)
        return gk, gu, gv, None, None


def iga_bilinear(kappa, u, v, plan, jac=None):
    """J = u^T K(kappa) v, differentiable with respect to kappa, u and v."""
    return IgaBilinear.apply(kappa, u, v, plan, jac)


class IgaApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kappa, x, plan, alpha=1.0, beta=0.0, rho=None, jac=None):
        if kappa is not None and kappa.dtype != torch.float64:
            raise TypeError("kappa must be float64 (one value per quadrature point)")
        kc = kappa.contiguous() if kappa is not None else None
        y = plan.apply(x.contiguous(), kappa=kc, rho=rho, jac=jac, alpha=alpha, beta=beta)
        ctx.save_for_backward(kappa, x)
        ctx.plan, ctx.alpha, ctx.beta, ctx.rho, ctx.jac = plan, alpha, beta, rho, jac
        return y

    @staticmethod
    def backward(ctx, gy):
        kappa, x = ctx.saved_tensors
        plan = ctx.plan
        gy = gy.contiguous().to(x.dtype)
        kc = kappa.detach().contiguous() if kappa is not None else None
        gk = gx = None
        if ctx.needs_input_grad[1]:
            gx = plan.apply(gy, kappa=kc, rho=ctx.rho, jac=ctx.jac, alpha=ctx.alpha, beta=ctx.beta)
        if ctx.needs_input_grad[0] and kappa is not None:
            g = torch.empty(kappa.numel(), dtype=x.dtype, device=x.device)
            plan.backward(kc, gy, x.detach().contiguous(), grad=g, J=None, jac=ctx.jac)
            gk = ctx.alpha * g.to(torch.float64).view_as(kappa)
        return gk, gx, None, None, None, None, None


def iga_apply(kappa, x, plan, alpha=1.0, beta=0.0, rho=None, jac=None):
    """y = alpha K(kappa) x + beta M(rho) x, differentiable with respect to kappa and x."""
    return IgaApply.apply(kappa, x, plan, alpha, beta, rho, jac)


class IgaIntegrate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kappa, rho, plan, jac=None):
        for name, c in (("kappa", kappa), ("rho", rho)):
            if c is not None and c.dtype != torch.float64:
                raise TypeError(f"{name} must be float64 (one value per quadrature point)")
        K, M, _ = plan.empty_outputs(device="cuda", dof=False)
        plan.integrate(kappa=kappa.contiguous() if kappa is not None else None,
                       rho=rho.contiguous() if rho is not None else None, jac=jac, K=K, M=M)
        ctx.plan, ctx.jac = plan, jac
        ctx.has = (kappa is not None, rho is not None)
        return K, M

    @staticmethod
    def backward(ctx, gK, gM):
        plan = ctx.plan
        want_k = ctx.needs_input_grad[0] and gK is not None
        want_r = ctx.needs_input_grad[1] and gM is not None
        gk = gr = None
        if want_k or want_r:
            dt = plan.out_dtype
            GK = gK.contiguous().to(dt) if want_k else None
            GM = gM.contiguous().to(dt) if want_r else None
            g1, g2 = plan.integrate_grad(GK=GK, GM=GM, jac=ctx.jac)
            gk = g1.to(torch.float64) if want_k else None
            gr = g2.to(torch.float64) if want_r else None
        return gk, gr, None, None


def iga_integrate(plan, kappa=None, rho=None, jac=None):
    """(K, M) element matrices (None where the plan skips one), differentiable
    with respect to kappa and rho."""
    return IgaIntegrate.apply(kappa, rho, plan, jac)
