"""torch.autograd bridge for the Helmholtz operator with coefficient fields.

y = H(lambda, kappa) u per element (FP64).  Backward, for an upstream
gradient g = dL/dy:
    dL/du      = H(lambda, kappa) g          (H is symmetric)
    dL/dlambda = JW (B g)(B u)   at every quadrature point
    dL/dkappa  = sum_ab G_ab (d_a g)(d_b u)
the last two from the adjoint kernel, which recomputes B u and grad u: the
forward pass stores only its inputs.
"""
import torch

from . import binding


class HelmholtzFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, lam_field, kappa_field, plan):
        if u.dtype != torch.float64:
            raise TypeError("HelmholtzFn works in FP64")
        ctx.plan = plan
        ctx.save_for_backward(u, lam_field, kappa_field)
        return binding.helmholtz(plan, u, lam_field=lam_field, kappa_field=kappa_field)

    @staticmethod
    def backward(ctx, g):
        u, lam, kap = ctx.saved_tensors
        plan = ctx.plan
        g = g.contiguous()
        gu = binding.helmholtz(plan, g, lam_field=lam, kappa_field=kap) if ctx.needs_input_grad[0] else None
        want_l, want_k = ctx.needs_input_grad[1], ctx.needs_input_grad[2]
        gl = gk = None
        if want_l or want_k:
            gl, gk = binding.helmholtz_adjoint(plan, u, g, want_lambda=want_l, want_kappa=want_k)
        return gu, gl, gk, None


def helmholtz_ad(plan, u, lam_field, kappa_field):
    """Differentiable H(lambda, kappa) u (fields are per-quadrature-point FP64 tensors)."""
    return HelmholtzFn.apply(u, lam_field, kappa_field, plan)
