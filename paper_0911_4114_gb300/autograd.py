"""torch.autograd.Function over the C-ABI apply: phi = A(y) q.

Backward: dL/dq = A^H g (hfmm_apply_adjoint) and dL/dy from hfmm_grad_sources, with
g = dL/d conj(phi) as complex autograd supplies it.  The plan (tree, quadratures) is
fixed at the positions it was built from; `y` must hold those positions.
"""
import torch


class FmmApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, y, plan):
        ctx.plan = plan
        ctx.save_for_backward(q)
        ctx.y_dtype = y.dtype
        return plan.apply(q)

    @staticmethod
    def backward(ctx, g):
        (q,) = ctx.saved_tensors
        plan = ctx.plan
        g = g.contiguous()
        gq = plan.apply_adjoint(g) if ctx.needs_input_grad[0] else None
        gy = None
        if ctx.needs_input_grad[1]:
            gy = plan.grad_sources(q, g).to(ctx.y_dtype)
        return gq, gy, None


def fmm_apply(q, y, plan):
    """phi = A(y) q with gradients for q (adjoint FMM) and y (position gradient)."""
    return FmmApply.apply(q, y, plan)
