"""torch.autograd wrapper of the FFT-PIM apply.

    u = PimApply.apply(q, xyz, plan)

forward: pim_apply (the positions are moved into the plan with
pim_update_positions, i.e. with the discrete structure of the plan's last
pim_set_points kept); backward: grad_q = A^H grad_u (pim_apply_adjoint) and
grad_xyz = Re sum conj(grad_u) dA/dxyz q (pim_position_grad), PyTorch's
convention for complex outputs.  When the forward apply is still the plan's
last one, the position gradient reuses the grid potentials of that apply and
of the adjoint apply just made (pim_position_grad_reuse).  All compute runs in
libpim.
"""
import torch

from .pim import PimError


class PimApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, xyz, plan):
        if xyz is not None:
            plan.update_positions(xyz.detach().contiguous())
        q = q.contiguous()
        u = plan.apply(q)
        ctx.plan = plan
        ctx.forward_seq = getattr(plan, "forward_applies", 0)
        ctx.save_for_backward(q)
        ctx.has_xyz = xyz is not None
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (q,) = ctx.saved_tensors
        plan = ctx.plan
        grad_u = grad_u.contiguous()
        gq = gx = None
        if ctx.needs_input_grad[0]:
            gq = plan.apply_adjoint(grad_u)
        if ctx.has_xyz and ctx.needs_input_grad[1]:
            same = getattr(plan, "forward_applies", 0) == ctx.forward_seq and q.ndim == 1
            if gq is not None and same:
                try:
                    gx = plan.position_grad_reuse(q, grad_u)
                except PimError:
                    gx = None
            if gx is None:
                gx = plan.position_grad(q, grad_u)
        return gq, gx, None


def pim_apply(q, xyz, plan):
    """u = A(xyz) q with autograd through q and xyz."""
    return PimApply.apply(q, xyz, plan)
