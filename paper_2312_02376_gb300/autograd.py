"""torch.autograd wrapper of the FFT-PIM apply.

    u = PimApply.apply(q, xyz, plan)

forward: pim_apply (the positions are moved into the plan with
pim_update_positions, i.e. with the discrete structure of the plan's last
pim_set_points kept); backward: grad_q = A^H grad_u (pim_apply_adjoint) and
grad_xyz = Re sum conj(grad_u) dA/dxyz q (pim_position_grad), PyTorch's
convention for complex outputs.  All compute runs in libpim.
"""
import torch


class PimApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, xyz, plan):
        if xyz is not None:
            plan.update_positions(xyz.detach().contiguous())
        q = q.contiguous()
        u = plan.apply(q)
        ctx.plan = plan
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
            gx = plan.position_grad(q, grad_u)
        return gq, gx, None


def pim_apply(q, xyz, plan):
    """u = A(xyz) q with autograd through q and xyz."""
    return PimApply.apply(q, xyz, plan)
