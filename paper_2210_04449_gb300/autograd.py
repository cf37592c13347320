"""torch.autograd wrapper of the Sec. 2.3 soft-shadow march and its
hand-written adjoint (``rtsdf_shadow`` / ``rtsdf_shadow_backward``)."""
from __future__ import annotations

import torch


class ShadowFn(torch.autograd.Function):
    """vis = shadow(sdf, light); gradients w.r.t. the fine SDF texels and the
    (unnormalised) light direction.  The backward pass re-runs the march in
    the kernel instead of storing it."""

    @staticmethod
    def forward(ctx, sdf, light, pos, nrm, rt, k, steps, step_max_vox, eps_vox):
        vis = rt.shadow(pos, nrm, light, k=k, steps=steps, step_max_vox=step_max_vox, eps_vox=eps_vox,
                        sdf=sdf.detach())
        ctx.save_for_backward(sdf, light, pos, nrm)
        ctx.rt = rt
        ctx.params = (k, steps, step_max_vox, eps_vox)
        return vis

    @staticmethod
    def backward(ctx, gvis):
        sdf, light, pos, nrm = ctx.saved_tensors
        k, steps, smax, eps = ctx.params
        dsdf = torch.zeros_like(sdf, dtype=torch.float32)
        dlight = torch.zeros(3, device=sdf.device, dtype=torch.float32)
        ctx.rt.shadow_backward(pos, nrm, light, gvis.float(), dsdf, dlight, k=k, steps=steps, step_max_vox=smax,
                               eps_vox=eps, sdf=sdf.detach())
        return dsdf.to(sdf.dtype), dlight.to(light.device, light.dtype).reshape(light.shape), None, None, None, \
            None, None, None, None


def soft_shadow(rt, sdf, light, pos, nrm, k=8.0, steps=64, step_max_vox=4.0, eps_vox=1.0):
    """Differentiable visibility of shading points ``pos``/``nrm`` (float32
    [..., 3] on the GPU) for the fine SDF ``sdf`` (float32 [(2N)^3])."""
    return ShadowFn.apply(sdf, light, pos, nrm, rt, k, steps, step_max_vox, eps_vox)
