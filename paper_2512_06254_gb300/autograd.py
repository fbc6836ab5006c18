"""Differentiable snapshot imaging for PyTorch.

image_snapshot(plan, uvw, freq, vis, ...) returns the standard-plane image of
one snapshot (toi_grid + toi_image) as a tensor that autograd can
differentiate with respect to the visibilities and the weights; the reverse
pass is toi_degrid_backward (the adjoint of the imaging map, Section 1 of the
paper).  The plane fit is held fixed (piecewise constant in the weights).
Gradients of point-source or other sky models follow by ordinary autograd
through the code that produces `vis`.
"""
from __future__ import annotations

import torch


class _ImageSnapshot(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vis, weight, plan, uvw, freq, flag, slot):
        if vis.dtype != torch.complex64:
            raise TypeError("differentiable imaging takes complex64 visibilities")
        plan.grid(uvw, freq, vis.detach(), flag=flag,
                  weight=None if weight is None else weight.detach(), slot=slot)
        img = torch.empty(plan.N, plan.N, dtype=torch.float32, device=vis.device)
        plan.image(slot, img)
        ctx.plan, ctx.slot = plan, slot
        ctx.generation = plan.slot_generation(slot)
        ctx.save_for_backward(vis, weight, img, uvw, freq, flag)
        return img

    @staticmethod
    def backward(ctx, grad_img):
        vis, weight, img, uvw, freq, flag = ctx.saved_tensors
        plan, slot = ctx.plan, ctx.slot
        if plan.slot_generation(slot) != ctx.generation:
            raise RuntimeError("the grid slot was used by another toi_grid call before backward; "
                               "use one slot per live differentiable image")
        need_vis, need_w = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        gv = torch.empty_like(vis) if need_vis else None
        gw = torch.empty_like(weight) if (need_w and weight is not None) else None
        if gv is None and gw is None:
            return (None,) * 7
        plan.degrid_backward(grad_img.contiguous(), image=img if gw is not None else None,
                             grad_vis=gv, grad_weight=gw, slot=slot)
        return gv, gw, None, None, None, None, None


def image_snapshot(plan, uvw, freq, vis, flag=None, weight=None, slot: int = 0):
    """Standard-plane image [N, N] of one snapshot, differentiable with
    respect to vis (complex64 [n_bl, n_ch, n_pol]) and weight (float32, same
    shape, or None for unit weights)."""
    return _ImageSnapshot.apply(vis, weight, plan, uvw, freq, flag, slot)


class _Localise(torch.autograd.Function):
    @staticmethod
    def forward(ctx, src, weight, plan, win, slot):
        n = win.shape[0]
        dev = src.device
        loss = torch.empty(n, dtype=torch.float64, device=dev)
        need_src, need_w = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        gsrc = torch.empty(n, 3, dtype=torch.float64, device=dev) if need_src else None
        gw = torch.empty_like(weight) if (need_w and weight is not None) else None
        plan.localise(win, src.detach().contiguous(), loss=loss, grad_src=gsrc, grad_weight=gw,
                      slot=slot)
        ctx.save_for_backward(gsrc, gw)
        return loss.sum()

    @staticmethod
    def backward(ctx, g):
        gsrc, gw = ctx.saved_tensors
        return (None if gsrc is None else g * gsrc, None if gw is None else g * gw.to(g.dtype),
                None, None, None)


def localise_loss(plan, win, src, weight=None, slot: int = 0):
    """Sum over the windows of the squared residual between the snapshot's
    tilted image and a point-source model (toi_localise), differentiable with
    respect to src (float64 [n_win, 3]: l, m, S) and weight (the float32
    weight tensor given to toi_grid for this slot, or None).  The gradients
    are computed with the loss by the same call.  With weight requiring grad
    the plan's tilted image is used as workspace (one call per image)."""
    return _Localise.apply(src, weight, plan, win, slot)
