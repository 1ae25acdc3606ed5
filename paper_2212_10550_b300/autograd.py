"""torch.autograd front of the training step (Sec. 3.2, Eq. 8 loss path).

One ia_train_step call runs the forward and the hand-written backward of the
whole path (compositing, MLP, hash-table scatter-add, implicit-function
gradient through the root), so the Function's forward already holds every
gradient; its backward only scales them by the incoming gradient of the loss.
The differentiable inputs are the hash table and the packed MLP, which the
forward installs in the library context (ia_set_params) before the step; the
same step's skinning-grid and bone-transform gradients are returned as
non-differentiable outputs (they belong to the context's skeleton and poses,
which are not torch tensors of the caller).
"""
from __future__ import annotations

import torch

from . import IA_OCC_UNION, ia_grad_sizes, ia_param_sizes, ia_set_params, ia_train_step


class TrainStep(torch.autograd.Function):
    """loss, rgb, skin_grad, bone_grad = TrainStep.apply(table, mlp, ctx, origin, direction, pose, target, occ_grid)

    table [entries * F], mlp (packed): fp32 CUDA tensors, the parameters the
    step differentiates; ctx: a library context with skeleton, poses and an
    occupancy grid; rays: CUDA tensors as ia_train_step takes them."""

    @staticmethod
    def forward(fctx, table, mlp, ctx, origin, direction, pose, target, occ_grid=IA_OCC_UNION):
        nt, nm = ia_param_sizes(ctx)
        if table.numel() != nt or mlp.numel() != nm:
            raise ValueError(f"table / mlp must hold {nt} / {nm} floats")
        ia_set_params(ctx, table.detach().contiguous(), mlp.detach().contiguous())
        dev = table.device
        n_skin, n_bones = ia_grad_sizes(ctx)
        g = {"table": torch.empty(nt, device=dev), "mlp": torch.empty(nm, device=dev),
             "skin": torch.empty(n_skin, device=dev), "bones": torch.empty(n_bones, device=dev)}
        loss = torch.zeros(1, device=dev)
        rgb = torch.empty(pose.shape[0], 3, device=dev)
        ia_train_step(ctx, origin, direction, pose, target, loss, g, occ_grid=occ_grid, rgb_out=rgb)
        fctx.save_for_backward(g["table"], g["mlp"])
        fctx.mark_non_differentiable(rgb, g["skin"], g["bones"])
        return loss[0], rgb, g["skin"], g["bones"]

    @staticmethod
    def backward(fctx, grad_loss, grad_rgb, grad_skin, grad_bones):
        g_table, g_mlp = fctx.saved_tensors
        return grad_loss * g_table, grad_loss * g_mlp, None, None, None, None, None, None


def train_loss(table, mlp, ctx, origin, direction, pose, target, occ_grid=IA_OCC_UNION):
    """The L2 photometric loss of a ray batch as a differentiable function of
    the hash table and the MLP (see TrainStep)."""
    return TrainStep.apply(table, mlp, ctx, origin, direction, pose, target, occ_grid)
