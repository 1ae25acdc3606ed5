"""torch.autograd front of the differentiable render path (Sec. 3.2: volume
rendering is differentiable, so the canonical field, the skinning weights and
the bone transforms are trained through it).

``render_rays(field, origin, direction, pose)`` returns the colour and opacity
of a batch of world-space rays as differentiable functions of the hash table
and the packed MLP (and, as gradient sinks, of the context's skinning-weight
grid and per-pose bone transforms).  Any loss the caller builds on them in
torch can be back-propagated:

* forward = ``ia_train_forward``: march, correspondence search, hash encoding,
  MLP and compositing in the library's kernels; the per-sample state (roots,
  density, colour) stays in the library context, activations are not stored;
* backward = ``ia_train_backward`` with the incoming dL/drgb and dL/dalpha:
  the reverse compositing sweep, the recomputed MLP and its backward, the
  hash-table scatter-add and the implicit-function gradient through the root
  (lambda = J(x*)^-T dL/dx*) to the skinning grid and the bone transforms.

The table and MLP tensors are read in place by the forward (nothing is copied
into the context) and must not change until the backward has run.  The
skinning grid and the bone transforms are the context's (set by
ia_set_skeleton / ia_adam_step and ia_set_pose); ``skin`` and ``bones`` are
tensors of their shapes that receive their gradients (their values are not
read).  One forward is kept per context: backward must come before the next
forward on the same context, which the Function checks.
"""
from __future__ import annotations

import torch

from . import (IA_OCC_UNION, IAError, ia_grad_sizes, ia_param_sizes, ia_train_backward,
               ia_train_forward)


class Field:
    """A library context used for differentiable rendering, with the count of
    forwards run on it (a backward must belong to the latest forward)."""

    def __init__(self, ctx, occ_grid=IA_OCC_UNION):
        self.ctx = ctx
        self.occ_grid = occ_grid
        self.forwards = 0
        self.table_floats, self.mlp_floats = ia_param_sizes(ctx)
        self.skin_floats, self.bone_floats = ia_grad_sizes(ctx)


class RenderRays(torch.autograd.Function):
    """rgb [n,3], alpha [n] = RenderRays.apply(field, table, mlp, skin, bones, origin, direction, pose)"""

    @staticmethod
    def forward(fctx, field, table, mlp, skin, bones, origin, direction, pose):
        if table.numel() != field.table_floats or mlp.numel() != field.mlp_floats:
            raise ValueError(f"table / mlp must hold {field.table_floats} / {field.mlp_floats} floats")
        if skin.numel() != field.skin_floats or bones.numel() != field.bone_floats:
            raise ValueError(f"skin / bones must hold {field.skin_floats} / {field.bone_floats} floats")
        n = pose.shape[0]
        dev = table.device
        rgb = torch.empty(n, 3, device=dev)
        alpha = torch.empty(n, device=dev)
        table_c, mlp_c = table.detach().contiguous(), mlp.detach().contiguous()
        ia_train_forward(field.ctx, origin, direction, pose, rgb, alpha, table=table_c, mlp=mlp_c,
                         occ_grid=field.occ_grid)
        field.forwards += 1
        fctx.field = field
        fctx.token = field.forwards
        fctx.keep = (table_c, mlp_c)  # read again by the backward
        fctx.shapes = (table.shape, mlp.shape, skin.shape, bones.shape)
        return rgb, alpha

    @staticmethod
    def backward(fctx, grad_rgb, grad_alpha):
        field = fctx.field
        if fctx.token != field.forwards:
            raise IAError(2, "RenderRays.backward: another forward ran on this context since this one")
        dev = grad_rgb.device
        g = {"table": torch.empty(field.table_floats, device=dev), "mlp": torch.empty(field.mlp_floats, device=dev),
             "skin": torch.empty(field.skin_floats, device=dev), "bones": torch.empty(field.bone_floats, device=dev)}
        ga = grad_alpha.contiguous() if grad_alpha is not None else None
        ia_train_backward(field.ctx, grad_rgb.contiguous(), g, grad_alpha=ga)
        ts, ms, ss, bs = fctx.shapes
        return (None, g["table"].view(ts), g["mlp"].view(ms), g["skin"].view(ss), g["bones"].view(bs),
                None, None, None)


def render_rays(field, table, mlp, skin, bones, origin, direction, pose):
    """Differentiable colour and opacity of a ray batch (see RenderRays)."""
    return RenderRays.apply(field, table, mlp, skin, bones, origin, direction, pose)
