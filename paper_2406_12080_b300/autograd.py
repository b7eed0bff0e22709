"""torch.autograd.Function over the library's render and its hand-written adjoint.

Hierarchy optimisation (Sec. 5.1 of the paper) renders random views at random target
granularities tau and back-propagates into the interior nodes through the interpolation between
a cut node and its parent.  The forward pass is `h3dgs_select_cut` + `h3dgs_render(save=1)`; the
backward pass is `h3dgs_render_backward`.  Activations stay in torch (Sec. 7.3): scales are
exp(raw), leaf opacities sigmoid(raw), interior opacities |raw| (the falloff may exceed 1);
leaves can be frozen (stop-gradient).

One H3dgsRender.apply per context at a time: the backward reads the state saved by the most
recent forward on that context.
"""
from __future__ import annotations

import numpy as np
import torch

from . import h3dgs

ATTRS = ("mean", "scale", "rot", "opacity", "sh")


class H3dgsRender(torch.autograd.Function):
    """images = render(mean, scale, rot, opacity, sh) for a batch of cameras.

    Inputs are ACTIVATED attributes ([N,3], [N,3], [N,4], [N], [N,48] fp32 CUDA tensors, contiguous);
    `topology` is a DeviceHierarchy supplying boxes, parent and child arrays (its attribute tensors
    are ignored).  Returns the packed images (sum of 3 H W floats over the cameras).
    """

    @staticmethod
    def forward(fctx, mean, scale, rot, opacity, sh, context: h3dgs.Context, topology: h3dgs.DeviceHierarchy,
                cams, opts, freeze_leaves: bool, capacity):
        attrs = [t.contiguous() for t in (mean, scale, rot, opacity, sh)]
        hier = h3dgs.DeviceHierarchy(*attrs, topology.box_min, topology.box_max, topology.parent,
                                     topology.child_start, topology.child_count)
        context.upload(hier)
        cut = context.select_cut(cams, capacity)
        images = context.render(cams, cut, opts, save_for_backward=1)
        fctx.context = context
        fctx.hier = hier
        fctx.cut = cut                      # the backward re-reads the cut buffers
        fctx.freeze = int(bool(freeze_leaves))
        return images

    @staticmethod
    def backward(fctx, dimages):
        hier = fctx.hier
        grads = {k: torch.zeros_like(getattr(hier, k)) for k in ATTRS}
        h3dgs.h3dgs_render_backward(fctx.context.ctx, dimages.contiguous(), grads, fctx.freeze)
        return (grads["mean"], grads["scale"], grads["rot"], grads["opacity"], grads["sh"],
                None, None, None, None, None, None)


class H3dgsRenderDepth(torch.autograd.Function):
    """(images, depth) = render with the expected-depth output and optional per-camera exposure
    affines (the appendix's depth regularisation and exposure compensation).  `exposure`: device
    tensor [n_cams, 3, 4] or None; it is held fixed (no gradient), as in hierarchy optimisation."""

    @staticmethod
    def forward(fctx, mean, scale, rot, opacity, sh, context: h3dgs.Context, topology: h3dgs.DeviceHierarchy,
                cams, opts, freeze_leaves: bool, capacity, exposure):
        attrs = [t.contiguous() for t in (mean, scale, rot, opacity, sh)]
        hier = h3dgs.DeviceHierarchy(*attrs, topology.box_min, topology.box_max, topology.parent,
                                     topology.child_start, topology.child_count)
        context.upload(hier)
        cut = context.select_cut(cams, capacity)
        images, depth = context.render(cams, cut, opts, save_for_backward=1, depth=True,
                                       exposure=None if exposure is None else exposure.contiguous())
        fctx.context = context
        fctx.hier = hier
        fctx.cut = cut
        fctx.freeze = int(bool(freeze_leaves))
        return images, depth

    @staticmethod
    def backward(fctx, dimages, ddepth):
        hier = fctx.hier
        grads = {k: torch.zeros_like(getattr(hier, k)) for k in ATTRS}
        dimages = torch.zeros_like(ddepth).repeat(3) if dimages is None else dimages.contiguous()
        h3dgs.h3dgs_render_backward_ex(fctx.context.ctx, dimages, None if ddepth is None else ddepth.contiguous(),
                                       grads, fctx.freeze)
        return (grads["mean"], grads["scale"], grads["rot"], grads["opacity"], grads["sh"],
                None, None, None, None, None, None, None)


def render_depth(context, topology, mean, scale, rot, opacity, sh, cams, opts=None, freeze_leaves=True,
                 capacity=None, exposure=None):
    opts = opts or h3dgs.default_opts()
    return H3dgsRenderDepth.apply(mean, scale, rot, opacity, sh, context, topology, cams, opts, freeze_leaves,
                                  capacity, exposure)


def render(context, topology, mean, scale, rot, opacity, sh, cams, opts=None, freeze_leaves=True, capacity=None):
    opts = opts or h3dgs.default_opts()
    return H3dgsRender.apply(mean, scale, rot, opacity, sh, context, topology, cams, opts, freeze_leaves, capacity)


class HierarchyParams(torch.nn.Module):
    """Raw (pre-activation) node parameters with the activations used for hierarchy optimisation."""

    def __init__(self, hier: h3dgs.DeviceHierarchy):
        super().__init__()
        leaf = hier.child_count == 0
        self.register_buffer("leaf", leaf)
        self.mean = torch.nn.Parameter(hier.mean.clone())
        self.log_scale = torch.nn.Parameter(torch.log(hier.scale.clamp_min(1e-12)))
        self.rot = torch.nn.Parameter(hier.rot.clone())
        op = hier.opacity.clamp(1e-6, None)
        logit = torch.log(op.clamp(max=1 - 1e-6) / (1 - op.clamp(max=1 - 1e-6)))
        self.opacity_raw = torch.nn.Parameter(torch.where(leaf, logit, op))
        self.sh = torch.nn.Parameter(hier.sh.clone())

    def activated(self):
        op = torch.where(self.leaf, torch.sigmoid(self.opacity_raw), self.opacity_raw.abs())
        return self.mean, torch.exp(self.log_scale), self.rot, op, self.sh


def sample_tau(tau_min: float, tau_max: float, xi: float) -> float:
    """Target granularity for one optimisation step: tau = tau_max^xi tau_min^(1 - xi) (Sec. 5.1)."""
    return float(tau_max ** xi * tau_min ** (1.0 - xi))


def l1_step(params: HierarchyParams, context, topology, cams, targets, optimizer, opts=None, capacity=None,
            freeze_leaves: bool = True):
    """One hierarchy-optimisation step (Sec. 5.1): render the views at their own tau, mean L1 against the
    target images (packed like the render's output), back-propagate through the adjoint, step."""
    optimizer.zero_grad(set_to_none=True)
    images = render(context, topology, *params.activated(), cams, opts, freeze_leaves=freeze_leaves,
                    capacity=capacity)
    loss = (images - targets).abs().mean()
    loss.backward()
    optimizer.step()
    return loss.detach()
