"""torch.autograd.Function wrappers: differentiable light-traced images.

``render(scene, albedo, Le, heights, method=..., ...)`` returns the light-traced image
I(theta) [H, W, 3]; ``I.backward(dI)`` (or any loss built on I) produces gradients of
albedo, Le and heights through liblt's constant-memory adjoints (LRB-3-pass or ResLRB) or
the naive baseline.  The forward pass refits the height field, then runs the primal kernel
of the chosen method; the backward pass refits the height field to the heights its forward
pass saw (another render of the same scene may have moved it in between) and replays the
same paths (same seed and path range).  The scene is left refitted to those heights.
Methods: "lrb3" (LRB-3-pass), "reslrb" (ResLRB), "naive" (tape AD), "lrb2" (buffered
two-pass).
All work runs in liblt's CUDA kernels.
"""
from __future__ import annotations

import torch

from . import lt

METHODS = ("lrb3", "reslrb", "naive", "lrb2")


class _LightTrace(torch.autograd.Function):
    @staticmethod
    def forward(ctx, scene, opts_kw, method, albedo, Le, heights):
        if method not in METHODS:
            raise ValueError(f"method must be one of {METHODS}")
        if scene.n_heights:
            scene.refit(heights.detach())
        aux = None
        if method == "lrb3":
            # LRB-3 state: the primal stores the validity masks, the backward reuses them
            aux = scene.new_lrb3_state(opts_kw["n_paths"])
            o = scene.opts(**opts_kw, lrb3_state=aux)
        else:
            o = scene.opts(**opts_kw)
        if method == "reslrb":
            aux = torch.empty((o.n_paths, 8), device=scene.device, dtype=torch.float32)
            est = lt.EST_RESLRB
        elif method == "naive":
            aux = torch.empty(scene.naive_workspace_bytes(o), device=scene.device, dtype=torch.uint8)
            est = lt.EST_NAIVE
        elif method == "lrb2":
            aux = torch.empty(scene.lrb2_buffer_bytes(o), device=scene.device, dtype=torch.uint8)
            est = lt.EST_BUFFERED
        else:
            est = lt.EST_PLAIN
        img = scene.primal(o, estimator=est, aux=None if method == "lrb3" else aux, albedo=albedo.detach(),
                           Le=Le.detach())
        ctx.scene, ctx.opts_kw, ctx.method, ctx.aux = scene, opts_kw, method, aux
        ctx.save_for_backward(albedo, Le, heights)
        return img

    @staticmethod
    def backward(ctx, grad_image):
        albedo, Le, heights = ctx.saved_tensors
        S = ctx.scene
        if S.n_heights:
            # the attached adjoints replay the paths against the scene's current geometry:
            # restore the geometry of this render's forward pass
            S.refit(heights.detach())
        if ctx.method == "lrb3":
            o = S.opts(**ctx.opts_kw, lrb3_state=ctx.aux, lrb3_mask_ready=1)
        else:
            o = S.opts(**ctx.opts_kw)
        gI = grad_image.contiguous().float()
        kw = dict(albedo=albedo.detach(), Le=Le.detach())
        if ctx.method == "lrb3":
            gA, gL, gH = S.backward_lrb3(o, gI, **kw)
        elif ctx.method == "reslrb":
            gA, gL, gH = S.backward_reslrb(o, gI, ctx.aux, **kw)
        elif ctx.method == "lrb2":
            gA, gL, gH = S.backward_lrb2(o, gI, ctx.aux, **kw)
        else:
            gA, gL, gH = S.backward_naive(o, gI, ctx.aux, **kw)
        ctx.aux = None
        gA = gA[: albedo.numel()].view_as(albedo) if ctx.needs_input_grad[3] else None
        gL = gL.view_as(Le) if ctx.needs_input_grad[4] else None
        gH = gH[: heights.numel()].view_as(heights) if ctx.needs_input_grad[5] else None
        return None, None, None, gA, gL, gH


def render(scene: "lt.Scene", albedo: torch.Tensor, Le: torch.Tensor, heights: torch.Tensor, method: str = "lrb3",
           seed: int = 0, n_paths: int = 1 << 16, max_depth: int = 4, attached: bool = True, **opts):
    """Differentiable light-traced image [H, W, 3] of `scene` at parameters (albedo, Le,
    heights).  Gradients flow to whichever of them require grad."""
    kw = dict(seed=seed, n_paths=n_paths, max_depth=max_depth, attached=int(attached), **opts)
    return _LightTrace.apply(scene, kw, method, albedo, Le, heights)
