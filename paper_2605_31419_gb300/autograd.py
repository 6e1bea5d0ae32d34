"""torch.autograd wrappers: rendering differentiable w.r.t. the map and the camera poses.

``render(rast, map, poses, tau)`` returns the packed colour, depth and opacity images; its
backward calls ``ts_render_bwd`` (map gradients) and ``ts_pose_grad`` (dL/dtau for the left
perturbation Exp(tau) o T_CW, Eq. 5-7).  ``tau`` is a [V, 6] tensor evaluated at zero: the
returned pose gradient is the manifold gradient at the given poses, which gradient-descent
tracking then applies with ``ts_pose_apply`` (T <- Exp(-lr * g) o T).
"""
from __future__ import annotations

import torch

from .rasterizer import Map, Rasterizer


class RenderFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rast: Rasterizer, faces, poses, pos, col, opa, tau):
        if tau is not None and bool(torch.any(tau != 0)):
            raise ValueError("tau is the pose perturbation at zero; apply steps with ts_pose_apply")
        m = Map(pos.contiguous(), col.contiguous(), opa.contiguous(), faces)
        C, D, A = rast.forward(m, poses)
        ctx.rast = rast
        ctx.generation = rast.generation
        ctx.map = m
        ctx.need_pose = tau is not None and tau.requires_grad
        return C.clone(), D.clone(), A.clone()

    @staticmethod
    def backward(ctx, gC, gD, gA):
        rast: Rasterizer = ctx.rast
        if rast.generation != ctx.generation:
            raise RuntimeError("the rasterizer was reused by another forward before this backward")
        m = ctx.map
        g = m.zeros_like()
        dA = gA.contiguous() if gA is not None else None
        dD = gD.contiguous() if gD is not None else None
        dC = gC.contiguous() if gC is not None else torch.zeros_like(rast.color)
        rast.backward(dC, dD, dA, g)
        dtau = rast.pose_grad().clone() if ctx.need_pose else None
        return None, None, None, g.pos, g.col, g.opa, dtau


def render(rast: Rasterizer, m: Map, poses: torch.Tensor, tau: torch.Tensor = None):
    """Differentiable render of all views of ``rast``: (color [3P], depth [P], alpha [P])."""
    return RenderFunction.apply(rast, m.faces, poses, m.pos, m.col, m.opa, tau)
