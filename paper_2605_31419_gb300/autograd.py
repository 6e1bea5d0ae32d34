"""torch.autograd wrappers: rendering differentiable w.r.t. the map and the camera poses.

``render(rast, map, poses, tau)`` returns the packed colour, depth and opacity images; its
backward calls ``ts_render_bwd`` (map gradients) and ``ts_pose_grad`` (dL/dtau for the left
perturbation Exp(tau) o T_CW, Eq. 5-7).  ``tau`` is a [V, 6] tensor of zeros that the caller
supplies to ask for the pose gradient: the returned gradient is the manifold gradient at the
given poses, which gradient-descent tracking then applies with ``ts_pose_apply``
(T <- Exp(-lr * g) o T).  Its values are not read on the hot path (reading them would
synchronise the host with the device); with the environment variable TS_DEBUG_CHECKS=1 the
forward checks that they are zero.
"""
from __future__ import annotations

import os

import torch

from .rasterizer import Map, Rasterizer

_DEBUG_CHECKS = os.environ.get("TS_DEBUG_CHECKS", "0") == "1"


class RenderFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rast: Rasterizer, faces, poses, pos, col, opa, tau):
        if tau is not None and _DEBUG_CHECKS and bool(torch.any(tau != 0)):  # host sync: debug only
            raise ValueError("tau is the pose perturbation at zero; apply steps with ts_pose_apply")
        m = Map(pos.contiguous(), col.contiguous(), opa.contiguous(), faces)
        C, D, A = rast.forward(m, poses)
        ctx.rast = rast
        ctx.generation = rast.generation
        ctx.done = False
        ctx.map = m
        ctx.need_pose = tau is not None and tau.requires_grad
        return C.clone(), D.clone(), A.clone()

    @staticmethod
    def backward(ctx, gC, gD, gA):
        rast: Rasterizer = ctx.rast
        if rast.generation != ctx.generation:
            raise RuntimeError("the rasterizer was reused by another forward before this backward")
        if ctx.done:  # the per-face sums of a projection serve one backward
            raise RuntimeError("a second backward through one render; render again to differentiate again")
        ctx.done = True
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
