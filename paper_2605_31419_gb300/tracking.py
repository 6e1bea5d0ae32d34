"""Differentiable camera tracking (Triangle Splatting SLAM, Sec. 3.3-3.4 "Tracking").

Many pose hypotheses of one frame are rendered as the views of one plan, so every iteration is a
single batched pass: project, bin, forward blend, the tracking loss E_track (Eq. 8-10: (1 - lambda)
L1 + lambda D-SSIM colour terms, lambda = 0.2, and the L1 depth term with lambda_dep), backward to the pose (Eq. 5-7, map gradients skipped) and an Adam step
on the manifold gradient applied as T <- Exp(-step) o T.  One iteration is captured once in a CUDA
graph and replayed, so 100 iterations cost 100 graph launches.  All arithmetic runs in libts.
"""
from __future__ import annotations

from typing import Optional

import numpy as np
import torch

from . import binding as B
from .rasterizer import Map, Rasterizer, poses_tensor


class Tracker:
    """Track ``len(init_poses)`` hypotheses of one camera against one RGB-D target.

    target_color: [3, H, W] and target_depth: [H, W] (numpy or tensors); the target is shared by
    all hypotheses.  Learning rates and loss weights default to Table S5 (rotation 0.003,
    translation 0.001, D-SSIM weight 0.2, depth weight 0.05); lambda_ssim = 0 drops the D-SSIM term
    and uses the plain L1 kernel."""

    def __init__(self, m: Map, cam, target_color, target_depth, init_poses, params: Optional[B.TsRasterParams] = None,
                 lr_rot: float = 0.003, lr_trans: float = 0.001, lambda_dep: float = 0.05, lambda_ssim: float = 0.2,
                 device="cuda"):
        cam = np.asarray(cam, np.float64).reshape(6)
        init_poses = np.asarray(init_poses, np.float32).reshape(-1, 12)
        self.n_hyp = len(init_poses)
        self.map = m
        self.rast = Rasterizer(np.tile(cam, (self.n_hyp, 1)), m.n_faces, params, device=device)
        self.poses = poses_tensor(init_poses, device=device)
        as_dev = lambda a: (a.to(device=device, dtype=torch.float32) if isinstance(a, torch.Tensor)  # noqa: E731
                            else torch.as_tensor(np.asarray(a, np.float32), device=device))
        tc = as_dev(target_color).reshape(-1)
        td = as_dev(target_depth).reshape(-1)
        self.tc = tc.repeat(self.n_hyp).contiguous()
        self.td = td.repeat(self.n_hyp).contiguous()
        self.state = torch.zeros(self.n_hyp, 13, dtype=torch.float32, device=device)
        self.lr_rot, self.lr_trans, self.lambda_dep = float(lr_rot), float(lr_trans), float(lambda_dep)
        self.lambda_ssim = float(lambda_ssim)
        self.graph: Optional[torch.cuda.CUDAGraph] = None

    def step(self):
        """One tracking iteration on the current stream (capturable)."""
        r = self.rast
        r.project(self.map, self.poses)
        r.bin()
        r.render_fwd()
        if self.lambda_ssim > 0:
            r.pho_loss(self.tc, self.td, self.lambda_ssim, self.lambda_dep)
        else:
            r.l1_loss(self.tc, self.td, self.lambda_dep)
        r.backward(r.dC, r.dD, None, None)
        r.pose_grad()
        B.ts_pose_adam(r.plan, self.poses, r.dtau, self.state, self.lr_trans, self.lr_rot)

    def capture(self):
        """Capture one iteration into a CUDA graph (state is not advanced by the capture)."""
        poses0, state0 = self.poses.clone(), self.state.clone()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step()  # warm-up outside the graph
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step()
        self.poses.copy_(poses0)
        self.state.copy_(state0)
        self.graph = g

    def run(self, iters: int, use_graph: bool = True):
        if use_graph:
            if self.graph is None:
                self.capture()
            for _ in range(iters):
                self.graph.replay()
        else:
            for _ in range(iters):
                self.step()
        return self.poses

    def loss(self) -> torch.Tensor:
        return self.rast.loss_v


def pose_error(P: np.ndarray, Q: np.ndarray):
    """Translation (m) and rotation (deg) distance between world-to-camera poses [12]."""
    P = np.asarray(P, np.float64).reshape(-1, 12)
    Q = np.asarray(Q, np.float64).reshape(-1, 12)
    out = []
    for p, q in zip(P, Q):
        Rp, Rq = p[:9].reshape(3, 3), q[:9].reshape(3, 3)
        cp, cq = -Rp.T @ p[9:], -Rq.T @ q[9:]  # camera centres
        c = np.clip((np.trace(Rp @ Rq.T) - 1) / 2, -1.0, 1.0)
        out.append((float(np.linalg.norm(cp - cq)), float(np.degrees(np.arccos(c)))))
    return np.array(out)
