"""Batched multi-view passes, CUDA-graph capture and the launch-shape autotuner.

``MultiViewStep`` runs the joint forward + backward of many views of one map -- the mapping
window of Sec. 3.4 (keyframes of uneven resolution replayed together) -- as one plan: one launch
per stage for all views, gradients of every view accumulated into shared vertex, colour and
opacity buffers, optionally persistent raster CTAs and a captured CUDA graph.  ``autotune`` times
the candidate tile shapes, stage sizes and launch forms on the actual workload and caches the
winner per workload signature.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Iterable, Optional

import numpy as np
import torch

from . import binding as B
from .rasterizer import Map, Rasterizer

TILE_SHAPES = ((16, 8), (8, 8), (16, 16), (32, 8), (16, 32), (32, 16))
STAGE_SIZES = (32, 64, 128)


class MultiViewStep:
    """Forward, loss and backward of all views of ``cams`` on ``m`` in one batched pass.

    The loss is the mapping loss E_map of Eq. 15, term by term:
      * E_pho + lambda_dep E_dep (Eq. 8, 13): (1 - lambda_ssim) L1 + lambda_ssim D-SSIM on colour
        (lambda_ssim = 0 uses the plain L1 kernel), L1 on depth;
      * lambda_norm E_norm (Eq. 12) when sensor normals ``tgt_normal`` ([3P] packed like colour,
        zero where there is none) are given: the plan then renders the normal map
        (TS_FLAG_NORMALS) and its gradient joins the backward;
      * lambda_equi E_equi (Eq. 14) on the map's faces when lambda_equi > 0 (needs ``grad``).
    Map gradients accumulate into ``grad``; per-view values are in ``losses()``.  With the plain L1
    loss (no D-SSIM, no normals) the step is the fused ts_render_step_l1 pass."""

    def __init__(self, m: Map, cams, poses: torch.Tensor, tgt_color: torch.Tensor, tgt_depth: torch.Tensor,
                 params: Optional[B.TsRasterParams] = None, grad: Optional[Map] = None, lambda_dep: float = 0.05,
                 pair_capacity: int = 0, want_pose: bool = True, lambda_ssim: float = 0.0,
                 tgt_normal: Optional[torch.Tensor] = None, lambda_norm: float = 0.05, lambda_equi: float = 0.0):
        self.map, self.poses = m, poses
        self.tc, self.td, self.tn = tgt_color, tgt_depth, tgt_normal
        if tgt_normal is not None:
            params = B.TsRasterParams.from_buffer_copy(params) if params is not None else B.ts_default_params()
            params.flags |= B.TS_FLAG_NORMALS
        self.rast = Rasterizer(cams, m.n_faces, params, pair_capacity=pair_capacity)
        self.grad = grad
        self.lambda_dep, self.lambda_ssim = float(lambda_dep), float(lambda_ssim)
        self.lambda_norm, self.lambda_equi = float(lambda_norm), float(lambda_equi)
        if self.lambda_equi > 0 and grad is None:
            raise ValueError("the equilateral term needs map gradient buffers")
        self.equi = torch.zeros(1, dtype=torch.float32, device=self.rast.ws.device)
        self.want_pose = want_pose
        self.graph: Optional[torch.cuda.CUDAGraph] = None

    @property
    def fused(self) -> bool:
        """True when the loss is the plain L1 colour + depth term: the step then runs the forward,
        the loss and the backward in one pass per tile (ts_render_step_l1)."""
        return self.lambda_ssim == 0 and self.tn is None

    def step(self):
        r = self.rast
        r.project(self.map, self.poses)
        r.bin()
        if self.fused:
            r.step_l1(self.tc, self.td, self.lambda_dep, self.grad)
            if self.lambda_equi > 0:
                r.equilateral(self.map, self.lambda_equi, self.grad, out=self.equi)
            if self.want_pose:
                r.pose_grad()
            return
        r.render_fwd()
        if self.lambda_ssim > 0:
            r.pho_loss(self.tc, self.td, self.lambda_ssim, self.lambda_dep)
        else:
            r.l1_loss(self.tc, self.td, self.lambda_dep)
        dN = None
        if self.tn is not None:
            _, dN = r.normal_loss(self.tn, self.lambda_norm)
        r.backward(r.dC, r.dD, None, self.grad, dN=dN)
        if self.lambda_equi > 0:
            r.equilateral(self.map, self.lambda_equi, self.grad, out=self.equi)
        if self.want_pose:
            r.pose_grad()

    def losses(self) -> dict:
        """Per-view E_pho + lambda_dep E_dep, per-view E_norm (if normals), and E_equi (if on)."""
        r = self.rast
        out = {"pho_dep": r.loss_v}
        if self.tn is not None:
            out["norm"] = r.nloss_v
        if self.lambda_equi > 0:
            out["equi"] = self.equi
        return out

    def capture(self):
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step()
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step()
        self.graph = g

    def run(self, n: int = 1, use_graph: bool = False):
        if use_graph and self.graph is None:
            self.capture()
        for _ in range(n):
            if use_graph:
                self.graph.replay()
            else:
                self.step()


def time_ms(fn, iters: int = 5, warmup: int = 2) -> float:
    """Mean device time of fn() with CUDA events on the current stream."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(iters):
        fn()
    b.record()
    b.synchronize()
    return a.elapsed_time(b) / iters


def signature(cams, n_faces: int) -> str:
    cams = np.asarray(cams, np.float64).reshape(-1, 6)
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    key = json.dumps([name, int(n_faces), sorted(map(tuple, cams[:, 4:6].astype(int).tolist()))])
    return hashlib.sha1(key.encode()).hexdigest()[:16]


def _cache_path() -> str:
    return os.environ.get("TS_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "ts_gb300_autotune.json"))


def autotune(m: Map, cams, poses, tgt_color, tgt_depth, grad: Optional[Map] = None,
             tiles: Iterable = TILE_SHAPES, stages: Iterable = STAGE_SIZES, persistent=(False, True),
             iters: int = 3, use_cache: bool = True, **param_overrides):
    """Pick (tile_w, tile_h, tris_per_stage, persistent) for this workload by timing the full
    forward + backward step.  Returns (best dict, all timings)."""
    sig = signature(cams, m.n_faces)
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
        if sig in cache:
            return cache[sig], None
    results = []
    best = None
    for (tw, th) in tiles:
        for S in stages:
            for per in persistent:
                p = B.ts_default_params(tile_w=tw, tile_h=th, tris_per_stage=S,
                                        flags=(B_FLAG_PERSISTENT if per else 0), **param_overrides)
                step = MultiViewStep(m, cams, poses, tgt_color, tgt_depth, p, grad)
                ms = time_ms(step.step, iters=iters, warmup=1)
                results.append(dict(tile_w=tw, tile_h=th, tris_per_stage=S, persistent=per, ms=ms))
                if best is None or ms < best["ms"]:
                    best = results[-1]
                del step
                torch.cuda.empty_cache()
    if use_cache:
        cache[sig] = best
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(cache, f, indent=1)
    return best, results


B_FLAG_PERSISTENT = B.TS_FLAG_PERSISTENT


def params_of(choice: dict, **overrides) -> B.TsRasterParams:
    return B.ts_default_params(tile_w=choice["tile_w"], tile_h=choice["tile_h"],
                               tris_per_stage=choice["tris_per_stage"],
                               flags=B_FLAG_PERSISTENT if choice.get("persistent") else 0, **overrides)
