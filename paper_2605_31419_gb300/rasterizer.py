"""Device-resident rasterizer objects over the libts C ABI.

``Map`` holds a triangle map as structure-of-arrays CUDA tensors; ``Rasterizer`` owns one plan,
one workspace and the output images of a fixed set of views, and calls the five stages of the
path (project, bin, forward, backward, pose gradient) plus the L1 loss.  Autograd wrappers live
in ``autograd.py``.  No computation happens here: every step is a libts kernel.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import binding as B


@dataclass
class Map:
    """Vertices as SoA float32 CUDA tensors: pos [3, N], col [3, N], opa [N]; faces int32 [M, 3] or
    None for triangle-soup mode (face m = vertices 3m, 3m+1, 3m+2); sigma [M] per-face window
    exponents for plans with TS_FLAG_FACE_SIGMA (in a gradient Map: dL/dsigma)."""
    pos: torch.Tensor
    col: torch.Tensor
    opa: torch.Tensor
    faces: Optional[torch.Tensor] = None
    sigma: Optional[torch.Tensor] = None

    @property
    def n_faces(self) -> int:
        return self.faces.shape[0] if self.faces is not None else self.pos.shape[1] // 3

    @staticmethod
    def from_numpy(pos, col, opa, faces=None, device="cuda", sigma=None) -> "Map":
        t = lambda a: torch.from_numpy(np.ascontiguousarray(np.asarray(a, np.float32).T)).to(device)  # noqa: E731
        f = None if faces is None else torch.from_numpy(np.ascontiguousarray(faces, np.int32)).to(device)
        sg = None if sigma is None else torch.from_numpy(np.ascontiguousarray(sigma, np.float32)).to(device)
        return Map(t(pos), t(col), torch.from_numpy(np.ascontiguousarray(opa, np.float32)).to(device), f, sg)

    def ts(self) -> B.TsMap:
        for name in ("pos", "col", "opa"):
            t = getattr(self, name)
            if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
                raise ValueError(f"Map.{name} must be a contiguous float32 CUDA tensor")
        return B.make_map(self.pos, self.col, self.opa, self.faces, self.sigma)

    def zeros_like(self) -> "Map":
        return Map(torch.zeros_like(self.pos), torch.zeros_like(self.col), torch.zeros_like(self.opa), self.faces,
                   None if self.sigma is None else torch.zeros_like(self.sigma))


def poses_tensor(poses, device="cuda") -> torch.Tensor:
    """[V, 12] float32 (row-major R | t, world to camera) on the device."""
    return torch.as_tensor(np.asarray(poses, np.float32).reshape(-1, 12), device=device).contiguous()


class Rasterizer:
    """One plan + workspace + images for ``cams`` ([V, 6]: fx, fy, cx, cy, W, H) and ``n_faces``."""

    def __init__(self, cams, n_faces: int, params: Optional[B.TsRasterParams] = None, pair_capacity: int = 0,
                 device="cuda", **param_overrides):
        self.cams = np.asarray(cams, np.float64).reshape(-1, 6)
        self.V = len(self.cams)
        self.n_faces = int(n_faces)
        self.params = params if params is not None else B.ts_default_params(**param_overrides)
        self.plan = B.ts_plan_init(self.cams, self.n_faces, self.params, pair_capacity)
        self.layout = B.ts_plan_layout(self.plan, self.V)
        self.n_pix = int(self.layout["pix_off"][-1])
        self.device = torch.device(device)
        self.ws_bytes = B.ts_workspace_size(self.plan)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        assert self.ws.data_ptr() % 256 == 0
        B.ts_workspace_init(self.plan, self.ws)
        self.color = torch.empty(3 * self.n_pix, dtype=torch.float32, device=self.device)
        self.depth = torch.empty(self.n_pix, dtype=torch.float32, device=self.device)
        self.alpha = torch.empty(self.n_pix, dtype=torch.float32, device=self.device)
        self.dtau = torch.empty(self.V, 6, dtype=torch.float32, device=self.device)
        self.loss_v = torch.empty(self.V, dtype=torch.float32, device=self.device)
        self.dC = torch.empty_like(self.color)
        self.dD = torch.empty_like(self.depth)
        # the normal map of Eq. 12 and its loss gradient, with TS_FLAG_NORMALS
        self.normals = bool(self.params.flags & B.TS_FLAG_NORMALS)
        self.normal = torch.empty_like(self.color) if self.normals else None
        self.dN = torch.empty_like(self.color) if self.normals else None
        self.nloss_v = torch.empty(self.V, dtype=torch.float32, device=self.device) if self.normals else None
        self._map: Optional[Map] = None
        self._poses: Optional[torch.Tensor] = None
        self.generation = 0

    # -- the path -------------------------------------------------------------------------------
    def project(self, m: Map, poses: torch.Tensor, stream=None):
        if m.n_faces != self.n_faces:
            raise ValueError(f"map has {m.n_faces} faces, plan expects {self.n_faces}")
        self._map, self._poses = m, poses
        self._tsmap = m.ts()
        B.ts_project(self.plan, self._tsmap, poses, self.ws, stream)
        self.generation += 1

    def bin(self, stream=None):
        B.ts_bin(self.plan, self.ws, stream)

    def render_fwd(self, stream=None, color=None, depth=None, alpha=None, normal=None):
        c = self.color if color is None else color
        d = self.depth if depth is None else depth
        a = self.alpha if alpha is None else alpha
        if self.normals:
            B.ts_render_fwd_n(self.plan, self.ws, c, d, a, self.normal if normal is None else normal, stream)
        else:
            B.ts_render_fwd(self.plan, self.ws, c, d, a, stream)

    def forward(self, m: Map, poses: torch.Tensor, stream=None):
        """Project, bin and composite all views; returns (color [3P], depth [P], alpha [P]) views of
        the rasterizer's own buffers (overwritten by the next call)."""
        self.project(m, poses, stream)
        self.bin(stream)
        self.render_fwd(stream)
        return self.color, self.depth, self.alpha

    def backward(self, dC, dD=None, dA=None, grad: Optional[Map] = None, stream=None, dN=None):
        """Adds dL/d(map) into ``grad`` (a Map of gradient tensors) and prepares the pose partials.
        dN: gradient w.r.t. the normal map (plans with TS_FLAG_NORMALS)."""
        g = B.make_grad(grad.pos, grad.col, grad.opa, grad.sigma) if grad is not None else None
        if dN is not None:
            B.ts_render_bwd_n(self.plan, self.ws, dC, dD, dA, dN, g, stream)
        else:
            B.ts_render_bwd(self.plan, self.ws, dC, dD, dA, g, stream)

    def step_l1(self, tgt_color, tgt_depth, lambda_dep: float = 0.05, grad: Optional[Map] = None, stream=None,
                loss_grads: bool = False):
        """The forward, the mean-L1 loss and the backward of one step in one pass per tile (after
        ``project`` and ``bin``): the images in the rasterizer's buffers, the per-view loss, and the
        map gradients added into ``grad``; ``pose_grad`` then gives the pose gradients.  With
        ``loss_grads`` the loss's image gradients are also written to ``dC`` and ``dD``."""
        g = B.make_grad(grad.pos, grad.col, grad.opa, grad.sigma) if grad is not None else None
        B.ts_render_step_l1(self.plan, self.ws, tgt_color, tgt_depth, lambda_dep, self.color, self.depth, self.alpha,
                            self.loss_v, self.dC if loss_grads else None, self.dD if loss_grads else None, g, stream)
        return self.loss_v

    def pose_grad(self, out=None, stream=None):
        out = self.dtau if out is None else out
        B.ts_pose_grad(self.plan, self.ws, out, stream)
        return out

    def l1_loss(self, tgt_color, tgt_depth, lambda_dep: float = 0.05, stream=None):
        B.ts_l1_loss(self.plan, self.ws, self.color, self.depth, tgt_color, tgt_depth, lambda_dep, self.loss_v,
                     self.dC, self.dD, stream)
        return self.loss_v, self.dC, self.dD

    def pho_loss(self, tgt_color, tgt_depth, lambda_ssim: float = 0.2, lambda_dep: float = 0.05, stream=None):
        """Eq. 8-10: (1 - lambda) L1 + lambda D-SSIM colour terms and the L1 depth term of the last
        forward's images, with their gradients (the rasterizer's loss buffers, overwritten)."""
        B.ts_pho_loss(self.plan, self.ws, self.color, self.depth, tgt_color, tgt_depth, lambda_ssim, lambda_dep,
                      self.loss_v, self.dC, self.dD, stream)
        return self.loss_v, self.dC, self.dD

    def face_stats(self, stream=None) -> dict:
        """Map statistics of the last forward (Sec. 3.4), per (view, face) [V, M]: projected area
        (pixels^2), and with TS_FLAG_STATS the pixel coverage, the visible-face bitsets
        [V, ceil(M/32)] (int32 views of uint32 words) and their counts [V]."""
        V, M = self.V, self.n_faces
        dev = self.ws.device
        out = {"area": torch.empty(V, M, dtype=torch.float32, device=dev)}
        stats = bool(self.params.flags & B.TS_FLAG_STATS)
        if stats:
            out["coverage"] = torch.empty(V, M, dtype=torch.int32, device=dev)
            out["visible"] = torch.empty(V, (M + 31) // 32, dtype=torch.int32, device=dev)
            out["n_visible"] = torch.empty(V, dtype=torch.int32, device=dev)
        B.ts_face_stats(self.plan, self.ws, out.get("coverage"), out["area"], out.get("visible"),
                        out.get("n_visible"), stream)
        return out

    def covisibility(self, visible, stream=None) -> torch.Tensor:
        """IoU [V, V] of the views' visible-face sets (bitsets from face_stats)."""
        iou = torch.empty(self.V, self.V, dtype=torch.float32, device=self.ws.device)
        B.ts_covisibility(self.plan, visible, iou, stream)
        return iou

    def normal_loss(self, tgt_normal, weight: float = 0.05, stream=None):
        """Eq. 12 on the last forward's normal map against sensor normals tgt_normal [3P] (zero =
        no normal): per-view loss [V] and its gradient (scaled by ``weight``, lambda_norm)."""
        if not self.normals:
            raise ValueError("the plan was made without TS_FLAG_NORMALS")
        B.ts_normal_loss(self.plan, self.ws, self.normal, tgt_normal, weight, self.nloss_v, self.dN, stream)
        return self.nloss_v, self.dN

    def equilateral(self, m: Map, weight: float = 1.2, grad: Optional[Map] = None, out=None, stream=None):
        """Eq. 14 on the map's faces: returns E (device [1]); adds weight * dE/dpos into grad.pos."""
        out = torch.empty(1, dtype=torch.float32, device=self.ws.device) if out is None else out
        g = B.make_grad(grad.pos, None, None) if grad is not None else None
        B.ts_equilateral(self.plan, m.ts(), self.ws, weight, out, g, stream)
        return out

    def counters(self, stream=None, raise_on_error=True) -> dict:
        return B.ts_sync_status(self.plan, self.ws, stream, raise_on_error)

    def debug(self, what: str) -> torch.Tensor:
        VM = self.V * self.n_faces
        cap = int(self.counters(raise_on_error=False)["pair_capacity"])
        n_tiles = int(self.layout["tile_off"][-1])
        shapes = dict(keys=(cap, torch.int64), ids=(cap, torch.int32), ranges=(2 * n_tiles, torch.int32),
                      rect=(4 * VM, torch.int16), zbits=(VM, torch.int32), count=(VM, torch.int32),
                      T_final=(self.n_pix, torch.float32), n_last=(self.n_pix, torch.int32),
                      records=(32 * VM, torch.float32))
        n, dt = shapes[what]
        out = torch.empty(max(n, 1), dtype=dt, device=self.device)
        if n:
            B.ts_debug_copy(self.plan, self.ws, what, out)
        torch.cuda.synchronize()
        return out[:n]

    # -- packing helpers --------------------------------------------------------------------------
    def unpack(self, flat: torch.Tensor, channels: int):
        """Split a packed image buffer into per-view [channels, H, W] (or [H, W]) tensors."""
        out = []
        for v in range(self.V):
            W, H = int(self.cams[v, 4]), int(self.cams[v, 5])
            o = int(self.layout["pix_off"][v])
            if channels == 1:
                out.append(flat[o:o + H * W].view(H, W))
            else:
                out.append(flat[channels * o:channels * (o + H * W)].view(channels, H, W))
        return out

    def pack(self, images, channels: int) -> torch.Tensor:
        return torch.cat([torch.as_tensor(i, dtype=torch.float32, device=self.device).reshape(-1) for i in images])
