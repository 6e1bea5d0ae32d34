"""Serving loop: a device-resident map answering render and track requests as they arrive.

Continuous batching: requests wait in an arrival queue; at every scheduler step, the arrived
ones are admitted while the batch fits the step's budget (views, pixels, and the workspace bytes
that ts_workspace_size reports for the candidate batch, against workspaces allocated once from
the free HBM), renders of the step are rendered in one batched forward on the render stream, and
every admitted track request advances one gradient iteration in one batched forward + backward +
pose update on the track stream; a track request keeps its slot for ``track_iters`` iterations
and leaves, new ones join at the next step.  The two streams let a step's renders and tracks
overlap on the device, and the host prepares the next step while the device works.  Latency is
arrival to completion (the completion event observed by the host).

Render requests run on forward-only plans (TS_FLAG_FORWARD_ONLY): no gradient slots are cleared
and no lane masks are stored for them, and their workspace is smaller.  ``serve_plain`` is the
baseline without batching: the same requests, one at a time in arrival order, each on its own
single-view plan.  A run ends ``drain_seconds`` after the last arrival; requests not finished by
then are reported as not served.

All arithmetic runs in libts kernels; torch moves pose rows, targets and results between request
slots and the batch buffers.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import torch

from . import binding as B
from .rasterizer import Map


@dataclass
class Request:
    rid: int
    kind: str                      # "render" | "track"
    cam: np.ndarray                # [6] fx, fy, cx, cy, W, H
    pose: np.ndarray               # [12] initial world-to-camera pose
    t_arrival: float = 0.0         # seconds after the start of the run
    target_color: Optional[torch.Tensor] = None  # track: [3, H, W] on the device
    target_depth: Optional[torch.Tensor] = None  # track: [H, W]
    # filled by the server
    iters_done: int = 0
    t_admit: float = -1.0
    t_done: float = -1.0
    color: Optional[torch.Tensor] = None
    depth: Optional[torch.Tensor] = None
    alpha: Optional[torch.Tensor] = None
    pose_out: Optional[torch.Tensor] = None
    _slot: int = -1

    @property
    def pixels(self) -> int:
        return int(self.cam[4]) * int(self.cam[5])


@dataclass
class _Lane:
    """One stream with its workspace and image buffers, reused by every step."""
    stream: torch.cuda.Stream
    ws: torch.Tensor
    color: torch.Tensor
    depth: torch.Tensor
    alpha: torch.Tensor
    pending: list = field(default_factory=list)  # (event, requests finished by that step)


class Server:
    def __init__(self, m: Map, params: Optional[B.TsRasterParams] = None, max_views: int = 32,
                 max_pixels: int = 32 * 1200 * 680, pair_capacity: Optional[int] = None, track_iters: int = 10,
                 lr_rot: float = 0.003, lr_trans: float = 0.001, lambda_dep: float = 0.05,
                 lambda_ssim: float = 0.2, hbm_fraction: float = 0.5, device="cuda"):
        self.map, self.params = m, (params if params is not None else B.ts_default_params())
        # render requests: the same launch shape on forward-only plans
        self.render_params = B.TsRasterParams.from_buffer_copy(self.params)
        self.render_params.flags |= B.TS_FLAG_FORWARD_ONLY
        self.max_views, self.max_pixels = int(max_views), int(max_pixels)
        self.track_iters, self.lambda_dep = int(track_iters), float(lambda_dep)
        self.lambda_ssim = float(lambda_ssim)
        self.lr_rot, self.lr_trans = float(lr_rot), float(lr_trans)
        self.device = torch.device(device)
        M = m.n_faces
        # (tile, face) pairs scale with the visible faces of a view, not with its pixels: the
        # default holds 4 tiles per face in every view of the largest batch
        self.pair_capacity = int(pair_capacity if pair_capacity is not None else 4 * self.max_views * M)
        # workspace budget: a plan of max_views views at the largest resolution, capped by free HBM
        probe = B.ts_plan_init(np.tile([[600.0, 600.0, 600.0, 340.0, 1200, 680]], (self.max_views, 1)), M,
                               self.params, self.pair_capacity)
        want = B.ts_workspace_size(probe)
        free = torch.cuda.mem_get_info(self.device)[0]
        self.ws_bytes = int(min(want, hbm_fraction * free / 2))
        mk = lambda: _Lane(torch.cuda.Stream(self.device),  # noqa: E731
                           torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device),
                           torch.empty(3 * self.max_pixels, device=self.device),
                           torch.empty(self.max_pixels, device=self.device),
                           torch.empty(self.max_pixels, device=self.device))
        self.render_lane, self.track_lane = mk(), mk()
        for lane in (self.render_lane, self.track_lane):
            # once: the device header (counters, error word) sits at the start of every plan's
            # layout, and every other region is written before it is read within a step
            lane.ws[:4096].zero_()
        # track state: pose and Adam rows per slot
        self.slots = max_views
        self.slot_pose = torch.zeros(self.slots, 12, device=self.device)
        self.slot_adam = torch.zeros(self.slots, 13, device=self.device)
        self.free_slots = list(range(self.slots))
        self.loss = torch.empty(self.max_views, device=self.device)
        self.dC = torch.empty(3 * self.max_pixels, device=self.device)
        self.dD = torch.empty(self.max_pixels, device=self.device)
        self.dtau = torch.empty(self.max_views, 6, device=self.device)
        self.stats = dict(steps=0, pixels=0, rejected_for_memory=0)
        self._warmup()

    def _warmup(self):
        """One render and one track step on a 16 x 16 view, so that one-time costs of the device
        code a step runs (module loading of this library's and PyTorch's kernels, which took
        seconds for PyTorch's index_select and index_copy_ on a fresh GB300) are paid here and
        not by the first requests.  All server state is restored afterwards."""
        cam = np.array([16.0, 16.0, 8.0, 8.0, 16, 16])
        pose = np.array([1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0], np.float32)
        tc = torch.zeros(3, 16, 16, device=self.device)
        td = torch.zeros(16, 16, device=self.device)
        render = Request(-1, "render", cam, pose)
        track = Request(-2, "track", cam, pose, 0.0, tc, td)
        track._slot = self.free_slots[0]
        self._launch_renders([render])
        self._launch_tracks([track])
        torch.cuda.synchronize(self.device)
        self.slot_pose.zero_()
        self.slot_adam.zero_()
        for lane in (self.render_lane, self.track_lane):
            lane.pending.clear()
        self.stats = dict(steps=0, pixels=0, rejected_for_memory=0)

    # ---------------------------------------------------------------- admission
    def _fits(self, cams: List[np.ndarray], render: bool = False) -> bool:
        if len(cams) > self.max_views or sum(int(c[4]) * int(c[5]) for c in cams) > self.max_pixels:
            return False
        return B.ts_workspace_size(self._plan(cams, render)) <= self.ws_bytes

    def _plan(self, cams: List[np.ndarray], render: bool = False):
        return B.ts_plan_init(np.stack(cams), self.map.n_faces, self.render_params if render else self.params,
                              self.pair_capacity)

    # ---------------------------------------------------------------- one scheduler step
    def _launch_renders(self, reqs: List[Request]):
        if not reqs:
            return
        lane = self.render_lane
        cams = [r.cam for r in reqs]
        plan = self._plan(cams, render=True)
        with torch.cuda.stream(lane.stream):
            s = lane.stream
            poses = torch.as_tensor(np.stack([r.pose for r in reqs]).astype(np.float32), device=self.device)
            B.ts_project(plan, self.map.ts(), poses, lane.ws, s)
            B.ts_bin(plan, lane.ws, s)
            B.ts_render_fwd(plan, lane.ws, lane.color, lane.depth, lane.alpha, s)
            o = 0
            for r in reqs:
                P = r.pixels
                H, W = int(r.cam[5]), int(r.cam[4])
                r.color = lane.color[3 * o:3 * (o + P)].view(3, H, W).clone()
                r.depth = lane.depth[o:o + P].view(H, W).clone()
                r.alpha = lane.alpha[o:o + P].view(H, W).clone()
                o += P
            ev = torch.cuda.Event()
            ev.record(s)
        lane.pending.append((ev, reqs))
        self.stats["pixels"] += sum(r.pixels for r in reqs)

    def _launch_tracks(self, reqs: List[Request]):
        if not reqs:
            return
        lane = self.track_lane
        cams = [r.cam for r in reqs]
        plan = self._plan(cams)
        with torch.cuda.stream(lane.stream):
            s = lane.stream
            # every temporary of the step is allocated on the step's stream: a block freed on
            # another stream could be reused before this stream has read it
            idx = torch.as_tensor([r._slot for r in reqs], device=self.device)
            poses = self.slot_pose.index_select(0, idx).contiguous()
            adam = self.slot_adam.index_select(0, idx).contiguous()
            tc = torch.cat([r.target_color.reshape(-1) for r in reqs])
            td = torch.cat([r.target_depth.reshape(-1) for r in reqs])
            B.ts_project(plan, self.map.ts(), poses, lane.ws, s)
            B.ts_bin(plan, lane.ws, s)
            B.ts_render_fwd(plan, lane.ws, lane.color, lane.depth, lane.alpha, s)
            if self.lambda_ssim > 0:
                B.ts_pho_loss(plan, lane.ws, lane.color, lane.depth, tc, td, self.lambda_ssim, self.lambda_dep,
                              self.loss, self.dC, self.dD, s)
            else:
                B.ts_l1_loss(plan, lane.ws, lane.color, lane.depth, tc, td, self.lambda_dep, self.loss, self.dC,
                             self.dD, s)
            B.ts_render_bwd(plan, lane.ws, self.dC, self.dD, None, None, s)
            B.ts_pose_grad(plan, lane.ws, self.dtau, s)
            B.ts_pose_adam(plan, poses, self.dtau, adam, self.lr_trans, self.lr_rot, stream=s)
            self.slot_pose.index_copy_(0, idx, poses)
            self.slot_adam.index_copy_(0, idx, adam)
            done = []
            for r in reqs:
                r.iters_done += 1
                if r.iters_done >= self.track_iters:
                    r.pose_out = self.slot_pose[r._slot].clone()
                    done.append(r)
            ev = torch.cuda.Event()
            ev.record(s)
        lane.pending.append((ev, done))
        self.stats["pixels"] += sum(r.pixels for r in reqs)

    def _poll(self, now: float, block: bool = False):
        for lane in (self.render_lane, self.track_lane):
            keep = []
            for ev, reqs in lane.pending:
                if block:
                    ev.synchronize()
                if ev.query():
                    for r in reqs:
                        r.t_done = now if not block else time.perf_counter() - self._t0
                else:
                    keep.append((ev, reqs))
            lane.pending = keep

    # ---------------------------------------------------------------- driver
    def run(self, requests: List[Request], realtime: bool = True, max_seconds: Optional[float] = None,
            drain_seconds: float = 5.0):
        """Serve ``requests`` (sorted by t_arrival) until all are done or until ``drain_seconds`` after
        the last arrival (``max_seconds``, if given, caps the run).  Returns the requests with results
        and times; unfinished ones keep t_done < 0."""
        queue = deque(sorted(requests, key=lambda r: r.t_arrival))
        if max_seconds is None:
            max_seconds = (queue[-1].t_arrival if queue else 0.0) + drain_seconds
        active: List[Request] = []
        self._t0 = time.perf_counter()
        while (queue or active) and time.perf_counter() - self._t0 < max_seconds:
            now = time.perf_counter() - self._t0
            self._poll(now)
            # admission: arrived requests, while the step's batch fits the budget
            renders: List[Request] = []
            tracks = [r for r in active if r.kind == "track"]
            while queue and (queue[0].t_arrival <= now or not realtime):
                r = queue[0]
                cams_r = [x.cam for x in renders] + [r.cam] if r.kind == "render" else None
                cams_t = [x.cam for x in tracks] + [r.cam] if r.kind == "track" else None
                ok = self._fits(cams_r, True) if r.kind == "render" else (self._fits(cams_t) and bool(self.free_slots))
                if not ok:
                    self.stats["rejected_for_memory"] += 1
                    break  # wait for the running work to leave room
                queue.popleft()
                r.t_admit = now
                if r.kind == "render":
                    renders.append(r)
                else:
                    r._slot = self.free_slots.pop()
                    # on the track stream: after the slot's previous owner's last copies
                    with torch.cuda.stream(self.track_lane.stream):
                        self.slot_pose[r._slot] = torch.as_tensor(r.pose, dtype=torch.float32, device=self.device)
                        self.slot_adam[r._slot].zero_()
                    tracks.append(r)
                    active.append(r)
            if not renders and not tracks:
                if queue and realtime:
                    time.sleep(max(0.0, min(queue[0].t_arrival - now, 0.002)))
                continue
            self._launch_renders(renders)
            self._launch_tracks(tracks)
            self.stats["steps"] += 1
            for r in tracks:
                if r.iters_done >= self.track_iters:
                    active.remove(r)
                    self.free_slots.append(r._slot)
        torch.cuda.synchronize()
        self._poll(time.perf_counter() - self._t0, block=False)
        for r in requests:
            if r.t_done < 0 and (r.color is not None or r.pose_out is not None):
                r.t_done = time.perf_counter() - self._t0
        self.stats["seconds"] = time.perf_counter() - self._t0
        # errors latched on the device by any step (capacity overflow, timeout, bounds)
        probe = self._plan([np.array([1.0, 1.0, 0.0, 0.0, 1, 1])])
        for lane in (self.render_lane, self.track_lane):
            st = B.ts_sync_status(probe, lane.ws, lane.stream, raise_on_error=False)
            if st["status"] != "TS_OK":
                raise B.TsError(3 if st["status"] == "TS_ERR_CAPACITY" else 2, f"serving step failed: {st}")
        return requests


def latency_stats(requests: List[Request], seconds: float):
    """Per request kind: completed and not-served counts, and p50/p99 latency over ALL submitted
    requests of the kind, a request that was not served counting as infinitely late (a percentile
    that falls on one is reported as null with ``..._not_served`` true).  Mpix/s counts the pixels
    of completed requests (a track request: pixels x iterations) over the run's wall time."""
    out = {}
    for kind in ("render", "track"):
        ks = [r for r in requests if r.kind == kind]
        if not ks:
            continue
        lat = np.array([(r.t_done - r.t_arrival) if r.t_done >= 0 else np.inf for r in ks])
        d = {"n": int(np.isfinite(lat).sum()), "not_served": int((~np.isfinite(lat)).sum()), "submitted": len(ks)}
        for q in (50, 99):
            v = float(np.percentile(lat, q, method="higher"))
            d[f"p{q}_ms"] = v * 1e3 if np.isfinite(v) else None
            if not np.isfinite(v):
                d[f"p{q}_not_served"] = True
        out[kind] = d
    done = [r for r in requests if r.t_done >= 0]
    px = sum(r.pixels * (1 if r.kind == "render" else max(r.iters_done, 1)) for r in done)
    out["mpix_s"] = px / max(seconds, 1e-9) / 1e6
    out["completed"] = len(done)
    out["not_served"] = len(requests) - len(done)
    out["submitted"] = len(requests)
    out["seconds"] = seconds
    return out


def serve_plain(m: Map, requests: List[Request], params: Optional[B.TsRasterParams] = None, track_iters: int = 10,
                lr_rot: float = 0.003, lr_trans: float = 0.001, lambda_dep: float = 0.05, lambda_ssim: float = 0.2,
                realtime: bool = True, drain_seconds: float = 5.0, device="cuda") -> float:
    """The baseline without batching: each request alone, in arrival order, on a single-view plan
    (one per resolution, reused): a render is one forward on a forward-only plan, a track request
    its ``track_iters`` gradient iterations back to back.  Same losses and optimiser as ``Server``.
    Returns the run's wall seconds; each request gets t_done (or keeps -1 if not served)."""
    from .rasterizer import Rasterizer
    params = params if params is not None else B.ts_default_params()
    rparams = B.TsRasterParams.from_buffer_copy(params)
    rparams.flags |= B.TS_FLAG_FORWARD_ONLY
    dev = torch.device(device)
    rasts = {}

    def rast(cam, render):
        key = (int(cam[4]), int(cam[5]), float(cam[0]), render)
        if key not in rasts:
            rasts[key] = Rasterizer(cam[None, :], m.n_faces, rparams if render else params, device=dev)
        return rasts[key]

    pose = torch.empty(1, 12, device=dev)
    adam = torch.empty(1, 13, device=dev)
    order = sorted(requests, key=lambda r: r.t_arrival)
    end = (order[-1].t_arrival if order else 0.0) + drain_seconds
    for r in order:  # plans and workspaces before the clock starts
        rast(r.cam, r.kind == "render")
    t0 = time.perf_counter()
    for r in order:
        now = time.perf_counter() - t0
        if now > end:
            break
        if realtime and r.t_arrival > now:
            time.sleep(r.t_arrival - now)
        R = rast(r.cam, r.kind == "render")
        pose.copy_(torch.as_tensor(np.asarray(r.pose, np.float32).reshape(1, 12)))
        if r.kind == "render":
            C, D, A = R.forward(m, pose)
            H, W = int(r.cam[5]), int(r.cam[4])
            r.color, r.depth, r.alpha = C.view(3, H, W).clone(), D.view(H, W).clone(), A.view(H, W).clone()
        else:
            adam.zero_()
            tc, td = r.target_color.reshape(-1), r.target_depth.reshape(-1)
            for _ in range(track_iters):
                R.forward(m, pose)
                if lambda_ssim > 0:
                    R.pho_loss(tc, td, lambda_ssim, lambda_dep)
                else:
                    R.l1_loss(tc, td, lambda_dep)
                R.backward(R.dC, R.dD, None, None)
                R.pose_grad()
                B.ts_pose_adam(R.plan, pose, R.dtau, adam, lr_trans, lr_rot)
            r.iters_done = track_iters
            r.pose_out = pose[0].clone()
        torch.cuda.synchronize(dev)
        r.t_done = time.perf_counter() - t0
    return time.perf_counter() - t0
