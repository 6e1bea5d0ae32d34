"""Benchmark: Mpix/s of forward + backward rasterization on the room workload.

Default workload: 1200x680 pinhole (fx = fy = 600), 300k-face room map, 20 seeded poses, one step =
project + bin + forward + L1 colour/depth loss + backward (map gradients) + pose gradients for all
20 views in one batched call sequence.  ``value`` = pixels of all views (all ranks) per second of
device time, inputs resident in HBM, L2 flushed (256 MB write) between timed steps.

Also reported: the same step done view by view (``plain_per_view``), the end-to-end metric with
inputs copied from pinned host memory and results read back (``e2e``), per-stage event times and
the roofline of the dominant kernel, sampled clocks, and the CPU oracle on a bounded sample.

``--impl reference`` times the CPU oracle instead (the reference arm of this metric).
Under torchrun (N > 1) every rank renders its own replica of the workload (replicas only: the
views are independent, there is no exchange step), timed with a barrier and the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOPS_FWD = 35.0   # algorithmic flops per blended (pixel, face) contribution, forward
FLOPS_BWD = 90.0   # per differentiated contribution, backward raster
# fused L1 + D-SSIM + depth loss, per pixel and channel: 5 window moments as separable 11 + 11-tap
# sums (FMA = 2 flops: 220) and their 3 products, SSIM with its 3 partials (~30), the adjoint as 3
# separable window sums (132), and the gradient and L1 terms (~9)
FLOPS_PHO = 394.0
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per view of one k_render_step launch of
# this workload, from a one-kernel, one-launch ncu capture of the same step cut to 4 views (tile
# 16x8, 64 faces per stage), scaled by the views of the launch; reported only for that configuration
STEP_TRAFFIC_PER_VIEW = (150.714112e6 + 77.189632e6) / 4
W, H, F, N_FACES, N_VIEWS = 1200, 680, 600.0, 300_000, 20
WORKLOAD = "room 1200x680 f=600, 300k faces, 20 poses, fwd+bwd (L1 colour+depth), batched"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the mapping-window, tracking and serving measurements")
    ap.add_argument("--faces", type=int, default=N_FACES)
    ap.add_argument("--views", type=int, default=N_VIEWS)
    ap.add_argument("--tile", default="16x8")
    ap.add_argument("--stage", type=int, default=64)
    ap.add_argument("--eager", action="store_true",
                    help="time the launches one by one instead of replaying the step from a CUDA graph")
    ap.add_argument("--separate", action="store_true",
                    help="time ts_render_fwd + ts_l1_loss + ts_render_bwd instead of the fused ts_render_step_l1")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(t: float, device=None) -> float:
    """The job's step time: the maximum of the ranks' times (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(t)
    tt = torch.tensor([float(t)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_value(pixels_per_rank: int, world: int, t_step: float) -> float:
    """Whole-job Mpix/s: every rank renders its own replica of the workload (weak scaling)."""
    return pixels_per_rank * world / t_step / 1e6


def scene(args):
    from ts_synth import room_scene
    return room_scene(3, args.faces, args.views, W, H, F, target_seed=4)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(sc, time_budget_s=20.0, single_thread=True):
    """The oracle (as it stands) on one view of the workload, all host cores: fwd + L1 + bwd."""
    from oracle.oracle import Oracle, Params, SceneArrays, pack_targets
    o = Oracle()
    sub = sc.subset_views([0])
    sa = SceneArrays.of(sub)
    prm = Params()
    nthreads = os.cpu_count() or 1
    prm.n_threads = nthreads
    tc, td = pack_targets(sub)
    times = []
    t_end = time.perf_counter() + time_budget_s
    while True:
        t0 = time.perf_counter()
        f = o.forward(sa, prm)
        lo = o.l1_loss(sa, f["color"], f["depth"], tc, td, 0.05)
        o.backward(sa, prm, lo["dC"], lo["dD"])
        times.append(time.perf_counter() - t0)
        if time.perf_counter() > t_end or len(times) >= 3 or times[-1] > 0.5 * time_budget_s:
            break
    t = float(np.median(times))
    out = {"value": W * H / t / 1e6, "unit": "Mpix/s", "cores": nthreads, "kind": "oracle",
           "sample": f"1 of {sc.n_views} views (1200x680, {sc.n_faces} faces): fwd + L1 loss + bwd, "
                     f"median of {len(times)} runs, {t:.2f} s each"}
    if single_thread:
        prm.n_threads = 1
        t0 = time.perf_counter()
        f = o.forward(sa, prm)
        lo = o.l1_loss(sa, f["color"], f["depth"], tc, td, 0.05)
        o.backward(sa, prm, lo["dC"], lo["dD"])
        t1 = time.perf_counter() - t0
        out["single_thread"] = {"value": W * H / t1 / 1e6, "unit": "Mpix/s", "cores": 1, "seconds": t1}
    return out


def bench_c1(ts, torch, dev, flush, stream, reps=50):
    """The plain single view: 160x120 (f = 150), 2,000 random triangles at the identity pose, one
    forward (colour, depth, opacity) and one backward of the L1 colour + depth loss against a
    seeded target.  Device time per step through the separate calls and through the fused step,
    each eager and replayed from a captured CUDA graph; and the oracle on the same view."""
    from oracle.oracle import Oracle, Params, SceneArrays, pack_targets
    from ts_synth import random_triangles_scene
    sc = random_triangles_scene(seed=1)
    r = ts.Rasterizer(sc.cams, sc.n_faces)
    m = ts.Map.from_numpy(sc.pos, sc.col, sc.opa, device=dev)
    poses = ts.poses_tensor(sc.poses, device=dev)
    tcn, tdn = pack_targets(sc)
    tc = torch.as_tensor(tcn, dtype=torch.float32, device=dev)
    td = torch.as_tensor(tdn, dtype=torch.float32, device=dev)
    g = m.zeros_like()

    def sep():
        g.pos.zero_(); g.col.zero_(); g.opa.zero_()
        r.forward(m, poses)
        r.l1_loss(tc, td, 0.05)
        r.backward(r.dC, r.dD, None, g)
        r.pose_grad()

    def fused():
        g.pos.zero_(); g.col.zero_(); g.opa.zero_()
        r.project(m, poses)
        r.bin()
        r.step_l1(tc, td, 0.05, g)
        r.pose_grad()

    def timed(fn):
        for _ in range(5):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return float(np.median(ms))

    out = {"workload": "160x120 f=150, 2,000 random faces (sides 2-10 cm, depth 0.5-4 m), identity pose, "
                       "fwd + L1 loss + bwd, one view", "pixels": 19200, "faces": sc.n_faces}
    res = {}
    for name, fn in (("separate", sep), ("fused", fused)):
        res[name + "_eager_ms"] = timed(fn)
        gr = torch.cuda.CUDAGraph()
        s2 = torch.cuda.Stream(device=dev)
        s2.wait_stream(stream)
        with torch.cuda.stream(s2):
            fn()
            with torch.cuda.graph(gr, stream=s2):
                fn()
        stream.wait_stream(s2)
        res[name + "_graph_ms"] = timed(gr.replay)
    best = min(res.values())
    cnt = r.counters()
    out.update({"ms": res, "mpix_s": 19200 / best / 1e3, "triangles_per_s": sc.n_faces / (best / 1e3),
                "visible_faces": int(cnt["n_visible"]), "best": min(res, key=res.get)})
    # the oracle on the same view, all host cores and one
    o = Oracle()
    sa = SceneArrays.of(sc)
    for label, nth in (("oracle_all_cores", os.cpu_count() or 1), ("oracle_1_thread", 1)):
        prm = Params(n_threads=nth)
        ts_ = []
        for _ in range(3):
            t0 = time.perf_counter()
            f = o.forward(sa, prm)
            lo = o.l1_loss(sa, f["color"], f["depth"], tcn, tdn, 0.05)
            o.backward(sa, prm, lo["dC"], lo["dD"])
            ts_.append(time.perf_counter() - t0)
        t = float(np.median(ts_))
        out[label] = {"mpix_s": 19200 / t / 1e6, "ms": t * 1e3, "cores": nth}
    return out


def bench_mapping_window(ts, torch, dev, n_faces=1_000_000, steps=5):
    """Mapping window: 12 keyframes (4 each of 320x240, 640x480, 1200x680) of a 1M-face map,
    joint forward + backward with gradients accumulated into shared map buffers.  Plain per-view
    calls vs one batched pass vs the autotuned, graph-captured batched pass."""
    from ts_synth.scenes import Scene, mixed_keyframe_cameras, noise_targets, room_map, trajectory_poses
    pos, col, opa = room_map(5, n_faces)
    cams = mixed_keyframe_cameras(4)
    poses_np = trajectory_poses(1005, len(cams))
    tcs, tds = noise_targets(6, cams)
    m = ts.Map.from_numpy(pos, col, opa, device=dev)
    grad = m.zeros_like()
    poses = ts.poses_tensor(poses_np, device=dev)
    tc = torch.as_tensor(np.concatenate([t.reshape(-1) for t in tcs]), device=dev)
    td = torch.as_tensor(np.concatenate([t.reshape(-1) for t in tds]), device=dev)
    pixels = int(sum(c[4] * c[5] for c in cams))
    off = np.concatenate([[0], np.cumsum(cams[:, 4] * cams[:, 5])]).astype(int)
    out = {"workload": "room 1M faces, 12 keyframes: 4x 320x240, 4x 640x480, 4x 1200x680, fwd+bwd", "pixels": pixels}
    # plain: one plan per keyframe, called one after another
    singles = [ts.MultiViewStep(m, cams[v:v + 1], poses[v:v + 1], tc[3 * off[v]:3 * off[v + 1]], td[off[v]:off[v + 1]],
                                None, grad) for v in range(len(cams))]
    ms_plain = ts.batch.time_ms(lambda: [s.step() for s in singles], iters=steps)
    del singles
    torch.cuda.empty_cache()
    batched = ts.MultiViewStep(m, cams, poses, tc, td, None, grad)
    ms_batched = ts.batch.time_ms(batched.step, iters=steps)
    # where the batched step's time goes: libts records events around each stage on the stream
    names = ts.binding.STAGES
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * len(names))]
    st_ = torch.cuda.current_stream()
    for e in ev:
        e.record(st_)
    ts.ts_set_stage_events(batched.rast.plan, ev)
    stage_ms = np.zeros(len(names))
    for _ in range(steps):
        batched.step()
        torch.cuda.synchronize()
        stage_ms += [ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(len(names))]
    ts.ts_set_stage_events(batched.rast.plan, None)
    stage_ms /= steps
    cnt = batched.rast.counters()
    out["batched_stages_ms"] = {("fused_fwd_loss_bwd" if n == "fwd" else n): float(t) for n, t in zip(names, stage_ms)
                                if n not in ("bwd_raster", "loss")}
    out["batched_counters"] = {k: int(cnt[k]) for k in ("n_visible", "n_pairs", "fwd_contrib")}
    out["batched_path"] = "ts_render_step_l1" if batched.fused else "separate calls"
    del batched
    torch.cuda.empty_cache()
    best, _ = ts.autotune(m, cams, poses, tc, td, grad, tiles=((16, 8), (8, 8), (16, 16), (32, 8)), stages=(64, 128),
                          iters=2, use_cache=False)
    tuned = ts.MultiViewStep(m, cams, poses, tc, td, ts.params_of(best), grad)
    tuned.capture()
    ms_tuned = ts.batch.time_ms(lambda: tuned.run(1, use_graph=True), iters=steps)
    del tuned
    torch.cuda.empty_cache()
    # the full mapping loss of Eq. 15 (0.8 L1 + 0.2 D-SSIM, 0.05 depth, 0.05 normal against sensor
    # normals with the normal map rendered, 1.2 equilateral), same shape, graph-captured
    from ts_synth.scenes import sensor_normals
    tn = torch.as_tensor(sensor_normals(7, cams), device=dev)
    emap = ts.MultiViewStep(m, cams, poses, tc, td, ts.params_of(best), grad, lambda_ssim=0.2, tgt_normal=tn,
                            lambda_norm=0.05, lambda_equi=1.2)
    emap.capture()
    ms_emap = ts.batch.time_ms(lambda: emap.run(1, use_graph=True), iters=steps)
    del emap
    torch.cuda.empty_cache()
    out.update({"plain_per_view_mpix_s": pixels / ms_plain / 1e3, "batched_mpix_s": pixels / ms_batched / 1e3,
                "batched_graph_autotuned_mpix_s": pixels / ms_tuned / 1e3,
                "full_mapping_loss_graph_mpix_s": pixels / ms_emap / 1e3,
                "ms": {"plain": ms_plain, "batched": ms_batched, "batched_graph_autotuned": ms_tuned,
                       "full_mapping_loss_graph": ms_emap}, "autotuned": best})
    return out


def bench_tracking(ts, torch, dev, n_hyp=64, iters=100):
    """Tracking: 64 pose hypotheses of a 640x480 (f = 525) camera on a 150k-face room map,
    100 gradient iterations each, replayed from one captured CUDA graph."""
    from ts_synth.scenes import perturb_pose, room_map, trajectory_poses
    pos, col, opa = room_map(7, 150_000)
    W_, H_, f = 640, 480, 525.0
    cam = np.array([f, f, W_ / 2, H_ / 2, W_, H_])
    gt = trajectory_poses(1007, 8)[2]
    m = ts.Map.from_numpy(pos, col, opa, device=dev)
    # target: the GT render plus noise (sigma 0.02 on colour, 1 % on depth)
    r0 = ts.Rasterizer(cam[None, :], m.n_faces)
    C, D, _ = r0.forward(m, ts.poses_tensor(gt[None, :], device=dev))
    g = torch.Generator(device=dev).manual_seed(8)
    tc = (C + 0.02 * torch.randn(C.shape, generator=g, device=dev)).contiguous()
    td = (D * (1 + 0.01 * torch.randn(D.shape, generator=g, device=dev))).contiguous()
    del r0
    rng = np.random.default_rng(9)
    init = np.stack([perturb_pose(gt, rng) for _ in range(n_hyp)])
    trk = ts.Tracker(m, cam, tc.view(3, H_, W_), td.view(H_, W_), init)
    trk.capture()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    trk.run(iters, use_graph=True)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b)
    e0 = ts.pose_error(init, np.tile(gt, (n_hyp, 1)))
    e1 = ts.pose_error(trk.poses.cpu().numpy(), np.tile(gt, (n_hyp, 1)))
    px = n_hyp * W_ * H_ * iters
    return {"workload": f"640x480 f=525, 150k-face room, {n_hyp} hypotheses x {iters} iterations (graph replay), "
                        "E_track = 0.8 L1 + 0.2 D-SSIM + 0.05 depth L1",
            "mpix_s": px / ms / 1e3, "ms_per_iteration": ms / iters,
            "median_error_before": {"cm": float(np.median(e0[:, 0]) * 100), "deg": float(np.median(e0[:, 1]))},
            "median_error_after": {"cm": float(np.median(e1[:, 0]) * 100), "deg": float(np.median(e1[:, 1]))}}


def bench_pho_loss(ts, torch, rast, tgt_c, tgt_d, flush, stream, pixels, alu_peak, sm_max, n_sm, reps=10):
    """The fused photometric loss of Eq. 8-10 ((1 - 0.2) L1 + 0.2 D-SSIM on colour, 0.05 L1 on depth)
    with its image gradients, on the bench's rendered views; device time with the L2 flushed."""
    call = (rast.plan, rast.ws, rast.color, rast.depth, tgt_c, tgt_d, 0.2, 0.05, rast.loss_v, rast.dC, rast.dD)
    for _ in range(3):
        ts.ts_pho_loss(*call)
    ms = []
    for _ in range(reps):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ts.ts_pho_loss(*call)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    t = float(np.median(ms))
    ach = FLOPS_PHO * 3 * pixels / (t / 1e3) / 1e12
    return {"workload": WORKLOAD.split(",")[0] + f", {rast.V} rendered views vs noise targets", "ms": t,
            "mpix_s": pixels / (t / 1e3) / 1e6,
            "roofline": {"kernel": "k_pho_tile", "bound": "alu", "achieved": ach, "peak": alu_peak,
                         "unit": "TFLOP/s", "frac": ach / alu_peak, "traffic": None,
                         "peak_source": f"derived: {n_sm} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz",
                         "work": f"{3 * pixels} pixel-channels x {FLOPS_PHO:.0f} flops"}}


def bench_variants(ts, torch, sc, m, poses, tgt_c, tgt_d, flush, stream, params, reps=5):
    """The bench step under each raster switch (same workload, L2 flushed, CUDA events): the normal
    map of Eq. 12 with its gradient, the map statistics of Sec. 3.4 (forward coverage counting plus
    ts_face_stats and ts_covisibility), the min-opacity faces and the per-face sigma variant."""
    from ts_synth.scenes import sensor_normals
    tn = torch.as_tensor(sensor_normals(7, sc.cams), device=m.pos.device)
    sigma = torch.full((sc.n_faces,), 0.5, dtype=torch.float32, device=m.pos.device)
    ms_sig = ts.Map(m.pos, m.col, m.opa, None, sigma)
    out = {"workload": WORKLOAD.split(",")[0] + ", the bench step with one switch on"}
    cases = (("plain", 0), ("normals", ts.TS_FLAG_NORMALS), ("stats", ts.TS_FLAG_STATS),
             ("min_opacity", ts.TS_FLAG_MIN_OPACITY), ("face_sigma", ts.TS_FLAG_FACE_SIGMA))
    for name, flag in cases:
        p = ts.batch.params_of({"tile_w": params.tile_w, "tile_h": params.tile_h,
                                "tris_per_stage": params.tris_per_stage})
        p.flags = flag
        r = ts.Rasterizer(sc.cams, sc.n_faces, p)
        mm = ms_sig if flag == ts.TS_FLAG_FACE_SIGMA else m
        g = mm.zeros_like()

        def step():
            g.pos.zero_(); g.col.zero_(); g.opa.zero_()
            r.forward(mm, poses)
            r.l1_loss(tgt_c, tgt_d, 0.05)
            dN = r.normal_loss(tn, 0.05)[1] if flag == ts.TS_FLAG_NORMALS else None
            r.backward(r.dC, r.dD, None, g, dN=dN)
            r.pose_grad()
            if flag == ts.TS_FLAG_STATS:
                st = r.face_stats()
                r.covisibility(st["visible"])

        for _ in range(2):
            step()
        ms = []
        for _ in range(reps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        out[name] = {"ms_per_step": float(np.median(ms)), "mpix_s": sc.pixels() / (float(np.median(ms)) / 1e3) / 1e6}
        del r, g
        torch.cuda.empty_cache()
    return out


def bench_serving(ts, torch, dev, rates=(200, 500, 1000, 2000), seconds=10.0, n_faces=2_000_000, drain=5.0):
    """Serving: device-resident 2M-face map; Poisson arrivals of render (one forward) and track
    (10 pose iterations) requests, resolutions uniform over 256x256, 640x480 and 1200x680, poses on
    a seeded trajectory, 10 s of arrivals per rate.  Each stream is served twice: by the continuous
    batching server and by the plain one-request-at-a-time loop (the baseline), each run ending 5 s
    after the last arrival; requests unfinished by then are counted as not served (and as infinitely
    late in the percentiles).  At 1000 req/s the served run is repeated with the plain L1 tracking
    loss (lambda_ssim = 0) to show the D-SSIM term's share."""
    from ts_synth.scenes import perturb_pose, request_stream, room_map, trajectory_poses
    res = ((256, 256, 256.0), (640, 480, 525.0), (1200, 680, 600.0))
    pos, col, opa = room_map(6, n_faces)
    m = ts.Map.from_numpy(pos, col, opa, device=dev)
    n_poses = 16
    gts = trajectory_poses(1006, n_poses)
    targets = {}
    for (W_, H_, f) in res:
        r = ts.Rasterizer(np.array([[f, f, W_ / 2, H_ / 2, W_, H_]]), m.n_faces)
        for k in range(n_poses):
            C, D, _ = r.forward(m, ts.poses_tensor(gts[k][None, :], device=dev))
            targets[(W_, H_, k)] = (C.clone().view(3, H_, W_), D.clone().view(H_, W_))
        del r
    out = {"workload": f"2M-face room, Poisson render/track 50/50, {seconds:.0f} s of arrivals per rate, resolutions "
                       f"256x256 / 640x480 / 1200x680, track = 10 pose iterations (0.8 L1 + 0.2 D-SSIM + 0.05 depth); "
                       f"runs end {drain:.0f} s after the last arrival; each run after an untimed 0.5 s warm-up stream"}

    def stream_of(rate, seed):
        rng = np.random.default_rng(seed)
        reqs = []
        for i, d in enumerate(request_stream(6 + rate, rate, seconds, resolutions=res, n_poses=n_poses)):
            W_, H_, f = d["W"], d["H"], d["f"]
            cam = np.array([f, f, W_ / 2, H_ / 2, W_, H_])
            gt = gts[d["pose_index"]]
            if d["kind"] == "render":
                reqs.append(ts.Request(i, "render", cam, gt, d["t"]))
            else:
                tc, td = targets[(W_, H_, d["pose_index"])]
                reqs.append(ts.Request(i, "track", cam, perturb_pose(gt, rng, 0.02, 1.0), d["t"], tc, td))
        return reqs

    # an untimed warm-up stream before each timed one: every kind and resolution, so that first-use
    # costs (plans, allocations) stay out of the latencies
    warm_seconds = 0.5

    def warm_stream():
        return [r for r in stream_of(200, 7) if r.t_arrival < warm_seconds]

    def served(rate, lambda_ssim=0.2):
        srv = ts.Server(m, max_views=32, max_pixels=16_000_000, track_iters=10, lambda_ssim=lambda_ssim)
        srv.run(warm_stream(), realtime=False, drain_seconds=drain)
        srv.stats.update(steps=0, pixels=0, rejected_for_memory=0)
        reqs = stream_of(rate, 6)
        srv.run(reqs, realtime=True, drain_seconds=drain)
        st = ts.latency_stats(reqs, srv.stats["seconds"])
        st["steps"] = srv.stats["steps"]
        del srv
        torch.cuda.empty_cache()
        return st

    for rate in rates:
        st = {"served": served(rate)}
        ts.serve_plain(m, warm_stream(), track_iters=10, realtime=False, drain_seconds=drain)
        reqs = stream_of(rate, 6)
        secs = ts.serve_plain(m, reqs, track_iters=10, realtime=True, drain_seconds=drain)
        st["plain"] = ts.latency_stats(reqs, secs)
        torch.cuda.empty_cache()
        st["served_over_plain_mpix"] = st["served"]["mpix_s"] / max(st["plain"]["mpix_s"], 1e-9)
        out[f"{rate}_req_s"] = st
    out["1000_req_s_served_l1_only"] = served(1000, lambda_ssim=0.0)
    return out


def bench_e2e(ts, torch, dev, rast, m, poses, tgt_c, tgt_d, grad, stream, pixels, args):
    """The step end to end through the public API, as a training loop with a double-buffered input
    pipeline runs it: every step copies its inputs (map, poses, targets) from pinned host memory
    and reads its results (map gradients, pose gradients, per-view loss) back into pinned host
    memory.  Step k+1's inputs cross on a copy stream while step k computes, and step k's results
    cross on another while step k+1 computes; each buffer is reused only after the step that read
    it has finished.  Each step's device work is captured once per input buffer in a CUDA graph and
    replayed (launched call by call with --eager).  The timed region spans all K steps: the first
    step's input copy and the last step's result copy are inside it.  L2 is not flushed: every
    step's inputs (286 MB at the default workload) are fresh copies, more than the 129 MB L2 holds,
    as a training loop has them."""
    h_in = [t.cpu().pin_memory() for t in (m.pos, m.col, m.opa, poses, tgt_c, tgt_d)]
    h_out = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in (grad.pos, grad.col, grad.opa)]
    h_out += [torch.empty(rast.V, 6).pin_memory(), torch.empty(rast.V).pin_memory()]
    h2d = sum(t.numel() * t.element_size() for t in h_in)
    d2h = sum(t.numel() * t.element_size() for t in h_out)
    d_in = [[torch.empty_like(t, device=dev) for t in h_in] for _ in range(2)]
    d_grad = [m.zeros_like() for _ in range(2)]
    d_tau = [torch.empty(rast.V, 6, device=dev) for _ in range(2)]
    d_loss = [torch.empty(rast.V, device=dev) for _ in range(2)]
    up, down = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    K = max(10, args.steps)

    def body(separate, b):
        # one step on input buffer b: the device work a training loop launches each step
        pos, col, opa, ps, tc, td = d_in[b]
        dm, g = ts.Map(pos, col, opa), d_grad[b]
        g.pos.zero_(); g.col.zero_(); g.opa.zero_()
        if separate:
            rast.forward(dm, ps)
            rast.l1_loss(tc, td, 0.05)
            rast.backward(rast.dC, rast.dD, None, g)
        else:
            rast.project(dm, ps)
            rast.bin()
            rast.step_l1(tc, td, 0.05, g)
        rast.pose_grad(out=d_tau[b])
        d_loss[b].copy_(rast.loss_v)

    def capture(separate):
        # the step captured once per input buffer and replayed every step (unless --eager)
        if args.eager:
            return None
        graphs = []
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            for b in range(2):
                body(separate, b)
                gr = torch.cuda.CUDAGraph()
                with torch.cuda.graph(gr, stream=side):
                    body(separate, b)
                graphs.append(gr)
        stream.wait_stream(side)
        torch.cuda.synchronize()
        return graphs

    def run(separate, graphs):
        comp_done = [None, None]
        out_read = [None, None]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        up.wait_stream(stream)
        for k in range(K):
            b = k % 2
            if comp_done[b] is not None:
                up.wait_event(comp_done[b])  # step k-2 has finished reading buffer b
            with torch.cuda.stream(up):
                for d, h in zip(d_in[b], h_in):
                    d.copy_(h, non_blocking=True)
            ready = torch.cuda.Event()
            ready.record(up)
            stream.wait_event(ready)
            if out_read[b] is not None:
                stream.wait_event(out_read[b])  # step k-2's results have left buffer b
            with torch.cuda.stream(stream):
                if graphs is None:
                    body(separate, b)
                else:
                    graphs[b].replay()
            g = d_grad[b]
            comp_done[b] = torch.cuda.Event()
            comp_done[b].record(stream)
            down.wait_event(comp_done[b])
            with torch.cuda.stream(down):
                for h, d in zip(h_out, (g.pos, g.col, g.opa, d_tau[b], d_loss[b])):
                    h.copy_(d, non_blocking=True)
            out_read[b] = torch.cuda.Event()
            out_read[b].record(down)
        stream.wait_stream(down)
        stream.wait_stream(up)
        t1.record(stream)
        t1.synchronize()
        return t0.elapsed_time(t1) / K

    vals = {}
    for separate in ((True,) if args.separate else (False, True)):
        graphs = capture(separate)
        run(separate, graphs)  # warm-up of the pipeline
        vals["ts_render_fwd + ts_l1_loss + ts_render_bwd" if separate else "ts_render_step_l1"] = \
            pixels / (run(separate, graphs) / 1e3) / 1e6
    best = max(vals, key=vals.get)
    return {"value": vals[best], "unit": "Mpix/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "path": best, "by_path": vals, "steps": K,
            "pipeline": "inputs of step k+1 cross while step k computes; results of step k cross while step k+1 "
                        "computes; first input copy and last result copy inside the timed region",
            "l2": f"not flushed: each step's inputs ({h2d / 1e6:.0f} MB) are fresh host copies larger than L2",
            "launch": "eager" if args.eager else "each step's device work replayed from a CUDA graph per input buffer"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    sc = scene(args)
    steps = []
    base = None
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(sc, time_budget_s=0.0, single_thread=False)
        if i >= args.warmup:
            steps.append(W * H / r["value"] / 1e6)
        base = r
    t = float(np.mean(steps))
    val = W * H / t / 1e6
    line = {"impl": "reference", "metric": "Mpix/s fwd+bwd raster", "value": val, "unit": "Mpix/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (oracle: one view per step)", "views_per_step": 1},
            "cpu_baseline": {"kind": "oracle", "cores": base["cores"], "sample": base["sample"], "value": val,
                             "unit": "Mpix/s"},
            "e2e": {"value": val, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    import paper_2605_31419_gb300 as ts

    sc = scene(args)
    tw, th = (int(x) for x in args.tile.split("x"))
    params = ts.ts_default_params(tile_w=tw, tile_h=th, tris_per_stage=args.stage)
    rast = ts.Rasterizer(sc.cams, sc.n_faces, params)
    m = ts.Map.from_numpy(sc.pos, sc.col, sc.opa, device=dev)
    poses = ts.poses_tensor(sc.poses, device=dev)
    tgt_c = torch.as_tensor(np.concatenate([t.reshape(-1) for t in sc.tgt_color]), device=dev)
    tgt_d = torch.as_tensor(np.concatenate([t.reshape(-1) for t in sc.tgt_depth]), device=dev)
    grad = m.zeros_like()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # per-stage events (forced into existence by one record each)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * len(ts.binding.STAGES))]
    for e in ev:
        e.record(stream)

    def step(r=rast, mp=m, ps=poses, tc=tgt_c, td=tgt_d, g=grad):
        g.pos.zero_(); g.col.zero_(); g.opa.zero_()
        if args.separate:
            r.forward(mp, ps)
            r.l1_loss(tc, td, 0.05)
            r.backward(r.dC, r.dD, None, g)
        else:
            r.project(mp, ps)
            r.bin()
            r.step_l1(tc, td, 0.05, g)
        r.pose_grad()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    cnt = rast.counters()
    # the step's launches captured once into a CUDA graph, replayed for the timed steps (the launch
    # gaps of an eager sequence of ~15 kernels go); --eager times the launches one by one
    graph = None
    if not args.eager:
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            step()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=side):
                step()
        stream.wait_stream(side)
        torch.cuda.synchronize()
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize()

    def timed_steps(k, run, with_stages):
        ms, st_ms = [], np.zeros(len(ts.binding.STAGES))
        if with_stages:
            ts.ts_set_stage_events(rast.plan, ev)
        for _ in range(k):
            flush.fill_(1.0)
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            run()
            s1.record(stream)
            s1.synchronize()
            ms.append(s0.elapsed_time(s1))
            if with_stages:
                st_ms += [ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(len(ts.binding.STAGES))]
        if with_stages:
            ts.ts_set_stage_events(rast.plan, None)
        return ms, st_ms / max(k, 1)

    sampler = ClockSampler(dev.index or 0)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    step_ms, stage_ms = timed_steps(args.steps, graph.replay if graph is not None else step, graph is None)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    t_step = max_over_ranks(float(np.sum(step_ms)) / args.steps / 1e3, dev if world > 1 else None)
    # stage times (CUDA events recorded by libts around each stage) from eager steps outside the
    # timed region when the timed steps are graph replays
    eager_ms = None
    if graph is not None:
        e_ms, stage_ms = timed_steps(max(3, args.steps // 2), step, True)
        eager_ms = float(np.mean(e_ms))
    pixels = sc.pixels()
    value = job_value(pixels, world, t_step)

    # -- plain per-view: the same work, one view per call sequence (its own plan) ------------------
    plain_ms = None
    if rank == 0:
        single = ts.Rasterizer(sc.cams[:1], sc.n_faces, params)
        P1 = W * H
        for _ in range(2):
            for v in range(sc.n_views):
                step(single, m, poses[v:v + 1], tgt_c[3 * P1 * v:3 * P1 * (v + 1)], tgt_d[P1 * v:P1 * (v + 1)])
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(1.0)
        a0.record(stream)
        for v in range(sc.n_views):
            step(single, m, poses[v:v + 1], tgt_c[3 * P1 * v:3 * P1 * (v + 1)], tgt_d[P1 * v:P1 * (v + 1)])
        a1.record(stream)
        a1.synchronize()
        plain_ms = a0.elapsed_time(a1)
        del single

    # -- end to end: pinned host inputs in, results out, through the same API ---------------------
    e2e = None
    if rank == 0:
        e2e = bench_e2e(ts, torch, dev, rast, m, poses, tgt_c, tgt_d, grad, stream, pixels, args)

    if rank == 0:
        peaks, peak_src = measured_peaks()
        names = ts.binding.STAGES
        dom = int(np.argmax(stage_ms))
        sm_max = float(peaks.get("sm_max_mhz", 2070.0))
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        alu_peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12  # FP32 FMA lanes x 2 flops x clock (TFLOP/s)
        if names[dom] in ("bwd_raster", "fwd"):
            fused = names[dom] == "fwd" and not args.separate  # the fwd stage times ts_render_step_l1
            per = (FLOPS_FWD + FLOPS_BWD) if fused else (FLOPS_BWD if names[dom] == "bwd_raster" else FLOPS_FWD)
            contrib = cnt["bwd_contrib"] if names[dom] == "bwd_raster" else cnt["fwd_contrib"]
            flops = per * contrib
            ach = flops / (stage_ms[dom] / 1e3) / 1e12
            kernel = "k_render_step" if fused else f"k_render_{'bwd' if names[dom] == 'bwd_raster' else 'fwd'}"
            per_view = {"k_render_step": STEP_TRAFFIC_PER_VIEW}.get(kernel)
            traffic = (per_view * sc.n_views if per_view is not None and args.tile == "16x8"
                       and args.stage == 64 else None)
            roof = {"kernel": kernel, "bound": "alu",
                    "achieved": ach, "peak": alu_peak, "unit": "TFLOP/s", "frac": ach / alu_peak,
                    "traffic": traffic,
                    "peak_source": f"derived: {n_sm} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz",
                    "work": f"{contrib} (pixel, face) contributions x {per:.0f} flops"}
            if traffic is not None:
                # the same launch against the memory roofline: its measured DRAM bytes over its time
                gbs = traffic / (stage_ms[dom] / 1e3) / 1e9
                roof.update({"hbm_achieved_gbs": gbs, "hbm_peak_gbs": peaks["hbm_gbs"],
                             "hbm_frac": gbs / peaks["hbm_gbs"], "hbm_peak_source": peak_src})
        else:
            roof = {"kernel": names[dom], "bound": "hbm", "achieved": None, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": None, "traffic": None}
        # setup + project, binning (tile counts, scan (3), places, warp and CTA segment sorts, the
        # warp sort also writing the ranges), then either forward, loss (2) and raster backward, or
        # the fused step and its loss reduction; the chain-rule pass (one kernel from 8 views on,
        # two below), pose reduction
        launches = 2 + 7 + (1 + 2 + 1 if args.separate else 2) + (1 if sc.n_views >= 8 else 2) + 1
        line = {
            "metric": "Mpix/s fwd+bwd raster", "value": value, "unit": "Mpix/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "views": sc.n_views, "W": W, "H": H, "faces": sc.n_faces,
                       "path": ("ts_render_fwd + ts_l1_loss + ts_render_bwd" if args.separate
                                else "ts_render_step_l1 (forward, L1 loss and backward in one pass per tile)"),
                       "tile": args.tile, "tris_per_stage": args.stage, "l2": "flushed (256 MB write) between steps",
                       "launch": "eager" if graph is None else "CUDA graph replay of the step's launches",
                       "eager_ms_per_step": eager_ms,
                       "parallelism": f"replicas x{world}"},
            "plain_per_view": {"value": pixels / (plain_ms / 1e3) / 1e6 if plain_ms else None, "unit": "Mpix/s",
                               "ms_per_step": plain_ms},
            "stages_ms": {n: float(t) for n, t in zip(names, stage_ms)},
            "counters": {k: int(v) for k, v in cnt.items() if isinstance(v, (int, np.integer))},
            "roofline": roof, "peaks": peak_src, "e2e": e2e, "gpu_launches": launches * args.steps,
            "clocks": clocks,
        }
        line["triangles_per_s"] = {
            "face_views": sc.n_faces * sc.n_views / t_step,
            "visible_records": cnt["n_visible"] / t_step,
            "tile_pairs": cnt["n_pairs"] / t_step,
            "note": "face_views: input faces x views per second of step time; visible_records: (view, face) "
                    "records that survived culling per second; tile_pairs: (tile, face) pairs per second"}
        line["pho_loss"] = bench_pho_loss(ts, torch, rast, tgt_c, tgt_d, flush, stream, pixels, alu_peak, sm_max,
                                          n_sm)
        line["c1_plain_single_view"] = bench_c1(ts, torch, dev, flush, stream)
        if not args.no_extras:
            del rast
            torch.cuda.empty_cache()
            line["variants"] = bench_variants(ts, torch, sc, m, poses, tgt_c, tgt_d, flush, stream, params)
            torch.cuda.empty_cache()
            line["mapping_window"] = bench_mapping_window(ts, torch, dev)
            line["tracking"] = bench_tracking(ts, torch, dev)
            torch.cuda.empty_cache()
            line["serving"] = bench_serving(ts, torch, dev)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(sc)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
