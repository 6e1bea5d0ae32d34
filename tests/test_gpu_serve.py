"""Serving loop (GPU): continuous batching of render and track requests on a resident map.

Each request's result is the same alone and in the mix: renders bit for bit (the forward pass of a
view does not depend on the other views of its batch), tracked poses within 1e-4 (the pose
gradient's atomic sums make the last bits order-dependent, and Adam normalises each step)."""
import numpy as np
import pytest

from ts_synth.scenes import perturb_pose, request_stream, room_map, trajectory_poses

pytestmark = pytest.mark.gpu

RES = ((64, 48, 60.0), (96, 64, 80.0), (120, 68, 60.0))


def _requests(seed, n_poses, targets, rate=400.0, duration=0.1):
    rng = np.random.default_rng(seed)
    gts = trajectory_poses(2000 + seed, n_poses)
    reqs = []
    import paper_2605_31419_gb300 as ts
    for i, d in enumerate(request_stream(seed, rate, duration, resolutions=RES, n_poses=n_poses)):
        W, H, f = d["W"], d["H"], d["f"]
        cam = np.array([f, f, W / 2, H / 2, W, H])
        gt = gts[d["pose_index"]]
        if d["kind"] == "render":
            reqs.append(ts.Request(i, "render", cam, gt, d["t"]))
        else:
            tc, td = targets[(W, H, d["pose_index"])]
            reqs.append(ts.Request(i, "track", cam, perturb_pose(gt, rng, 0.02, 1.0), d["t"], tc, td))
    return reqs


def test_results_alone_equal_results_in_the_mix():
    import torch
    import paper_2605_31419_gb300 as ts
    pos, col, opa = room_map(11, 40000, side_lo=0.05, side_hi=0.12)
    m = ts.Map.from_numpy(pos, col, opa)
    n_poses = 6
    gts = trajectory_poses(2000 + 3, n_poses)
    targets = {}
    for (W, H, f) in RES:
        cam = np.array([[f, f, W / 2, H / 2, W, H]])
        r = ts.Rasterizer(cam, m.n_faces)
        for k in range(n_poses):
            C, D, _ = r.forward(m, ts.poses_tensor(gts[k][None, :]))
            targets[(W, H, k)] = (C.clone().view(3, H, W), D.clone().view(H, W))
    reqs = _requests(3, n_poses, targets)
    assert sum(r.kind == "track" for r in reqs) >= 2 and sum(r.kind == "render" for r in reqs) >= 2
    srv = ts.Server(m, max_views=16, max_pixels=16 * 120 * 68, track_iters=10)
    mixed = srv.run(reqs, realtime=False)
    torch.cuda.synchronize()
    assert all(r.t_done >= 0 for r in mixed)
    for r in mixed:
        alone = ts.Server(m, max_views=2, max_pixels=2 * 120 * 68, track_iters=10)
        r2 = ts.Request(r.rid, r.kind, r.cam, r.pose, 0.0, r.target_color, r.target_depth)
        alone.run([r2], realtime=False)
        torch.cuda.synchronize()
        if r.kind == "render":
            assert torch.equal(r.color, r2.color) and torch.equal(r.depth, r2.depth)
        else:
            assert r.iters_done == r2.iters_done == 10
            assert np.allclose(r.pose_out.cpu().numpy(), r2.pose_out.cpu().numpy(), atol=1e-4)


def test_admission_waits_for_memory():
    """A request that does not fit the step's budget waits and is served later, not dropped."""
    import torch
    import paper_2605_31419_gb300 as ts
    pos, col, opa = room_map(11, 20000)
    m = ts.Map.from_numpy(pos, col, opa)
    gts = trajectory_poses(2003, 4)
    cam = np.array([60.0, 60.0, 60.0, 34.0, 120, 68])
    reqs = [ts.Request(i, "render", cam, gts[i % 4], 0.0) for i in range(6)]
    srv = ts.Server(m, max_views=2, max_pixels=2 * 120 * 68)
    out = srv.run(reqs, realtime=False)
    torch.cuda.synchronize()
    assert all(r.color is not None for r in out)
    assert srv.stats["steps"] >= 3 and srv.stats["rejected_for_memory"] >= 2
    st = ts.latency_stats(out, srv.stats["seconds"])
    assert st["completed"] == 6 and st["render"]["p99_ms"] >= st["render"]["p50_ms"]


def test_forward_only_plan_renders_the_same_images():
    """TS_FLAG_FORWARD_ONLY (the server's render plans) changes what is stored, not what is
    rendered: colour, depth and opacity bit for bit against a full plan, on one view and on three
    views of uneven size."""
    import torch
    import paper_2605_31419_gb300 as ts
    from ts_synth.scenes import random_triangles_scene
    pos, col, opa = room_map(3, 20000)
    cams = np.array([[70.0, 70.0, 50.0, 37.5, 100, 75], [40.0, 40.0, 28.5, 16.5, 57, 33],
                     [90.0, 90.0, 61.0, 40.0, 123, 81]])
    sc1 = random_triangles_scene(seed=1)
    cases = [(ts.Map.from_numpy(sc1.pos, sc1.col, sc1.opa), sc1.cams, sc1.poses),
             (ts.Map.from_numpy(pos, col, opa), cams, trajectory_poses(1003, 3))]
    for m, cm, ps in cases:
        full = ts.Rasterizer(cm, m.n_faces)
        fwd = ts.Rasterizer(cm, m.n_faces, ts.ts_default_params(flags=ts.TS_FLAG_FORWARD_ONLY))
        assert fwd.ws_bytes < full.ws_bytes
        a = [t.clone() for t in full.forward(m, ts.poses_tensor(ps))]
        b = fwd.forward(m, ts.poses_tensor(ps))
        torch.cuda.synchronize()
        for x, y in zip(a, b):
            assert torch.equal(x, y)
        assert fwd.counters()["status"] == "TS_OK"


def test_plain_baseline_gives_the_served_results():
    """serve_plain (one request at a time, single-view plans) returns the renders of the batching
    server bit for bit and its tracked poses within 1e-4."""
    import torch
    import paper_2605_31419_gb300 as ts
    pos, col, opa = room_map(11, 40000, side_lo=0.05, side_hi=0.12)
    m = ts.Map.from_numpy(pos, col, opa)
    n_poses = 6
    gts = trajectory_poses(2000 + 5, n_poses)
    targets = {}
    for (W, H, f) in RES:
        r = ts.Rasterizer(np.array([[f, f, W / 2, H / 2, W, H]]), m.n_faces)
        for k in range(n_poses):
            C, D, _ = r.forward(m, ts.poses_tensor(gts[k][None, :]))
            targets[(W, H, k)] = (C.clone().view(3, H, W), D.clone().view(H, W))
    a = _requests(5, n_poses, targets)
    b = _requests(5, n_poses, targets)
    srv = ts.Server(m, max_views=16, max_pixels=16 * 120 * 68, track_iters=10)
    srv.run(a, realtime=False)
    secs = ts.serve_plain(m, b, track_iters=10, realtime=False)
    torch.cuda.synchronize()
    st = ts.latency_stats(b, secs)
    assert st["not_served"] == 0 and st["completed"] == len(b)
    for x, y in zip(a, b):
        if x.kind == "render":
            assert torch.equal(x.color, y.color) and torch.equal(x.depth, y.depth)
        else:
            assert y.iters_done == 10
            assert np.allclose(x.pose_out.cpu().numpy(), y.pose_out.cpu().numpy(), atol=1e-4)
