"""The fused L1 step (ts_render_step_l1) against the separate calls and the oracle (needs a GB300).

Against ts_render_fwd + ts_l1_loss + ts_render_bwd on the same inputs: the images and the loss's
image gradients bit for bit (the same per-pixel arithmetic), the per-view loss to float rounding
(other partial sums).  Against the oracle: the loss, the map gradients and the pose gradient with
the tolerances of the separate path.  The scenes cover tiles whose lists span many stages (the
backward stages them again) and tiles whose pixels all stop early (a prefetched stage replaced the
one before the last).
"""
import numpy as np
import pytest

from harness import assert_grad, assert_images, assert_pose_grad, gpu_run, oracle_run, pack_targets, params_pair
from ts_synth.scenes import random_triangles_scene, room_map, room_scene, trajectory_poses, noise_targets, Scene

pytestmark = pytest.mark.gpu


def _ragged_room():
    pos, col, opa = room_map(3, 20000)
    cams = np.array([[70.0, 70.0, 50.0, 37.5, 100, 75], [40.0, 40.0, 28.5, 16.5, 57, 33],
                     [90.0, 90.0, 61.0, 40.0, 123, 81]])
    sc = Scene(pos, col, opa, None, cams, trajectory_poses(1003, 3))
    sc.tgt_color, sc.tgt_depth = noise_targets(4, cams)
    return sc


SCENES = {
    "c1": lambda: random_triangles_scene(seed=1),
    "ragged_room": _ragged_room,
    # lists of ~1500 faces per tile: 24 stages of 64, all but the last two staged again
    "long_lists": lambda: random_triangles_scene(seed=6, n_faces=3000, W=48, H=32, f=40.0, side_lo=0.6,
                                                 side_hi=1.2, z_lo=1.0, z_hi=2.0),
    # faint faces, lists of ~100: no pixel stops, the last two stages are both still staged
    "translucent": lambda: random_triangles_scene(seed=8, n_faces=150, W=64, H=48, f=60.0, side_lo=0.6,
                                                  side_hi=1.2, z_lo=1.0, z_hi=2.0, opa_lo=0.02, opa_hi=0.05),
    # nearly opaque faces: pixels stop after a few faces, most tiles end the forward early
    "opaque": lambda: random_triangles_scene(seed=7, n_faces=4000, W=96, H=64, f=80.0, side_lo=0.3, side_hi=0.8,
                                             opa_lo=0.995, opa_hi=1.0),
}


def step_run(sc, p, lambda_dep=0.05, pair_capacity=0):
    import torch
    import paper_2605_31419_gb300 as ts
    pair_capacity = pair_capacity or getattr(sc, "pair_capacity", 0)
    rast = ts.Rasterizer(sc.cams, sc.n_faces, p, pair_capacity=pair_capacity)
    m = ts.Map.from_numpy(sc.pos, sc.col, sc.opa, sc.faces)
    poses = ts.poses_tensor(sc.poses)
    tc, td = pack_targets(sc)
    tc = torch.as_tensor(tc, dtype=torch.float32, device="cuda")
    td = torch.as_tensor(td, dtype=torch.float32, device="cuda")
    rast.project(m, poses)
    rast.bin()
    g = m.zeros_like()
    loss = rast.step_l1(tc, td, lambda_dep, g, loss_grads=True)
    dtau = rast.pose_grad()
    torch.cuda.synchronize()
    f = lambda t: t.cpu().numpy().astype(np.float64)  # noqa: E731
    return dict(color=f(rast.color), depth=f(rast.depth), alpha=f(rast.alpha), loss_v=f(loss), dC=f(rast.dC),
                dD=f(rast.dD), dpos=f(g.pos).T, dcol=f(g.col).T, dopa=f(g.opa), dtau=f(dtau),
                counters=rast.counters())  # raises on a latched device error


@pytest.mark.parametrize("name", list(SCENES))
def test_step_matches_separate_calls_and_oracle(oracle, name):
    sc = SCENES[name]()
    p, po = params_pair()
    s = step_run(sc, p, pair_capacity=1_000_000)
    assert s["counters"]["status"] == "TS_OK"
    g = gpu_run(sc, p, pair_capacity=1_000_000)
    for k in ("color", "depth", "alpha", "dC", "dD"):
        assert np.array_equal(s[k], g[k]), f"{k} differs from the separate calls"
    assert_images(s["loss_v"], g["loss_v"], "loss vs separate", atol=1e-7, rtol=1e-6)
    assert s["counters"]["fwd_contrib"] == s["counters"]["bwd_contrib"] == g["counters"]["bwd_contrib"] > 0
    r = oracle_run(oracle, sc, po)
    assert_images(s["loss_v"], r["loss_v"], "loss", atol=1e-6, rtol=1e-5)
    assert_grad(s["dpos"], r["dpos"], "dpos")
    assert_grad(s["dcol"], r["dcol"], "dcol")
    assert_grad(s["dopa"], r["dopa"], "dopa")
    assert_pose_grad(s["dtau"], r["dtau"], r["dtau_abs"])


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 8)], ids=lambda t: f"{t[0]}x{t[1]}")
def test_step_tiles_and_persistent(oracle, tile):
    import paper_2605_31419_gb300 as ts
    sc = SCENES["c1"]()
    for flags in (0, ts.TS_FLAG_PERSISTENT):
        p, po = params_pair(tile_w=tile[0], tile_h=tile[1], flags=flags)
        s = step_run(sc, p)
        g = gpu_run(sc, p)
        for k in ("color", "dC", "dD"):
            assert np.array_equal(s[k], g[k]), k
        r = oracle_run(oracle, sc, po)
        assert_grad(s["dpos"], r["dpos"], "dpos")
        assert_grad(s["dopa"], r["dopa"], "dopa")


def test_step_with_map_statistics(oracle):
    """With TS_FLAG_STATS the fused step counts each face's blended pixels (in the shared memory
    its backward later uses for the rings): the same counts as the separate forward."""
    import torch
    import paper_2605_31419_gb300 as ts
    sc = _ragged_room()
    p, po = params_pair(flags=ts.TS_FLAG_STATS)
    rast = ts.Rasterizer(sc.cams, sc.n_faces, p)
    m = ts.Map.from_numpy(sc.pos, sc.col, sc.opa, sc.faces)
    poses = ts.poses_tensor(sc.poses)
    tc, td = pack_targets(sc)
    tc = torch.as_tensor(tc, dtype=torch.float32, device="cuda")
    td = torch.as_tensor(td, dtype=torch.float32, device="cuda")
    rast.forward(m, poses)
    sep = rast.face_stats()
    sep = {k: v.cpu().numpy() for k, v in sep.items()}
    rast.project(m, poses)
    rast.bin()
    g = m.zeros_like()
    rast.step_l1(tc, td, 0.05, g)
    fused = {k: v.cpu().numpy() for k, v in rast.face_stats().items()}
    assert sep["coverage"].sum() > 0
    for k in ("coverage", "area", "visible", "n_visible"):
        assert np.array_equal(fused[k], sep[k]), k
    r = oracle_run(oracle, sc, po)
    assert_grad(g.pos.cpu().numpy().astype(np.float64).T, r["dpos"], "dpos")


@pytest.mark.parametrize("case", ["empty", "all_culled", "single_bg", "offscreen_partial", "sigma1", "opaque_stack"])
def test_step_edge_cases(oracle, case):
    """The fused step on the separate path's edge cases: the same images and loss gradients as the
    separate calls, and the oracle's gradients."""
    from test_gpu_parity import _single
    kw = {}
    if case == "empty":
        sc = _single(np.zeros((0, 3)))
    elif case == "all_culled":
        sc = _single([[0, 0, -1], [1, 0, -1], [0, 1, -1], [0, 0, 0.001], [1, 0, 0.001], [0, 1, 0.001]])
    elif case == "single_bg":
        sc = _single([[-0.5, -0.4, 1.5], [0.6, -0.2, 2.0], [0.0, 0.5, 1.8]])
        kw = dict(bg=(0.2, 0.4, 0.6))
    elif case == "offscreen_partial":
        sc = _single([[-1.5, -0.4, 1.5], [0.6, -1.2, 2.0], [0.0, 0.5, 1.8], [0.2, 0.2, 1.0], [3.0, 0.3, 1.0],
                      [0.4, 2.0, 1.0]])
    elif case == "sigma1":
        sc = random_triangles_scene(seed=8, n_faces=300, W=48, H=36, f=40.0)
        kw = dict(sigma=1.0)
    else:
        z = np.array([1.0, 2.0, 4.0, 8.0, 0.5, 16.0])
        tri = np.array([[-0.3, -0.3], [0.4, -0.3], [-0.3, 0.35]])
        sc = _single([[x * zz, y * zz, zz] for zz in z for (x, y) in tri])
        sc.opa[:] = 0.9
    p, po = params_pair(**kw)
    s = step_run(sc, p)
    g = gpu_run(sc, p)
    for k in ("color", "depth", "alpha", "dC", "dD"):
        assert np.array_equal(s[k], g[k]), k
    assert_images(s["loss_v"], g["loss_v"], "loss vs separate", atol=1e-7, rtol=1e-6)
    r = oracle_run(oracle, sc, po)
    assert_images(s["loss_v"], r["loss_v"], "loss", atol=1e-6, rtol=1e-5)
    if sc.n_faces:
        assert_grad(s["dpos"], r["dpos"], "dpos")
        assert_grad(s["dcol"], r["dcol"], "dcol")
        assert_grad(s["dopa"], r["dopa"], "dopa")


# ------------------------------------------------------------ the benchmarked launch at full size
def test_step_full_size_room(oracle):
    """ts_render_step_l1 in the launch the benchmark times: 1200x680, 300k faces, 20 views, tile
    16x8, 64 faces per stage.

    (1) With the benchmark's noise targets: colour, depth, alpha and the loss gradients of all 20
    views bit for bit against ts_render_fwd + ts_l1_loss (the same per-pixel arithmetic), the loss
    to float rounding and the map gradients within the gradient tolerance (atomic order).
    (2) Against the oracle: views 0 and 13 get targets at +-0.01 from the oracle's own render
    (random sign per element), so the sign of every L1 residual is the same on both sides; the
    other 18 views get the separate calls' render as their target, so every residual there is
    exactly 0 and, with sign(0) = 0, they add nothing to the map gradients.  The fused step's map
    gradients, the sampled views' pose gradients and loss then match the oracle on those 2 views."""
    import torch
    import paper_2605_31419_gb300 as ts
    from oracle.oracle import SceneArrays
    sc = room_scene(3, 300_000, 20, 1200, 680, 600.0, target_seed=4)
    p, po = params_pair(tile_w=16, tile_h=8, tris_per_stage=64)
    off = np.concatenate([[0], np.cumsum(sc.cams[:, 4] * sc.cams[:, 5])]).astype(int)
    # (1) the benchmark's own targets
    s = step_run(sc, p)
    g = gpu_run(sc, p)
    assert s["counters"]["status"] == "TS_OK" and g["counters"]["status"] == "TS_OK"
    for k in ("color", "depth", "alpha", "dC", "dD"):
        assert np.array_equal(s[k], g[k]), f"{k} differs from the separate calls"
    assert_images(s["loss_v"], g["loss_v"], "loss vs separate", atol=1e-7, rtol=1e-6)
    assert s["counters"]["fwd_contrib"] == s["counters"]["bwd_contrib"] == g["counters"]["bwd_contrib"] > 0
    for k in ("dpos", "dcol", "dopa"):
        assert_grad(s[k], g[k], f"{k} vs separate")
    assert np.allclose(s["dtau"], g["dtau"], rtol=1e-3, atol=1e-3 * np.abs(g["dtau"]).max())
    # (2) targets that pin every residual's sign
    views = (0, 13)
    sub = sc.subset_views(list(views))
    sa = SceneArrays.of(sub)
    f = oracle.forward(sa, po)
    rng = np.random.default_rng(31)
    tc_o = f["color"] + 0.01 * np.where(rng.random(f["color"].size) < 0.5, -1.0, 1.0)
    td_o = f["depth"] + 0.01 * np.where(rng.random(f["depth"].size) < 0.5, -1.0, 1.0)
    tc_o, td_o = tc_o.astype(np.float32).astype(np.float64), td_o.astype(np.float32).astype(np.float64)
    lo = oracle.l1_loss(sa, f["color"], f["depth"], tc_o, td_o, 0.05)
    r = oracle.backward(sa, po, lo["dC"], lo["dD"])
    so = np.concatenate([[0], np.cumsum(sub.cams[:, 4] * sub.cams[:, 5])]).astype(int)
    tc, td = g["color"].copy(), g["depth"].copy()
    for i, v in enumerate(views):
        tc[3 * off[v]:3 * off[v + 1]] = tc_o[3 * so[i]:3 * so[i + 1]]
        td[off[v]:off[v + 1]] = td_o[so[i]:so[i + 1]]
        HW = int(off[v + 1] - off[v])
        sc.tgt_color[v] = tc[3 * off[v]:3 * off[v + 1]].astype(np.float32).reshape(3, -1, sc.cams[v, 4].astype(int))
        sc.tgt_depth[v] = td[off[v]:off[v + 1]].astype(np.float32).reshape(-1, sc.cams[v, 4].astype(int))
        assert sc.tgt_depth[v].size == HW
    for v in range(sc.n_views):
        if v not in views:
            W_ = int(sc.cams[v, 4])
            sc.tgt_color[v] = g["color"][3 * off[v]:3 * off[v + 1]].astype(np.float32).reshape(3, -1, W_)
            sc.tgt_depth[v] = g["depth"][off[v]:off[v + 1]].astype(np.float32).reshape(-1, W_)
    del g
    torch.cuda.empty_cache()
    s = step_run(sc, p)
    for v in range(sc.n_views):
        if v not in views:
            assert not s["dC"][3 * off[v]:3 * off[v + 1]].any() and not s["dD"][off[v]:off[v + 1]].any(), v
            assert s["loss_v"][v] == 0.0, v
    for i, v in enumerate(views):
        # the same residual signs; magnitudes 1/(3HW) and lambda_dep/HW, formed in FP32 on the GPU
        assert_images(s["dC"][3 * off[v]:3 * off[v + 1]], lo["dC"][3 * so[i]:3 * so[i + 1]], f"dC[{v}]", 0.0, 1e-6)
        assert_images(s["dD"][off[v]:off[v + 1]], lo["dD"][so[i]:so[i + 1]], f"dD[{v}]", 0.0, 1e-6)
        assert_images(s["color"][3 * off[v]:3 * off[v + 1]], f["color"][3 * so[i]:3 * so[i + 1]], f"color[{v}]")
        assert_pose_grad(s["dtau"][v], r["dtau"][i], r["dtau_abs"][i])
    assert_images(s["loss_v"][list(views)], lo["loss_v"], "loss", atol=1e-6, rtol=1e-5)
    assert_grad(s["dpos"], r["dpos"], "dpos")
    assert_grad(s["dcol"], r["dcol"], "dcol")
    assert_grad(s["dopa"], r["dopa"], "dopa")


@pytest.mark.parametrize("stage", [32, 128])
def test_step_stage_sizes(oracle, stage):
    """32- and 128-face stages (the backward numbers one and four faces per lane): the fused step on
    long lists that span several stages equals the separate calls and the oracle."""
    sc = SCENES["long_lists"]()
    p, po = params_pair(tris_per_stage=stage)
    s = step_run(sc, p, pair_capacity=1_000_000)
    g = gpu_run(sc, p, pair_capacity=1_000_000)
    for k in ("color", "depth", "alpha", "dC", "dD"):
        assert np.array_equal(s[k], g[k]), k
    assert s["counters"]["fwd_contrib"] == s["counters"]["bwd_contrib"] == g["counters"]["bwd_contrib"] > 0
    r = oracle_run(oracle, sc, po)
    assert_images(s["loss_v"], r["loss_v"], "loss", atol=1e-6, rtol=1e-5)
    assert_grad(s["dpos"], r["dpos"], "dpos")
    assert_grad(s["dcol"], r["dcol"], "dcol")
    assert_grad(s["dopa"], r["dopa"], "dopa")
    assert_pose_grad(s["dtau"], r["dtau"], r["dtau_abs"])
