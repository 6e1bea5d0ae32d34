"""Batched multi-view passes: graph replay equals eager execution, mixed resolutions in one plan
equal each view alone, and the autotuner returns a valid choice (GPU)."""
import numpy as np
import pytest

from harness import assert_grad
from ts_synth.scenes import Scene, mixed_keyframe_cameras, noise_targets, room_map, trajectory_poses

pytestmark = pytest.mark.gpu


def _window(n_faces=60000, per_res=1):
    pos, col, opa = room_map(5, n_faces)
    cams = mixed_keyframe_cameras(per_res)
    poses = trajectory_poses(1005, len(cams))
    sc = Scene(pos, col, opa, None, cams, poses)
    sc.tgt_color, sc.tgt_depth = noise_targets(6, cams)
    return sc


def _step(sc, params, graph=False):
    import torch
    import paper_2605_31419_gb300 as ts
    m = ts.Map.from_numpy(sc.pos, sc.col, sc.opa)
    grad = m.zeros_like()
    tc = torch.as_tensor(np.concatenate([t.reshape(-1) for t in sc.tgt_color]), device="cuda")
    td = torch.as_tensor(np.concatenate([t.reshape(-1) for t in sc.tgt_depth]), device="cuda")
    st = ts.MultiViewStep(m, sc.cams, ts.poses_tensor(sc.poses), tc, td, params, grad)
    if graph:
        st.capture()
        grad.pos.zero_(); grad.col.zero_(); grad.opa.zero_()
        st.run(1, use_graph=True)
    else:
        st.run(1)
    torch.cuda.synchronize()
    return st, grad


@pytest.mark.parametrize("persistent", [0, 1])
def test_graph_replay_equals_eager(persistent):
    import paper_2605_31419_gb300 as ts
    sc = _window()
    p = ts.ts_default_params(flags=persistent)
    a, ga = _step(sc, p)
    b, gb = _step(sc, p, graph=True)
    assert np.array_equal(a.rast.color.cpu().numpy(), b.rast.color.cpu().numpy())
    assert np.array_equal(a.rast.loss_v.cpu().numpy(), b.rast.loss_v.cpu().numpy())
    assert_grad(gb.pos.cpu().numpy(), ga.pos.cpu().numpy(), "dpos graph vs eager", rtol=1e-4)
    assert np.allclose(b.rast.dtau.cpu().numpy(), a.rast.dtau.cpu().numpy(), rtol=1e-4, atol=1e-6)


def test_mixed_resolutions_batched_equal_alone():
    import paper_2605_31419_gb300 as ts
    sc = _window()
    p = ts.ts_default_params(flags=1)
    both, gboth = _step(sc, p)
    off = np.concatenate([[0], np.cumsum(sc.cams[:, 4] * sc.cams[:, 5])]).astype(int)
    gsum = np.zeros_like(gboth.pos.cpu().numpy())
    for v in range(sc.n_views):
        one, g1 = _step(sc.subset_views([v]), p)
        assert np.array_equal(one.rast.color.cpu().numpy(), both.rast.color.cpu().numpy()[3 * off[v]:3 * off[v + 1]])
        gsum += g1.pos.cpu().numpy()
    assert_grad(gsum, gboth.pos.cpu().numpy(), "dpos per-view sum vs batched", rtol=1e-4)


def test_autotune_picks_a_valid_shape(tmp_path, monkeypatch):
    import torch
    import paper_2605_31419_gb300 as ts
    monkeypatch.setenv("TS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    sc = _window(20000)
    m = ts.Map.from_numpy(sc.pos, sc.col, sc.opa)
    tc = torch.as_tensor(np.concatenate([t.reshape(-1) for t in sc.tgt_color]), device="cuda")
    td = torch.as_tensor(np.concatenate([t.reshape(-1) for t in sc.tgt_depth]), device="cuda")
    best, res = ts.autotune(m, sc.cams, ts.poses_tensor(sc.poses), tc, td, tiles=((16, 8), (8, 8)), stages=(64,),
                            iters=1)
    assert best["ms"] == min(r["ms"] for r in res)
    again, res2 = ts.autotune(m, sc.cams, ts.poses_tensor(sc.poses), tc, td)
    assert again == best and res2 is None  # served from the cache


def test_mapping_loss_step_composes_the_terms():
    """MultiViewStep with all terms of E_map (Eq. 15: D-SSIM photometric, depth, normal against
    sensor normals, equilateral) equals the same kernels called one by one."""
    import torch
    import paper_2605_31419_gb300 as ts
    from ts_synth.scenes import sensor_normals
    sc = _window()
    m = ts.Map.from_numpy(sc.pos, sc.col, sc.opa)
    poses = ts.poses_tensor(sc.poses)
    dev = lambda a: torch.as_tensor(np.asarray(a, np.float32), device="cuda")  # noqa: E731
    tc = dev(np.concatenate([t.reshape(-1) for t in sc.tgt_color]))
    td = dev(np.concatenate([t.reshape(-1) for t in sc.tgt_depth]))
    tn = dev(sensor_normals(7, sc.cams))
    g_full = m.zeros_like()
    full = ts.MultiViewStep(m, sc.cams, poses, tc, td, None, g_full, lambda_ssim=0.2, tgt_normal=tn,
                            lambda_norm=0.05, lambda_equi=1.2)
    full.run(1)
    g_man = m.zeros_like()
    r = ts.Rasterizer(sc.cams, m.n_faces, ts.ts_default_params(flags=ts.TS_FLAG_NORMALS))
    r.forward(m, poses)
    r.pho_loss(tc, td, 0.2, 0.05)
    _, dN = r.normal_loss(tn, 0.05)
    r.backward(r.dC, r.dD, None, g_man, dN=dN)
    e = r.equilateral(m, 1.2, g_man)
    r.pose_grad()
    torch.cuda.synchronize()
    L = full.losses()
    assert np.array_equal(L["pho_dep"].cpu().numpy(), r.loss_v.cpu().numpy())
    assert np.array_equal(L["norm"].cpu().numpy(), r.nloss_v.cpu().numpy())
    assert np.array_equal(L["equi"].cpu().numpy(), e.cpu().numpy())
    assert np.all(L["norm"].cpu().numpy() > 0) and float(L["equi"].item()) > 0
    for name in ("pos", "col", "opa"):
        assert_grad(getattr(g_full, name).cpu().numpy(), getattr(g_man, name).cpu().numpy(), f"d{name}", rtol=1e-4)
    assert np.allclose(full.rast.dtau.cpu().numpy(), r.dtau.cpu().numpy(), rtol=1e-4, atol=1e-6)
    # the normal and equilateral terms move the position gradient
    g_pho = m.zeros_like()
    ts.MultiViewStep(m, sc.cams, poses, tc, td, None, g_pho, lambda_ssim=0.2).run(1)
    torch.cuda.synchronize()
    assert np.abs(g_pho.pos.cpu().numpy() - g_full.pos.cpu().numpy()).max() > 1e-3 * np.abs(g_full.pos.cpu().numpy()).max()


def test_fused_window_step_equals_separate_calls():
    """With the plain L1 loss MultiViewStep runs the fused ts_render_step_l1 pass: on mixed
    resolutions it gives the images, the loss and (to atomic order) the map and pose gradients of
    the separate forward, loss and backward calls."""
    import torch
    import paper_2605_31419_gb300 as ts
    sc = _window()
    p = ts.ts_default_params()
    st, g = _step(sc, p)
    assert st.fused
    m = ts.Map.from_numpy(sc.pos, sc.col, sc.opa)
    g2 = m.zeros_like()
    r = ts.Rasterizer(sc.cams, sc.n_faces, p)
    tc = torch.as_tensor(np.concatenate([t.reshape(-1) for t in sc.tgt_color]), device="cuda")
    td = torch.as_tensor(np.concatenate([t.reshape(-1) for t in sc.tgt_depth]), device="cuda")
    r.forward(m, ts.poses_tensor(sc.poses))
    r.l1_loss(tc, td, 0.05)
    r.backward(r.dC, r.dD, None, g2)
    r.pose_grad()
    torch.cuda.synchronize()
    for k in ("color", "depth", "alpha"):
        assert torch.equal(getattr(st.rast, k), getattr(r, k)), k
    assert np.allclose(st.rast.loss_v.cpu().numpy(), r.loss_v.cpu().numpy(), rtol=1e-6, atol=1e-7)
    for k in ("pos", "col", "opa"):
        assert_grad(getattr(g, k).cpu().numpy(), getattr(g2, k).cpu().numpy(), f"d{k} fused vs separate", rtol=1e-4)
    assert np.allclose(st.rast.dtau.cpu().numpy(), r.dtau.cpu().numpy(), rtol=1e-4,
                       atol=1e-4 * np.abs(r.dtau.cpu().numpy()).max())
