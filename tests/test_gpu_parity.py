"""CUDA path vs the oracle, element by element, through the C ABI (needs a GB300).

Bit-exact: culling, tile boxes, depth keys, tiles touched, the sorted (key, face) pairs, tile
ranges and each pixel's last-contribution position.  Images: |x - y| <= 1e-5 + 1e-4 |y|.
Gradients: 1e-3 relative per element plus 1e-5 of the tensor's largest entry; the pose gradient
against 1e-3 (|g| + 1e-2 * sum of |per-term contributions|), because it is a cancelling sum.
"""
import numpy as np
import pytest

from harness import (assert_grad, assert_images, assert_pose_grad, gpu_run, oracle_run, params_pair)
from ts_synth.scenes import Scene, random_triangles_scene, room_map, room_scene, tiny_scene, noise_targets

pytestmark = pytest.mark.gpu


def _ragged_room():
    pos, col, opa = room_map(3, 20000)
    cams = np.array([[70.0, 70.0, 50.0, 37.5, 100, 75], [40.0, 40.0, 28.5, 16.5, 57, 33],
                     [90.0, 90.0, 61.0, 40.0, 123, 81]])
    from ts_synth.scenes import trajectory_poses
    sc = Scene(pos, col, opa, None, cams, trajectory_poses(1003, 3))
    sc.tgt_color, sc.tgt_depth = noise_targets(4, cams)
    return sc


def _indexed():
    sc = tiny_scene(31, n_faces=40, W=40, H=30, f=50.0, indexed=True)
    return sc


def _room_10v():
    # ten views: the chain rule takes its one-pass form from 8 views on
    return room_scene(5, 20000, 10, 100, 75, 70.0, target_seed=6)


def _indexed_9v():
    # a regular shared-vertex strip (faces (m, m+1, m+2), 10 x 20 px, inradius ~3.6 px) seen from
    # nine camera positions: the one-pass chain rule with atomic adds over shared vertices
    rng = np.random.default_rng(39)
    k = np.arange(42)
    pos = np.stack([-2.0 + 0.1 * k, np.where(k % 2 == 0, -0.2, 0.2), 2.0 + 0.05 * np.sin(0.7 * k)], 1)
    col = rng.uniform(0.1, 0.9, size=(42, 3))
    opa = rng.uniform(0.3, 0.9, size=42)
    faces = np.stack([k[:40], k[:40] + 1, k[:40] + 2], 1)
    n = 9
    poses = np.tile(np.array([[1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0]], np.float64), (n, 1))
    poses[:, 9] = np.linspace(-0.3, 0.3, n)
    poses[:, 10] = np.linspace(0.05, -0.05, n)
    cams = np.tile(np.array([[100.0, 100.0, 40.0, 30.0, 80, 60]]), (n, 1))
    out = Scene(pos.astype(np.float32), col.astype(np.float32), opa.astype(np.float32), faces.astype(np.int32),
                cams, poses)
    out.tgt_color, out.tgt_depth = noise_targets(38, cams)
    return out


SCENES = {"c1": lambda: random_triangles_scene(seed=1), "ragged_room": _ragged_room, "indexed": _indexed,
          "room_10v": _room_10v, "indexed_9v": _indexed_9v}
TILES = [(16, 8), (16, 16), (8, 8), (32, 8), (16, 32)]
_cache = {}


def run(name, tile=(16, 8), S=64, **kw):
    key = (name, tile, S, tuple(sorted(kw.items())))
    if key not in _cache:
        from oracle.oracle import Oracle
        sc = SCENES[name]()
        p, po = params_pair(tile_w=tile[0], tile_h=tile[1], tris_per_stage=S, **kw)
        r = oracle_run(Oracle(), sc, po)
        _cache[key] = (sc, p, po, gpu_run(sc, p, dC=r["dC_used"], dD=r["dD_used"]), r)
    return _cache[key]


@pytest.mark.parametrize("name", list(SCENES))
@pytest.mark.parametrize("tile", TILES, ids=lambda t: f"{t[0]}x{t[1]}")
def test_project_and_bin_bitexact(oracle, name, tile):
    from oracle.oracle import SceneArrays
    sc, p, po, g, _ = run(name, tile)
    rast = g["rast"]
    sa = SceneArrays.of(sc)
    pr = oracle.project(sa, po)
    rect = rast.debug("rect").cpu().numpy().reshape(-1, 4).astype(np.int32)
    assert np.array_equal(rect, pr["rect"])
    assert np.array_equal(rast.debug("count").cpu().numpy().astype(np.uint32), pr["count"])
    vis = pr["count"] > 0
    assert np.array_equal(rast.debug("zbits").cpu().numpy().view(np.uint32)[vis], pr["zbits"][vis])
    b = oracle.bin(sa, po)
    n = int(g["counters"]["n_pairs"])
    assert n == len(b["keys"])
    assert np.array_equal(rast.debug("keys").cpu().numpy().view(np.uint64)[:n], b["keys"])
    assert np.array_equal(rast.debug("ids").cpu().numpy().view(np.uint32)[:n], b["ids"])
    rg = rast.debug("ranges").cpu().numpy().view(np.uint32).reshape(-1, 2).astype(np.int64)
    empty = b["ranges"][:, 1] == 0
    assert np.array_equal(rg[~empty], b["ranges"][~empty])
    assert (rg[empty, 1] - rg[empty, 0] == 0).all()


@pytest.mark.parametrize("name", list(SCENES))
@pytest.mark.parametrize("tile", TILES, ids=lambda t: f"{t[0]}x{t[1]}")
def test_forward(name, tile):
    sc, p, po, g, r = run(name, tile)
    for k in ("color", "depth", "alpha", "T_final"):
        assert_images(g[k], r[k], k)
    assert np.array_equal(g["n_last"], r["n_last"]), "last-contribution positions differ"


@pytest.mark.parametrize("S", [32, 128])
def test_forward_stage_sizes(S):
    _, _, _, g, r = run("c1", (16, 8), S)
    assert_images(g["color"], r["color"], "color")
    assert np.array_equal(g["n_last"], r["n_last"])


@pytest.mark.parametrize("name", list(SCENES))
@pytest.mark.parametrize("tile", [(16, 8), (16, 16), (8, 8)], ids=lambda t: f"{t[0]}x{t[1]}")
def test_backward(name, tile):
    sc, p, po, g, r = run(name, tile)
    assert_images(g["loss_v"], r["loss_v"], "loss", atol=1e-6, rtol=1e-5)
    assert_grad(g["dpos"], r["dpos"], "dpos")
    assert_grad(g["dcol"], r["dcol"], "dcol")
    assert_grad(g["dopa"], r["dopa"], "dopa")
    assert_pose_grad(g["dtau"], r["dtau"], r["dtau_abs"])
    c = g["counters"]
    assert c["fwd_contrib"] == c["bwd_contrib"] > 0


def test_loss_kernel_matches_definition(oracle):
    import torch
    import paper_2605_31419_gb300 as ts
    from oracle.oracle import SceneArrays, pack_targets
    sc = _ragged_room()
    rast = ts.Rasterizer(sc.cams, sc.n_faces)
    rast.forward(ts.Map.from_numpy(sc.pos, sc.col, sc.opa), ts.poses_tensor(sc.poses))
    rng = np.random.default_rng(0)
    P = rast.n_pix
    C = rng.random(3 * P).astype(np.float32)
    D = (rng.random(P) * 4).astype(np.float32)
    tc, td = pack_targets(sc)
    td = td.copy()
    td[::5] = 0.0
    dev = lambda a: torch.as_tensor(np.asarray(a, np.float32), device="cuda")  # noqa: E731
    loss, dC, dD = dev(np.zeros(3)), dev(np.zeros(3 * P)), dev(np.zeros(P))
    ts.ts_l1_loss(rast.plan, rast.ws, dev(C), dev(D), dev(tc), dev(td), 0.05, loss, dC, dD)
    lo = oracle.l1_loss(SceneArrays.of(sc), C, D, tc.astype(np.float32), td.astype(np.float32), 0.05)
    assert_images(loss.cpu().numpy().astype(np.float64), lo["loss_v"], "loss", atol=1e-7, rtol=1e-5)
    assert_images(dC.cpu().numpy().astype(np.float64), lo["dC"], "dC", atol=0, rtol=1e-6)
    assert_images(dD.cpu().numpy().astype(np.float64), lo["dD"], "dD", atol=0, rtol=1e-6)


# ------------------------------------------------------------------------------- edge cases
def _single(verts, bg=(0.2, 0.4, 0.6), **kw):
    pos = np.asarray(verts, np.float32)
    n = len(pos)
    sc = Scene(pos, np.tile(np.array([[0.9, 0.5, 0.1]], np.float32), (n, 1)), np.full(n, 0.7, np.float32), None,
               np.array([[30.0, 30.0, 20.0, 16.0, 40, 32]]), np.array([[1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0]], np.float32))
    sc.tgt_color, sc.tgt_depth = noise_targets(9, sc.cams)
    return sc


@pytest.mark.parametrize("case", ["empty", "all_culled", "single_bg", "offscreen_partial", "sigma1", "opaque_stack"])
def test_edge_cases(oracle, case):
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
    r = oracle_run(oracle, sc, po)
    g = gpu_run(sc, p, dC=r["dC_used"], dD=r["dD_used"])
    for k in ("color", "depth", "alpha"):
        assert_images(g[k], r[k], k)
    assert np.array_equal(g["n_last"], r["n_last"])
    if sc.n_faces:
        assert_grad(g["dpos"], r["dpos"], "dpos")
        assert_grad(g["dcol"], r["dcol"], "dcol")
        assert_grad(g["dopa"], r["dopa"], "dopa")


def test_bin_global_counts_path_bitexact(oracle):
    """A view with more tiles than the shared-memory tile counts hold (4096 x 2560 at 8 x 8 tiles:
    163,840 tiles) takes the global-count path of the binning; its pairs and ranges are the same."""
    from oracle.oracle import SceneArrays
    sc = random_triangles_scene(seed=5, n_faces=600, W=4096, H=2560, f=1500.0, side_lo=0.05, side_hi=0.4)
    p, po = params_pair(tile_w=8, tile_h=8)
    g = gpu_run(sc, p, backward=False, pair_capacity=1_000_000)
    assert g["counters"]["status"] == "TS_OK"
    rast = g["rast"]
    b = oracle.bin(SceneArrays.of(sc), po)
    n = int(g["counters"]["n_pairs"])
    assert n == len(b["keys"]) and n > 0
    assert np.array_equal(rast.debug("keys").cpu().numpy().view(np.uint64)[:n], b["keys"])
    assert np.array_equal(rast.debug("ids").cpu().numpy().view(np.uint32)[:n], b["ids"])
    rg = rast.debug("ranges").cpu().numpy().view(np.uint32).reshape(-1, 2).astype(np.int64)
    empty = b["ranges"][:, 1] == 0
    assert np.array_equal(rg[~empty], b["ranges"][~empty])
    assert (rg[empty, 1] - rg[empty, 0] == 0).all()


@pytest.mark.parametrize("n_faces", [3000, 40000])
def test_bin_long_tile_lists_bitexact(oracle, n_faces):
    """Large faces over a 48 x 32 image: every tile's list holds most faces, so the lists go to
    the CTA-wide sort (3000: in shared memory; 40000: beyond its 16,384 keys, in place)."""
    from oracle.oracle import SceneArrays
    sc = random_triangles_scene(seed=6, n_faces=n_faces, W=48, H=32, f=40.0, side_lo=0.6, side_hi=1.2,
                                z_lo=1.0, z_hi=2.0)
    p, po = params_pair()
    g = gpu_run(sc, p, backward=False, pair_capacity=400_000)
    assert g["counters"]["status"] == "TS_OK"
    rast = g["rast"]
    b = oracle.bin(SceneArrays.of(sc), po)
    n = int(g["counters"]["n_pairs"])
    assert n == len(b["keys"])
    lens = b["ranges"][:, 1] - b["ranges"][:, 0]
    assert lens.max() > (16384 if n_faces > 16384 else 512)
    assert np.array_equal(rast.debug("keys").cpu().numpy().view(np.uint64)[:n], b["keys"])
    assert np.array_equal(rast.debug("ids").cpu().numpy().view(np.uint32)[:n], b["ids"])
    rg = rast.debug("ranges").cpu().numpy().view(np.uint32).reshape(-1, 2).astype(np.int64)
    empty = b["ranges"][:, 1] == 0
    assert np.array_equal(rg[~empty], b["ranges"][~empty])


def test_capacity_overflow_is_reported():
    import paper_2605_31419_gb300 as ts
    sc = random_triangles_scene(seed=1)
    p, _ = params_pair()
    g = gpu_run(sc, p, backward=False, pair_capacity=1024, expect_error=True)
    assert g["counters"]["status"] == "TS_ERR_CAPACITY"
    assert g["counters"]["n_pairs"] > 1024
    with pytest.raises(ts.TsError):
        g["rast"].counters()


def test_deterministic_forward():
    sc = random_triangles_scene(seed=1)
    p, _ = params_pair()
    a = gpu_run(sc, p, backward=False)
    b = gpu_run(sc, p, backward=False)
    for k in ("color", "depth", "alpha"):
        assert np.array_equal(a[k], b[k])


def test_batched_equals_plain():
    """All views in one plan vs each view alone: forward bit-identical, gradients within tolerance."""
    sc = _ragged_room()
    p, _ = params_pair()
    both = gpu_run(sc, p)
    off = np.concatenate([[0], np.cumsum(sc.cams[:, 4] * sc.cams[:, 5])]).astype(int)
    dpos = np.zeros_like(both["dpos"])
    for v in range(sc.n_views):
        one = gpu_run(sc.subset_views([v]), p)
        P = off[v + 1] - off[v]
        assert np.array_equal(one["color"], both["color"][3 * off[v]:3 * off[v + 1]])
        assert np.array_equal(one["depth"], both["depth"][off[v]:off[v + 1]])
        assert np.allclose(one["dtau"][0], both["dtau"][v], rtol=1e-5, atol=1e-7)
        dpos += one["dpos"]
        del P
    assert_grad(dpos, both["dpos"], "dpos batched vs plain", rtol=1e-4)


# ------------------------------------------------------------ full size, sampled outputs
@pytest.mark.parametrize("views", [(0, 13)])
def test_full_size_room_sampled_views(oracle, views):
    """The 1200x680, 300k-face, 20-view workload in one batched call (the benchmark's launch);
    two of its views and the map gradient of those views' loss are checked against the oracle."""
    from oracle.oracle import pack_targets
    sc = room_scene(3, 300_000, 20, 1200, 680, 600.0, target_seed=4)
    p, po = params_pair()
    # image gradients: the L1 loss of the sampled views only (other views contribute nothing)
    sub = sc.subset_views(list(views))
    r = oracle_run(oracle, sub, po)
    off = np.concatenate([[0], np.cumsum(sc.cams[:, 4] * sc.cams[:, 5])]).astype(int)
    P = off[-1]
    dC, dD = np.zeros(3 * P), np.zeros(P)
    so = np.concatenate([[0], np.cumsum(sub.cams[:, 4] * sub.cams[:, 5])]).astype(int)
    for i, v in enumerate(views):
        dC[3 * off[v]:3 * off[v + 1]] = r["dC_used"][3 * so[i]:3 * so[i + 1]]
        dD[off[v]:off[v + 1]] = r["dD_used"][so[i]:so[i + 1]]
    g = gpu_run(sc, p, dC=dC, dD=dD)
    for i, v in enumerate(views):
        for k, ch in (("color", 3), ("depth", 1), ("alpha", 1), ("T_final", 1)):
            assert_images(g[k][ch * off[v]:ch * off[v + 1]], r[k][ch * so[i]:ch * so[i + 1]], f"{k}[{v}]")
        assert np.array_equal(g["n_last"][off[v]:off[v + 1]], r["n_last"][so[i]:so[i + 1]])
        assert_pose_grad(g["dtau"][v], r["dtau"][i], r["dtau_abs"][i])
    assert_grad(g["dpos"], r["dpos"], "dpos")
    assert_grad(g["dcol"], r["dcol"], "dcol")
    assert_grad(g["dopa"], r["dopa"], "dopa")
    del pack_targets


@pytest.mark.parametrize("name", ["c1", "ragged_room"])
def test_persistent_launch_matches_oracle(name):
    """Persistent raster CTAs taking tiles from a device counter give the same images."""
    sc, p, po, g, r = run(name, (16, 8), 64, flags=1)
    for k in ("color", "depth", "alpha", "T_final"):
        assert_images(g[k], r[k], k)
    assert np.array_equal(g["n_last"], r["n_last"])
    assert_grad(g["dpos"], r["dpos"], "dpos")
    assert_grad(g["dcol"], r["dcol"], "dcol")
    assert_grad(g["dopa"], r["dopa"], "dopa")
    assert_pose_grad(g["dtau"], r["dtau"], r["dtau_abs"])
    _, _, _, g1, _ = run(name, (16, 8), 64)
    for k in ("color", "depth", "alpha"):
        assert np.array_equal(g[k], g1[k])


@pytest.mark.parametrize("name", ["c1", "ragged_room"])
def test_counters_match_oracle(oracle, name):
    """The device counters (summed from their slots by ts_sync_status) against the oracle: visible
    (view, face) records, (tile, face) pairs, and blended contributions of the forward and backward."""
    from oracle.oracle import SceneArrays
    sc = random_triangles_scene(seed=1) if name == "c1" else _ragged_room()
    p, po = params_pair()
    g = gpu_run(sc, p)
    c = g["counters"]
    sa = SceneArrays.of(sc)
    pr = oracle.project(sa, po)
    b = oracle.bin(sa, po)
    st = oracle.face_stats(sa, po)
    assert c["n_visible"] == int((pr["count"] > 0).sum())
    assert c["n_pairs"] == len(b["ids"])
    assert c["fwd_contrib"] == c["bwd_contrib"] == int(st["coverage"].sum()) > 0


def test_chain_rule_forms_agree():
    """The chain rule's one-pass form (8 views and more) and its two-pass form (fewer) on the same
    work: the C1 view alone (two-pass), and the C1 view with seven more views that see nothing, the
    camera 100 m behind the map (one-pass).  Both forms sum each face's views in view order and each
    view's faces in face order, so they differ only by the order of the raster's atomic adds into
    the slots."""
    sc = random_triangles_scene(seed=1)
    n = 8
    poses = np.repeat(sc.poses[:1], n, axis=0).copy()
    poses[1:, 11] -= 100.0
    cams = np.repeat(sc.cams[:1], n, axis=0)
    big = Scene(sc.pos, sc.col, sc.opa, sc.faces, cams, poses)
    tc, td = noise_targets(44, cams)
    big.tgt_color = [sc.tgt_color[0]] + list(tc[1:])
    big.tgt_depth = [sc.tgt_depth[0]] + list(td[1:])
    p, _ = params_pair()
    one = gpu_run(sc, p)
    many = gpu_run(big, p)
    assert many["counters"]["n_visible"] == one["counters"]["n_visible"] > 0
    assert many["counters"]["fwd_contrib"] == one["counters"]["fwd_contrib"]
    for k in ("dpos", "dcol", "dopa"):
        scale = np.abs(one[k]).max()
        assert np.allclose(many[k], one[k], rtol=1e-5, atol=1e-7 * scale), k
    assert np.allclose(many["dtau"][0], one["dtau"][0], rtol=1e-5, atol=1e-7 * np.abs(one["dtau"][0]).max())
    assert not np.any(many["dtau"][1:])


def test_second_backward_through_one_render_is_refused():
    """The per-face sums of a projection serve one backward, so the autograd wrapper refuses a second
    backward through the same render (a retained graph) instead of returning summed gradients."""
    import torch
    import paper_2605_31419_gb300 as ts
    sc = random_triangles_scene(seed=1)
    p, _ = params_pair()
    rast = ts.Rasterizer(sc.cams, sc.n_faces, p)
    m = ts.Map.from_numpy(sc.pos, sc.col, sc.opa)
    tau = torch.zeros(1, 6, device="cuda", requires_grad=True)
    C, D, _ = ts.render(rast, m, ts.poses_tensor(sc.poses), tau)
    J = C.sum() + D.sum()
    J.backward(retain_graph=True)
    g1 = tau.grad.clone()
    assert torch.any(g1 != 0)
    with pytest.raises(RuntimeError, match="second backward"):
        J.backward()


def test_plans_sharing_a_workspace():
    """Two plans of different layouts (one view; ten views) take turns on one workspace, each call
    sequence starting with the projection, and give what each gives on a workspace of its own."""
    import torch
    import paper_2605_31419_gb300 as ts
    from harness import pack_targets
    p, _ = params_pair()
    scenes = [random_triangles_scene(seed=1), _room_10v()]

    def make(sc):
        r = ts.Rasterizer(sc.cams, sc.n_faces, p)
        m = ts.Map.from_numpy(sc.pos, sc.col, sc.opa, sc.faces)
        tc, td = pack_targets(sc)
        return r, m, ts.poses_tensor(sc.poses), torch.as_tensor(tc, device="cuda"), torch.as_tensor(td, device="cuda")

    def step(r, m, poses, tc, td):
        g = m.zeros_like()
        r.project(m, poses)
        r.bin()
        r.step_l1(tc, td, 0.05, g)
        dtau = r.pose_grad().clone()
        torch.cuda.synchronize()
        assert r.counters()["error_bits"] == 0
        return g.pos.cpu().numpy().astype(np.float64), dtau.cpu().numpy().astype(np.float64)

    alone = [step(*make(sc)) for sc in scenes]
    shared = [make(sc) for sc in scenes]
    big = max(s[0].ws_bytes for s in shared)
    ws = torch.empty(big, dtype=torch.uint8, device="cuda")
    for s in shared:
        s[0].ws, s[0].ws_bytes = ws, big
    ts.ts_workspace_init(shared[1][0].plan, ws)
    for turn in range(4):
        k = turn % 2
        got = step(*shared[k])
        for a, b in zip(alone[k], got):
            scale = np.abs(a).max()
            assert scale > 0 and np.allclose(b, a, rtol=1e-5, atol=1e-7 * scale), (turn, k)
