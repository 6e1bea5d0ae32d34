"""Raster variants switched by ts_raster_params.flags, on the GPU against the oracle through the C
ABI, at the tolerances of tests/test_gpu_parity.py (images 1e-5 + 1e-4 |y|, bins bit-exact,
gradients 1e-3 relative; the pose gradient condition-aware)."""
import numpy as np
import pytest

from harness import assert_grad, assert_images, assert_pose_grad, gpu_run, oracle_run, params_pair
from oracle.oracle import SceneArrays
from ts_synth.scenes import random_triangles_scene

pytestmark = pytest.mark.gpu


def _scenes():
    from test_gpu_parity import _indexed, _indexed_9v, _ragged_room, _room_10v
    return {"c1": lambda: random_triangles_scene(seed=1), "ragged_room": _ragged_room, "indexed": _indexed,
            "room_10v": _room_10v, "indexed_9v": _indexed_9v}


@pytest.mark.parametrize("name", ["c1", "ragged_room", "indexed", "room_10v", "indexed_9v"])
def test_min_opacity_variant(oracle, name):
    import paper_2605_31419_gb300 as ts
    sc = _scenes()[name]()
    p, po = params_pair(flags=ts.TS_FLAG_MIN_OPACITY)
    assert po.min_opacity
    P = int(SceneArrays.of(sc).pix_offsets()[-1])
    rng = np.random.default_rng(29)
    dC = rng.normal(size=3 * P).astype(np.float32) * 1e-3
    dD = rng.normal(size=P).astype(np.float32) * 1e-3
    g = gpu_run(sc, p, dC=dC, dD=dD)
    r = oracle_run(oracle, sc, po, dC=dC, dD=dD)
    assert np.array_equal(g["n_last"], r["n_last"])
    for k in ("color", "depth", "alpha"):
        assert_images(g[k], r[k], k)
    assert_grad(g["dpos"], r["dpos"], "dpos")
    assert_grad(g["dcol"], r["dcol"], "dcol")
    assert_grad(g["dopa"], r["dopa"], "dopa")
    assert_pose_grad(g["dtau"], r["dtau"], r["dtau_abs"])
    # only one vertex of each soup face receives an opacity gradient
    if sc.faces is None:
        nz = (np.abs(g["dopa"].reshape(-1, 3)) > 0).sum(1)
        assert nz.max() <= 1


@pytest.mark.parametrize("name", ["c1", "ragged_room", "indexed", "room_10v", "indexed_9v"])
def test_face_sigma_variant(oracle, name):
    """Per-face window exponents sigma_F ~ U[0.5, 1.5] (float32), with dL/dsigma_F."""
    import paper_2605_31419_gb300 as ts
    sc = _scenes()[name]()
    sc.sigma = np.random.default_rng(31).uniform(0.5, 1.5, size=sc.n_faces).astype(np.float32)
    p, po = params_pair(flags=ts.TS_FLAG_FACE_SIGMA)
    P = int(SceneArrays.of(sc).pix_offsets()[-1])
    rng = np.random.default_rng(32)
    dC = rng.normal(size=3 * P).astype(np.float32) * 1e-3
    dD = rng.normal(size=P).astype(np.float32) * 1e-3
    g = gpu_run(sc, p, dC=dC, dD=dD)
    r = oracle_run(oracle, sc, po, dC=dC, dD=dD)
    assert np.array_equal(g["n_last"], r["n_last"])
    for k in ("color", "depth", "alpha"):
        assert_images(g[k], r[k], k)
    assert_grad(g["dpos"], r["dpos"], "dpos")
    assert_grad(g["dcol"], r["dcol"], "dcol")
    assert_grad(g["dopa"], r["dopa"], "dopa")
    assert_grad(g["dsigma"], r["dsigma"], "dsigma")
    assert np.abs(r["dsigma"]).max() > 0
    assert_pose_grad(g["dtau"], r["dtau"], r["dtau_abs"])


def test_face_sigma_equal_to_global_reproduces_global():
    """sigma_F = 0.5 for every face renders bit for bit what the global sigma = 0.5 renders."""
    import torch
    import paper_2605_31419_gb300 as ts
    sc = _scenes()["ragged_room"]()
    outs = []
    for flags, sig in ((0, None), (ts.TS_FLAG_FACE_SIGMA, np.full(sc.n_faces, 0.5, np.float32))):
        rast = ts.Rasterizer(sc.cams, sc.n_faces, ts.ts_default_params(flags=flags))
        m = ts.Map.from_numpy(sc.pos, sc.col, sc.opa, sigma=sig)
        C, D, A = rast.forward(m, ts.poses_tensor(sc.poses))
        torch.cuda.synchronize()
        outs.append((C.cpu().numpy(), D.cpu().numpy(), A.cpu().numpy()))
    assert all(np.array_equal(a, b) for a, b in zip(*outs))
