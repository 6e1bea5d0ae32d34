"""Rendered normal map (Eq. 12, TS_FLAG_NORMALS) on the GPU against the oracle, through the C ABI.

The normal map is an image (|x - y| <= 1e-5 + 1e-4 |y|); the map and pose gradients with a normal-map
gradient dN in the backward use the rasterizer's gradient tolerances; the normal loss uses the
loss tolerances of the other loss kernels.  Colour, depth, opacity and the per-pixel state of the
forward are bit-identical with and without the flag.
"""
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


def _params(**kw):
    import paper_2605_31419_gb300 as ts
    return params_pair(flags=ts.TS_FLAG_NORMALS, **kw)


@pytest.mark.parametrize("name", ["c1", "ragged_room", "indexed", "room_10v", "indexed_9v"])
def test_normal_map_matches_oracle(oracle, name):
    sc = _scenes()[name]()
    p, po = _params()
    g = gpu_run(sc, p, backward=False)
    r = oracle_run(oracle, sc, po, backward=False)
    assert_images(g["normal"], r["normal"], "normal")
    # unit-length normals composited with weights that sum to 1 - T_final (up to the image
    # tolerance, which both sides carry)
    off = SceneArrays.of(sc).pix_offsets()
    for v in range(len(off) - 1):
        a, b = int(off[v]), int(off[v + 1])
        for out, rel, ab in ((r, 0.0, 1e-12), (g, 4e-4, 4e-5)):
            nrm = np.linalg.norm(out["normal"][3 * a:3 * b].reshape(3, b - a), axis=0)
            assert np.all(nrm <= out["alpha"][a:b] * (1 + rel) + ab), v
    p0, _ = params_pair()
    g0 = gpu_run(sc, p0, backward=False)
    for k in ("color", "depth", "alpha", "T_final", "n_last"):
        assert np.array_equal(g[k], g0[k]), k


@pytest.mark.parametrize("name", ["c1", "ragged_room", "indexed", "room_10v", "indexed_9v"])
def test_backward_with_normal_gradient(oracle, name):
    sc = _scenes()[name]()
    p, po = _params()
    P = int(SceneArrays.of(sc).pix_offsets()[-1])
    rng = np.random.default_rng(17)
    dC = rng.normal(size=3 * P).astype(np.float32) * 1e-3
    dD = rng.normal(size=P).astype(np.float32) * 1e-3
    dN = rng.normal(size=3 * P).astype(np.float32) * 1e-3
    g = gpu_run(sc, p, dC=dC, dD=dD, dN=dN)
    r = oracle_run(oracle, sc, po, dC=dC, dD=dD, dN=dN)
    assert_grad(g["dpos"], r["dpos"], "dpos")
    assert_grad(g["dcol"], r["dcol"], "dcol")
    assert_grad(g["dopa"], r["dopa"], "dopa")
    assert_pose_grad(g["dtau"], r["dtau"], r["dtau_abs"])
    c = g["counters"]
    assert c["error_bits"] == 0 and c["fwd_contrib"] == c["bwd_contrib"] > 0


def test_normal_gradient_alone_reaches_positions_and_pose(oracle):
    """dN only (no colour or depth gradient): everything the map and pose receive comes through the
    normal map, i.e. through n_F and through alpha and T."""
    sc = _scenes()["ragged_room"]()
    p, po = _params()
    P = int(SceneArrays.of(sc).pix_offsets()[-1])
    dN = np.random.default_rng(18).normal(size=3 * P).astype(np.float32)
    zeros = np.zeros(3 * P, np.float32)
    g = gpu_run(sc, p, dC=zeros, dD=np.zeros(P, np.float32), dN=dN)
    r = oracle_run(oracle, sc, po, dC=zeros, dD=np.zeros(P), dN=dN)
    assert np.abs(r["dpos"]).max() > 0
    assert_grad(g["dpos"], r["dpos"], "dpos")
    assert_grad(g["dopa"], r["dopa"], "dopa")
    assert np.abs(g["dcol"]).max() == 0
    assert_pose_grad(g["dtau"], r["dtau"], r["dtau_abs"])


def test_normal_loss_matches_oracle(oracle):
    import torch
    import paper_2605_31419_gb300 as ts
    cams = np.array([[80.0, 80.0, 50.0, 30.0, 100, 60], [40.0, 40.0, 20.0, 15.0, 37, 29]])
    sc = random_triangles_scene(seed=3, n_faces=4, W=100, H=60, f=80.0)
    from ts_synth.scenes import Scene
    sa = SceneArrays.of(Scene(sc.pos, sc.col, sc.opa, None, cams, np.repeat(sc.poses[:1], 2, axis=0)))
    P = 100 * 60 + 37 * 29
    rng = np.random.default_rng(19)
    N = rng.normal(size=3 * P).astype(np.float32)
    Nb = rng.normal(size=(3, P))
    Nb /= np.linalg.norm(Nb, axis=0)
    Nb[:, rng.random(P) < 0.2] = 0.0
    Nb = Nb.reshape(-1).astype(np.float32)
    p, _ = _params()
    rast = ts.Rasterizer(cams, 4, p)
    dev = lambda a: torch.as_tensor(a, device="cuda")  # noqa: E731
    rast.normal.copy_(dev(N))
    loss, dN = rast.normal_loss(dev(Nb), weight=0.05)
    torch.cuda.synchronize()
    ref = oracle.normal_loss(sa, N, Nb, weight=0.05)
    assert np.allclose(loss.cpu().numpy(), ref["loss_v"], rtol=1e-5, atol=1e-6)
    assert np.allclose(dN.cpu().numpy(), ref["dN"], rtol=1e-6, atol=0)
