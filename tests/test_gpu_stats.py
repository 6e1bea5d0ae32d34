"""Map statistics of Sec. 3.4 on the GPU against the oracle, through the C ABI: per-(view, face)
pixel coverage and the visible sets bit-exact (integer work), projected area bit-exact (the same
FP32 operations on the same projected vertices), co-visibility IoU against numpy on the bitsets."""
import numpy as np
import pytest

from harness import params_pair
from oracle.oracle import SceneArrays
from ts_synth.scenes import random_triangles_scene

pytestmark = pytest.mark.gpu


def _scenes():
    from test_gpu_parity import _indexed, _ragged_room
    return {"c1": lambda: random_triangles_scene(seed=1), "ragged_room": _ragged_room, "indexed": _indexed}


@pytest.mark.parametrize("name", ["c1", "ragged_room", "indexed"])
@pytest.mark.parametrize("tile", [(16, 8), (16, 16)])
def test_face_stats_match_oracle(oracle, name, tile):
    import torch
    import paper_2605_31419_gb300 as ts
    sc = _scenes()[name]()
    p, po = params_pair(flags=ts.TS_FLAG_STATS, tile_w=tile[0], tile_h=tile[1])
    rast = ts.Rasterizer(sc.cams, sc.n_faces, p)
    m = ts.Map.from_numpy(sc.pos, sc.col, sc.opa, sc.faces)
    rast.forward(m, ts.poses_tensor(sc.poses))
    st = rast.face_stats()
    torch.cuda.synchronize()
    ref = oracle.face_stats(SceneArrays.of(sc), po)
    V, M = len(sc.cams), sc.n_faces
    cov = st["coverage"].cpu().numpy().view(np.uint32).reshape(-1)
    assert np.array_equal(cov, ref["coverage"])
    area = st["area"].cpu().numpy().reshape(-1).astype(np.float64)
    assert np.array_equal(area, ref["area"])
    vis = ref["coverage"].reshape(V, M) > 0
    bits = st["visible"].cpu().numpy().view(np.uint32)
    got = np.unpackbits(bits.view(np.uint8).reshape(V, -1), axis=1, bitorder="little")[:, :M].astype(bool)
    assert np.array_equal(got, vis)
    assert np.array_equal(st["n_visible"].cpu().numpy(), vis.sum(1))
    assert int(cov.sum()) == rast.counters()["fwd_contrib"]
    iou = rast.covisibility(st["visible"]).cpu().numpy()
    for i in range(V):
        for j in range(V):
            u = (vis[i] | vis[j]).sum()
            ref_iou = (vis[i] & vis[j]).sum() / u if u else 0.0
            assert abs(iou[i, j] - ref_iou) < 1e-6


def test_stats_flag_leaves_render_unchanged():
    import torch
    import paper_2605_31419_gb300 as ts
    sc = _scenes()["ragged_room"]()
    m = ts.Map.from_numpy(sc.pos, sc.col, sc.opa)
    out = []
    for flags in (0, ts.TS_FLAG_STATS):
        rast = ts.Rasterizer(sc.cams, sc.n_faces, ts.ts_default_params(flags=flags))
        C, D, A = rast.forward(m, ts.poses_tensor(sc.poses))
        torch.cuda.synchronize()
        out.append((C.cpu().numpy(), D.cpu().numpy(), A.cpu().numpy()))
    assert all(np.array_equal(a, b) for a, b in zip(*out))
