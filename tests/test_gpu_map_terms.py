"""Map-space terms of the mapping loss (Eq. 14-15) on the GPU against the oracle, through the C ABI.

Equilateral regulariser: the value within 1e-5 relative (FP32 per face, a fixed-order sum in
double); the position gradient per element within 1e-3 of its size plus 1e-5 of the largest
entry, the rasterizer's gradient tolerance.  It is added into the gradient buffers (+=).
"""
import numpy as np
import pytest

from oracle.oracle import SceneArrays
from ts_synth.scenes import Scene, room_map, tiny_scene

pytestmark = pytest.mark.gpu


def _with_degenerate(pos):
    pos = pos.copy()
    pos[4] = pos[3]      # face 1: a zero-length edge
    pos[8] = pos[6]      # face 2: another
    return pos


def _scene(kind):
    cams = np.array([[100.0, 100.0, 50.0, 40.0, 100, 80]])
    pose = np.array([[1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0]], np.float32)
    if kind == "room_soup":
        pos, col, opa = room_map(9, 300_000)
        pos = _with_degenerate(pos)
        return Scene(pos, col, opa, None, cams, pose)
    if kind == "slivers":
        rng = np.random.default_rng(3)
        n = 5000
        a = rng.normal(size=(n, 3))
        b = a + rng.normal(size=(n, 3))
        c = a + (b - a) * rng.uniform(0.2, 0.8, size=(n, 1)) + 1e-3 * rng.normal(size=(n, 3))  # near-collinear
        pos = np.stack([a, b, c], 1).reshape(-1, 3).astype(np.float32)
        return Scene(pos, np.full((3 * n, 3), 0.5, np.float32), np.full(3 * n, 0.8, np.float32), None, cams, pose)
    sc = tiny_scene(5, n_faces=200, indexed=True)
    return Scene(sc.pos, sc.col, sc.opa, sc.faces, cams, pose)


@pytest.mark.parametrize("kind", ["room_soup", "slivers", "indexed"])
def test_equilateral_matches_oracle(oracle, kind):
    import torch
    import paper_2605_31419_gb300 as ts
    sc = _scene(kind)
    m = ts.Map.from_numpy(sc.pos, sc.col, sc.opa, faces=sc.faces)
    rast = ts.Rasterizer(sc.cams, m.n_faces)
    grad = m.zeros_like()
    # the kernel adds: start from values of the gradients' own size, so the sum keeps their digits
    pre = torch.rand(grad.pos.shape, generator=torch.Generator().manual_seed(0)) * 1e-6
    grad.pos.copy_(pre)
    e = rast.equilateral(m, weight=1.2, grad=grad)
    torch.cuda.synchronize()
    ref = oracle.equilateral(SceneArrays.of(sc))
    assert abs(float(e.item()) - ref["loss"]) <= 1e-5 * abs(ref["loss"]), (e.item(), ref["loss"])
    g = (grad.pos.cpu().numpy().astype(np.float64) - pre.numpy().astype(np.float64)).T  # [N, 3]
    r = 1.2 * ref["dpos"]
    tol = 1e-3 * np.abs(r) + 1e-5 * np.abs(r).max()
    bad = np.abs(g - r) > tol
    assert not bad.any(), (int(bad.sum()), float(np.abs(g - r).max()), float(np.abs(r).max()))
    assert rast.counters()["error_bits"] == 0


def test_equilateral_deterministic_and_weight_zero():
    import torch
    import paper_2605_31419_gb300 as ts
    sc = _scene("room_soup")
    m = ts.Map.from_numpy(sc.pos, sc.col, sc.opa)
    rast = ts.Rasterizer(sc.cams, m.n_faces)
    outs = []
    for _ in range(2):
        grad = m.zeros_like()
        e = rast.equilateral(m, weight=1.0, grad=grad)
        torch.cuda.synchronize()
        outs.append((e.cpu().numpy(), grad.pos.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    grad = m.zeros_like()
    e0 = rast.equilateral(m, weight=0.0, grad=grad)
    torch.cuda.synchronize()
    assert float(e0.item()) == float(outs[0][0][0]) and float(grad.pos.abs().max()) == 0.0
