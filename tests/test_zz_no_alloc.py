"""ts_l1_loss_noalloc, the loss entry point for callers that cannot allocate device memory for the
library (it has no plan or workspace; its partial sums live in a static device array), against
the workspace-based ts_l1_loss on two consecutive calls with different data.

Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs(rng, cams):
    P = int(sum(int(c[4]) * int(c[5]) for c in cams))
    C = rng.random(3 * P).astype(np.float32)
    D = (rng.random(P) * 4).astype(np.float32)
    tC = rng.random(3 * P).astype(np.float32)
    tD = (0.5 + 3.5 * rng.random(P)).astype(np.float32)
    tD[rng.random(P) < 0.1] = 0.0  # invalid depth pixels
    return C, D, tC, tD


def test_noalloc_loss_matches_workspace_loss_twice():
    import torch
    import paper_2605_31419_gb300 as ts
    cams = np.array([[600.0, 600.0, 600.0, 340.0, 1200, 680], [40.0, 40.0, 28.5, 16.5, 57, 33],
                     [525.0, 525.0, 320.0, 240.0, 640, 480]])
    rast = ts.Rasterizer(cams, 1)  # plan + workspace for the reference call
    dev = lambda a: torch.as_tensor(a, device="cuda")  # noqa: E731
    rng = np.random.default_rng(123)
    for call in range(2):
        C, D, tC, tD = (dev(a) for a in _inputs(rng, cams))
        lam = 0.05 if call == 0 else 0.3
        ref_loss = torch.empty(3, device="cuda")
        ref_dC, ref_dD = torch.empty_like(C), torch.empty_like(D)
        # the workspace-based call reads the view table written by ts_project: run it once
        if call == 0:
            m = ts.Map.from_numpy(np.zeros((3, 3)), np.zeros((3, 3)), np.ones(3))
            rast.project(m, ts.poses_tensor(np.tile([1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0], (3, 1))))
        ts.ts_l1_loss(rast.plan, rast.ws, C, D, tC, tD, lam, ref_loss, ref_dC, ref_dD)
        loss = torch.full((3,), -1.0, device="cuda")
        dC, dD = torch.full_like(C, 7.0), torch.full_like(D, 7.0)
        ts.ts_l1_loss_noalloc(cams, C, D, tC, tD, lam, loss, dC, dD)
        torch.cuda.synchronize()
        l, rl = loss.cpu().numpy().astype(np.float64), ref_loss.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(l - rl) <= 1e-7 + 1e-5 * np.abs(rl)), (call, l, rl)
        assert torch.equal(dC, ref_dC) and torch.equal(dD, ref_dD)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    import paper_2605_31419_gb300 as ts
    big = np.tile([[600.0, 600.0, 600.0, 340.0, 16384, 16384]], (1, 1))  # 131072 blocks > 65536 slots
    t = torch.empty(1, device="cuda")
    with pytest.raises(ts.TsError) as e:
        ts.ts_l1_loss_noalloc(big, t, t, t, t, 0.05, t, t, t)
    assert e.value.status == 1
