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


def _limit_cams(n_views):
    """One 1024 x 1024 view (512 blocks of 2048 pixels) and n_views - 1 views of one pixel: the
    scratch holds n_views * 512 slots, 65536 for 128 views."""
    cams = np.tile([[1.0, 1.0, 0.5, 0.5, 1, 1]], (n_views, 1))
    cams[0] = [500.0, 500.0, 512.0, 512.0, 1024, 1024]
    return cams


def _tensors(cams, seed):
    import torch
    rng = np.random.default_rng(seed)
    C, D, tC, tD = (torch.as_tensor(a, device="cuda") for a in _inputs(rng, cams))
    P = D.numel()
    return C, D, tC, tD, torch.empty(len(cams), device="cuda"), torch.empty(3 * P, device="cuda"), \
        torch.empty(P, device="cuda")


def test_noalloc_at_the_limit_matches_and_allocates_nothing():
    """128 views of which one is 1024 x 1024: exactly the 65536 slots of the scratch.  The result
    equals ts_l1_loss, and a second call leaves the device's free memory unchanged."""
    import torch
    import paper_2605_31419_gb300 as ts
    cams = _limit_cams(128)
    rast = ts.Rasterizer(cams, 1)
    C, D, tC, tD, loss, dC, dD = _tensors(cams, 5)
    ref_loss, ref_dC, ref_dD = torch.empty_like(loss), torch.empty_like(dC), torch.empty_like(dD)
    ts.ts_l1_loss(rast.plan, rast.ws, C, D, tC, tD, 0.05, ref_loss, ref_dC, ref_dD)
    ts.ts_l1_loss_noalloc(cams, C, D, tC, tD, 0.05, loss, dC, dD)  # warm-up: the scratch lookup
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    loss.fill_(-1.0)
    ts.ts_l1_loss_noalloc(cams, C, D, tC, tD, 0.05, loss, dC, dD)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    l, rl = loss.cpu().numpy().astype(np.float64), ref_loss.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(l - rl) <= 1e-7 + 1e-5 * np.abs(rl)), (l, rl)
    assert torch.equal(dC, ref_dC) and torch.equal(dD, ref_dD)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    import paper_2605_31419_gb300 as ts
    # one huge view: 131072 blocks > 65536 slots (the C entry point rejects it; the tensors are
    # placeholders of one element, so the binding's own size check is bypassed by calling libts)
    big = ts.binding.cameras(np.array([[600.0, 600.0, 600.0, 340.0, 16384, 16384]]))
    t = torch.empty(1, device="cuda")
    p = t.data_ptr()
    st = ts.binding.lib().ts_l1_loss_noalloc(big, 1, p, p, p, p, 0.05, p, p, p, None)
    assert st == 1
    # 129 views of the limit's shape: 66048 slots, one view more than the scratch holds
    cams = _limit_cams(129)
    C, D, tC, tD, loss, dC, dD = _tensors(cams, 6)
    loss.fill_(-1.0)
    with pytest.raises(ts.TsError) as e:
        ts.ts_l1_loss_noalloc(cams, C, D, tC, tD, 0.05, loss, dC, dD)
    assert e.value.status == 1
    torch.cuda.synchronize()
    assert torch.all(loss == -1.0)  # nothing was launched
    # a non-finite depth weight
    cams = _limit_cams(2)
    C, D, tC, tD, loss, dC, dD = _tensors(cams, 7)
    with pytest.raises(ts.TsError):
        ts.ts_l1_loss_noalloc(cams, C, D, tC, tD, float("inf"), loss, dC, dD)
