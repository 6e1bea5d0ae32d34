"""Photometric loss of Eq. 8-10 (L1 + D-SSIM + depth): the CUDA path against the oracle.

Loss per view within 1e-6 + 1e-5 relative; dD within 1e-6 relative (its values are +-lambda_dep/HW
or 0).  dC per element within 1e-3 of its own size plus 1e-5 of its condition scale a_q, which the
oracle returns: the window sum that makes up dC_q with every term replaced by its magnitude and
weighted by 1 + kappa_p, kappa_p = (second moments + squared means) / (sigma_x^2 + sigma_y^2 + C2)
at the term's pixel p.  In flat image regions dC_q is a sum of terms of size ~1/C2 that cancel, and
the variances are differences of moments that cancel; an FP32 evaluation (2^-24 per operation, a
chain of some 60 operations) can promise no better than a few 1e-6 of that scale.
"""
import numpy as np
import pytest

from oracle.oracle import SceneArrays
from ts_synth.scenes import Scene, loss_images, random_triangles_scene

pytestmark = pytest.mark.gpu


def _cams(sizes):
    return np.asarray([[0.8 * W, 0.8 * W, W / 2, H / 2, W, H] for W, H in sizes], np.float64)


def _scene_arrays(cams):
    sc = random_triangles_scene(seed=3, n_faces=4, W=int(cams[0, 4]), H=int(cams[0, 5]), f=10.0)
    poses = np.repeat(sc.poses[:1], len(cams), axis=0)
    return SceneArrays.of(Scene(sc.pos, sc.col, sc.opa, None, cams, poses))


def _gpu(cams, C, D, tC, tD, lam, lam_dep, fn="pho"):
    import torch
    import paper_2605_31419_gb300 as ts
    rast = ts.Rasterizer(cams, 4)
    dev = lambda a: torch.as_tensor(np.asarray(a, np.float32), device="cuda")  # noqa: E731
    V, P = len(cams), len(D)
    loss, dC, dD = dev(np.zeros(V)), dev(np.full(3 * P, np.nan)), dev(np.full(P, np.nan))
    if fn == "pho":
        ts.ts_pho_loss(rast.plan, rast.ws, dev(C), dev(D), dev(tC), dev(tD), lam, lam_dep, loss, dC, dD)
    else:
        ts.ts_l1_loss(rast.plan, rast.ws, dev(C), dev(D), dev(tC), dev(tD), lam_dep, loss, dC, dD)
    torch.cuda.synchronize()
    return loss.cpu().numpy().astype(np.float64), dC.cpu().numpy().astype(np.float64), dD.cpu().numpy().astype(np.float64)


def _check(cams, got, ref, label=""):
    loss, dC, dD = got
    assert np.all(np.isfinite(dC)) and np.all(np.isfinite(dD)), "unwritten or non-finite gradient"
    err = np.abs(loss - ref["loss_v"])
    assert np.all(err <= 1e-6 + 1e-5 * np.abs(ref["loss_v"])), (label, loss, ref["loss_v"])
    assert np.all(np.abs(dD - ref["dD"]) <= 1e-6 * np.abs(ref["dD"])), label
    off = 0
    for v, c in enumerate(cams):
        HW = int(c[4]) * int(c[5])
        g, r = dC[3 * off:3 * off + 3 * HW], ref["dC"][3 * off:3 * off + 3 * HW]
        a = ref["dC_abs"][3 * off:3 * off + 3 * HW]
        tol = 1e-3 * np.abs(r) + 1e-5 * a
        bad = np.abs(g - r) > tol
        assert not bad.any(), (label, v, int(bad.sum()), float((np.abs(g - r) / a).max()), float(np.abs(r).max()))
        off += HW


SIZES = {
    "mixed_ragged": [(160, 120), (37, 29), (64, 32), (33, 65)],
    "tiny": [(7, 5), (1, 1), (11, 3)],
    "keyframes": [(320, 240), (200, 150)],
}


@pytest.mark.parametrize("name", sorted(SIZES))
@pytest.mark.parametrize("lam", [0.2, 1.0])
def test_pho_loss_matches_oracle(oracle, name, lam):
    cams = _cams(SIZES[name])
    C, D, tC, tD = loss_images(11, cams)
    got = _gpu(cams, C, D, tC, tD, lam, 0.05)
    ref = oracle.pho_loss(_scene_arrays(cams), C, D, tC, tD, lam, 0.05)
    _check(cams, got, ref, f"{name} lambda={lam}")


def test_pho_loss_lambda0_is_l1(oracle):
    cams = _cams(SIZES["mixed_ragged"])
    C, D, tC, tD = loss_images(12, cams)
    a = _gpu(cams, C, D, tC, tD, 0.0, 0.05)
    b = _gpu(cams, C, D, tC, tD, 0.0, 0.05, fn="l1")
    assert np.allclose(a[0], b[0], rtol=1e-6, atol=1e-7)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_pho_loss_identical_images_and_determinism(oracle):
    cams = _cams(SIZES["mixed_ragged"])
    C, D, _, _ = loss_images(13, cams)
    loss, dC, dD = _gpu(cams, C, D, C, D, 0.2, 0.05)
    ref = oracle.pho_loss(_scene_arrays(cams), C, D, C, D, 0.2, 0.05)
    assert np.all(np.abs(loss) < 1e-6)  # SSIM = 1 and L1 = 0
    assert np.abs(dD).max() == 0
    assert np.abs(ref["dC"]).max() < 1e-12  # x = y is stationary: what is left on the GPU is rounding
    assert np.all(np.abs(dC) <= 1e-5 * ref["dC_abs"])
    C, D, tC, tD = loss_images(14, cams)
    a, b = _gpu(cams, C, D, tC, tD, 0.2, 0.05), _gpu(cams, C, D, tC, tD, 0.2, 0.05)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_pho_loss_full_size_view(oracle):
    """The 1200 x 680 view of the room workload next to a 640 x 480 one: every element."""
    cams = _cams([(1200, 680), (640, 480)])
    C, D, tC, tD = loss_images(15, cams)
    got = _gpu(cams, C, D, tC, tD, 0.2, 0.05)
    ref = oracle.pho_loss(_scene_arrays(cams), C, D, tC, tD, 0.2, 0.05)
    _check(cams, got, ref, "full size")
