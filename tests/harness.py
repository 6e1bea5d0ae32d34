"""Run one seeded scene through the CUDA path and through the oracle, with identical parameters.

GPU parameters are float32 (ts_raster_params); the oracle receives the same float32 values
widened to double, so thresholds and culling see identical numbers on both sides.
"""
from __future__ import annotations

import numpy as np

from oracle.oracle import Oracle, Params, SceneArrays, pack_targets

GRAD_RTOL = 1e-3


def params_pair(**kw):
    import paper_2605_31419_gb300 as ts
    p = ts.ts_default_params(**kw)
    o = Params(sigma=p.sigma, alpha_min=p.alpha_min, alpha_max=p.alpha_max, T_min=p.T_min, z_near=p.z_near,
               r_min=p.r_min, bg=tuple(p.bg), tile_w=p.tile_w, tile_h=p.tile_h,
               min_opacity=bool(p.flags & ts.TS_FLAG_MIN_OPACITY))
    return p, o


def gpu_run(scene, p, *, backward=True, dC=None, dD=None, dA=None, dN=None, lambda_dep=0.05, pair_capacity=0,
            expect_error=False):
    """Forward (and backward of the L1 loss, or of the given image gradients) on the GPU.  With
    TS_FLAG_NORMALS in p.flags the normal map is returned and dN (if given) joins the backward.
    pair_capacity 0 takes the scene's own ``pair_capacity`` if it has one, else the plan default.
    A run that latched a device error (a dropped pair, a timed-out wait) fails unless expect_error."""
    import torch
    import paper_2605_31419_gb300 as ts
    pair_capacity = pair_capacity or getattr(scene, "pair_capacity", 0)
    rast = ts.Rasterizer(scene.cams, scene.n_faces, p, pair_capacity=pair_capacity)
    m = ts.Map.from_numpy(scene.pos, scene.col, scene.opa, scene.faces, sigma=getattr(scene, "sigma", None))
    poses = ts.poses_tensor(scene.poses)
    C, D, A = rast.forward(m, poses)
    out = dict(color=C.cpu().numpy().astype(np.float64), depth=D.cpu().numpy().astype(np.float64),
               alpha=A.cpu().numpy().astype(np.float64))
    out["T_final"] = rast.debug("T_final").cpu().numpy().astype(np.float64)
    out["n_last"] = rast.debug("n_last").cpu().numpy()
    out["counters"] = rast.counters(raise_on_error=False)
    if rast.normals:
        out["normal"] = rast.normal.cpu().numpy().astype(np.float64)
    if backward:
        dev = lambda a: None if a is None else torch.as_tensor(np.asarray(a), dtype=torch.float32, device="cuda")  # noqa
        if scene.tgt_color:
            tc, td = pack_targets(scene)
            loss, gC, gD = rast.l1_loss(dev(tc), dev(td), lambda_dep)
            out["loss_v"] = loss.cpu().numpy().astype(np.float64)
            out["dC"] = gC.cpu().numpy().astype(np.float64)
            out["dD"] = gD.cpu().numpy().astype(np.float64)
            gA = None
        if dC is not None:
            # image gradients supplied by the caller (the L1 gradient is a sign: where the two renders
            # differ by ~1e-5 around C = Cbar it may flip, so parity of the backward uses one dC)
            gC, gD, gA = dev(dC), dev(dD), dev(dA)
        g = m.zeros_like()
        rast.backward(gC, gD, gA, g, dN=dev(dN))
        dtau = rast.pose_grad()
        torch.cuda.synchronize()
        out["dpos"] = g.pos.cpu().numpy().T.astype(np.float64)
        out["dcol"] = g.col.cpu().numpy().T.astype(np.float64)
        out["dopa"] = g.opa.cpu().numpy().astype(np.float64)
        out["dtau"] = dtau.cpu().numpy().astype(np.float64)
        if g.sigma is not None:
            out["dsigma"] = g.sigma.cpu().numpy().astype(np.float64)
        out["counters"] = rast.counters(raise_on_error=False)
    if not expect_error:
        assert out["counters"]["error_bits"] == 0, f"device error latched: {out['counters']}"
    out["rast"] = rast
    return out


def oracle_run(o: Oracle, scene, po: Params, *, backward=True, dC=None, dD=None, dA=None, dN=None, lambda_dep=0.05):
    sa = SceneArrays.of(scene)
    f = o.forward(sa, po)
    out = dict(f)
    if backward:
        if dC is None:
            tc, td = pack_targets(scene)
            lo = o.l1_loss(sa, f["color"], f["depth"], tc, td, lambda_dep)
            dC, dD = lo["dC"], lo["dD"]
            out["loss_v"] = lo["loss_v"]
        out.update(o.backward(sa, po, dC, dD, dA, dN))
        out["dC_used"], out["dD_used"] = dC, dD
    return out


def assert_images(g, r, name="image", atol=1e-5, rtol=1e-4):
    bad = np.abs(g - r) > atol + rtol * np.abs(r)
    assert not bad.any(), f"{name}: {bad.sum()} elements out of tolerance, max err {np.abs(g - r).max():.3g}"


def assert_grad(g, r, name, rtol=GRAD_RTOL):
    """|g - r| <= rtol |r| + rtol * 1e-2 * max|r| per tensor."""
    scale = np.abs(r).max()
    bad = np.abs(g - r) > rtol * np.abs(r) + rtol * 1e-2 * scale + 1e-12
    if bad.any():
        i = np.unravel_index(np.argmax(np.abs(g - r) - rtol * np.abs(r)), r.shape)
        raise AssertionError(f"{name}: {bad.sum()}/{bad.size} out of tolerance; worst {i}: gpu {g[i]:.6g} "
                             f"oracle {r[i]:.6g} (scale {scale:.3g})")


def assert_pose_grad(g, r, r_abs, rtol=GRAD_RTOL):
    """Condition-aware: |g - r| <= rtol (|r| + 1e-2 sum_k |term_k|)."""
    bad = np.abs(g - r) > rtol * (np.abs(r) + 1e-2 * r_abs) + 1e-12
    assert not bad.any(), f"dtau: gpu {g[bad]} oracle {r[bad]} scale {r_abs[bad]}"
