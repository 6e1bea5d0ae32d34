"""libts builds, loads without a GPU and exports every entry point include/ts_api.h declares;
host-side plan logic and argument validation (no device work)."""
import json
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ts_api.h")


@pytest.fixture(scope="module")
def ts():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2605_31419_gb300 as ts
    return ts


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+(ts_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(ts):
    names = declared_functions()
    assert len(names) >= 16, names
    out = subprocess.run(["nm", "-D", "--defined-only", ts.binding.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (ts_[a-z0-9_]+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    # and the Python binding declares the same set with the same names
    assert set(names) == set(ts.binding.SIGNATURES), set(names) ^ set(ts.binding.SIGNATURES)
    for n in names:
        getattr(ts.binding.lib(), n)


def test_default_params_match_paper(ts):
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))
    p = ts.ts_default_params()
    assert p.sigma == g["sigma"]["value"]
    assert (p.tile_w, p.tile_h, p.tris_per_stage) == (16, 8, 64)


def test_plan_layout_and_workspace(ts):
    cams = np.array([[150, 150, 80, 60, 160, 120], [40, 40, 28.5, 16.5, 57, 33]])
    plan = ts.ts_plan_init(cams, 2000, ts.ts_default_params(tile_h=16))
    lay = ts.ts_plan_layout(plan, 2)
    assert list(lay["pix_off"]) == [0, 19200, 19200 + 57 * 33]
    assert list(lay["tiles_x"]) == [10, 4] and list(lay["tiles_y"]) == [8, 3]
    assert list(lay["tile_off"]) == [0, 80, 92]
    ws = ts.ts_workspace_size(plan)
    # records (128 B), gradients (96 B) and pair buffers dominate
    assert ws > 2 * 2000 * (128 + 96) + 4 * 2 * 2000 * 24
    assert ws % 256 == 0


@pytest.mark.parametrize("bad", [
    dict(tile_w=12), dict(tile_h=5), dict(tris_per_stage=48), dict(sigma=0.0), dict(alpha_max=1.0),
    dict(T_min=1.0), dict(z_near=0.0), dict(flags=1 << 20)])
def test_plan_rejects_bad_params(ts, bad):
    with pytest.raises(ts.TsError) as e:
        ts.ts_plan_init(np.array([[150, 150, 80, 60, 160, 120]]), 10, ts.ts_default_params(**bad))
    assert e.value.status == 1


def test_plan_rejects_bad_views(ts):
    p = ts.ts_default_params()
    for cams in (np.zeros((0, 6)), np.array([[150, 150, 80, 60, 0, 120]]), np.array([[-1, 150, 80, 60, 16, 16]]),
                 np.tile([[10, 10, 5, 5, 16, 16]], (257, 1))):
        with pytest.raises(ts.TsError):
            ts.ts_plan_init(cams, 10, p)
    with pytest.raises(ts.TsError):
        ts.ts_plan_init(np.array([[10, 10, 5, 5, 16, 16]]), -1, p)


def test_device_calls_reject_null_arguments(ts):
    """Argument checks run before any CUDA call, so they are testable without a GPU."""
    import ctypes as C
    L = ts.binding.lib()
    plan = ts.ts_plan_init(np.array([[10, 10, 5, 5, 16, 16]]), 4, ts.ts_default_params())
    assert L.ts_project(C.byref(plan), None, None, None, 0, None) == 1
    assert L.ts_bin(None, None, None) == 1
    assert L.ts_render_fwd(C.byref(plan), None, None, None, None, None) == 1
    assert L.ts_render_bwd(C.byref(plan), C.c_void_p(256), None, None, None, None, None) == 1
    assert L.ts_pose_grad(C.byref(plan), None, None, None) == 1
    vp = [C.c_void_p(256)] * 4
    # fused L1 step: null targets or outputs, a negative or non-finite depth weight, and a plan with
    # the normal map
    z = C.c_void_p(256)
    assert L.ts_render_step_l1(C.byref(plan), z, None, z, C.c_float(0.05), z, None, None, z, None, None, None,
                               None) == 1
    assert L.ts_render_step_l1(C.byref(plan), z, z, z, C.c_float(0.05), None, None, None, z, None, None, None,
                               None) == 1
    for lam in (-1.0, float("inf"), float("nan")):
        assert L.ts_render_step_l1(C.byref(plan), z, z, z, C.c_float(lam), z, None, None, z, None, None, None,
                                   None) == 1
    nplan = ts.ts_plan_init(np.array([[10, 10, 5, 5, 16, 16]]), 4, ts.ts_default_params(flags=ts.TS_FLAG_NORMALS))
    assert L.ts_render_step_l1(C.byref(nplan), z, z, z, C.c_float(0.05), z, None, None, z, None, None, None,
                               None) == 1
    # photometric loss: null buffers, lambda_ssim outside [0, 1], negative or non-finite lambda_dep
    assert L.ts_pho_loss(C.byref(plan), C.c_void_p(256), *vp, C.c_float(0.2), C.c_float(0.05), None, None, None,
                         None) == 1
    # normal map outputs and gradients need a plan with TS_FLAG_NORMALS; the normal loss needs buffers
    assert L.ts_render_fwd_n(C.byref(plan), C.c_void_p(256), None, None, None, C.c_void_p(512), None) == 1
    assert L.ts_render_bwd_n(C.byref(plan), C.c_void_p(256), C.c_void_p(512), None, None, C.c_void_p(1024),
                             None, None) == 1
    assert L.ts_normal_loss(C.byref(plan), C.c_void_p(256), None, None, C.c_float(0.05), None, None, None) == 1
    # coverage, visibility and counts need TS_FLAG_STATS; co-visibility needs its buffers
    assert L.ts_face_stats(C.byref(plan), C.c_void_p(256), C.c_void_p(512), None, None, None, None) == 1
    assert L.ts_face_stats(C.byref(plan), C.c_void_p(256), None, None, None, C.c_void_p(512), None) == 1
    assert L.ts_covisibility(C.byref(plan), None, None, None) == 1
    # equilateral regulariser: null map or loss, a non-finite weight
    assert L.ts_equilateral(C.byref(plan), None, C.c_void_p(256), 1 << 30, C.c_float(1.0), C.c_void_p(256),
                            None, None) == 1
    for lam, lam_dep in ((-0.1, 0.05), (1.5, 0.05), (0.2, -1.0), (0.2, float("inf")), (float("nan"), 0.05)):
        assert L.ts_pho_loss(C.byref(plan), C.c_void_p(256), *vp, C.c_float(lam), C.c_float(lam_dep), *vp,
                             None) == 1
    # misaligned workspace
    assert L.ts_bin(C.byref(plan), C.c_void_p(8), None) == 1
    assert ts.ts_status_string(3) == "pair capacity exceeded"


def test_noalloc_binding_checks_tensors_before_any_launch(ts):
    """ts_l1_loss_noalloc has no plan: the cameras alone fix how far its kernels reach, so the
    binding checks every tensor's size, type, layout and device on the host (CPU tensors here)."""
    import torch
    cams = np.array([[40.0, 40.0, 28.5, 16.5, 57, 33], [10.0, 10.0, 4.0, 3.0, 8, 6]])
    P = 57 * 33 + 8 * 6
    ok = dict(color=torch.zeros(3 * P), depth=torch.zeros(P), tgt_color=torch.zeros(3 * P), tgt_depth=torch.zeros(P),
              loss=torch.zeros(2), dC=torch.zeros(3 * P), dD=torch.zeros(P))
    for name in ok:
        bad = dict(ok)
        bad[name] = torch.zeros(ok[name].numel() - 1)  # one element short
        with pytest.raises(ValueError, match=name):
            ts.ts_l1_loss_noalloc(cams, bad["color"], bad["depth"], bad["tgt_color"], bad["tgt_depth"], 0.05,
                                  bad["loss"], bad["dC"], bad["dD"])
    bad = dict(ok)
    bad["dD"] = torch.zeros(P, dtype=torch.float64)
    with pytest.raises(ValueError, match="float32"):
        ts.binding.check_noalloc_args(cams, **bad)
    bad = dict(ok)
    bad["color"] = torch.zeros(2 * 3 * P)[::2]
    with pytest.raises(ValueError, match="contiguous"):
        ts.binding.check_noalloc_args(cams, **bad)
    with pytest.raises(ValueError, match="CUDA"):  # right sizes, but host memory
        ts.binding.check_noalloc_args(cams, **ok)


def test_forward_only_plan_is_smaller_and_refuses_backward(ts):
    """A TS_FLAG_FORWARD_ONLY plan lays out no gradient slots and no lane masks, and the calls that
    need them return TS_ERR_INVALID_ARG before launching anything (checked with placeholder
    pointers that are never dereferenced)."""
    import ctypes as C
    cams = np.array([[600.0, 600.0, 600.0, 340.0, 1200, 680]] * 2)
    full = ts.ts_plan_init(cams, 50_000, ts.ts_default_params())
    fwd = ts.ts_plan_init(cams, 50_000, ts.ts_default_params(flags=ts.TS_FLAG_FORWARD_ONLY))
    saved = ts.ts_workspace_size(full) - ts.ts_workspace_size(fwd)
    # gradient slots (128 B per (view, face)) and lane masks (16 B per pair of the capacity)
    assert saved >= 2 * 50_000 * 128 + 4 * 2 * 50_000 * 16 - 4096, saved
    L = ts.binding.lib()
    fake = C.c_void_p(1 << 20)  # 256-byte aligned, never touched
    g = ts.binding.TsMapGrad()
    assert L.ts_render_bwd(C.byref(fwd), fake, fake, None, None, C.byref(g), None) == 1
    assert L.ts_render_bwd_n(C.byref(fwd), fake, fake, None, None, None, C.byref(g), None) == 1
    assert L.ts_pose_grad(C.byref(fwd), fake, fake, None) == 1
    assert L.ts_render_step_l1(C.byref(fwd), fake, fake, fake, 0.05, fake, None, None, fake, None, None,
                               C.byref(g), None) == 1
