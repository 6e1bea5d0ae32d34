"""ctypes binding of libts (include/ts_api.h): the same entry points, argument marshalling only.

Every computation runs in libts's CUDA kernels; these functions only translate torch tensors
into device pointers and raise on a non-OK status.  Importing this module loads the in-tree
``libts.so`` and fails loudly when it has not been built (``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libts.so")

TS_MAX_VIEWS = 256
TS_PLAN_BYTES = 24576
STATUS = {0: "TS_OK", 1: "TS_ERR_INVALID_ARG", 2: "TS_ERR_CUDA", 3: "TS_ERR_CAPACITY", 4: "TS_ERR_TIMEOUT",
          5: "TS_ERR_UNSUPPORTED"}
STAGES = ["project", "bin", "fwd", "bwd_raster", "bwd_project", "pose", "loss"]
TS_FLAG_PERSISTENT = 1  # ts_raster_params.flags bits of include/ts_api.h
TS_FLAG_NORMALS = 2
TS_FLAG_STATS = 4
TS_FLAG_MIN_OPACITY = 8
TS_FLAG_FACE_SIGMA = 16
TS_FLAG_FORWARD_ONLY = 32
DEBUG = dict(keys=0, ids=1, ranges=2, rect=3, zbits=4, count=5, T_final=6, n_last=7, records=8)


class TsError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS.get(status, status)}")
        self.status = status


class TsCamera(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32)]


class TsPose(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3)]


class TsRasterParams(C.Structure):
    _fields_ = [("sigma", C.c_float), ("alpha_min", C.c_float), ("alpha_max", C.c_float), ("T_min", C.c_float),
                ("z_near", C.c_float), ("r_min", C.c_float), ("bg", C.c_float * 3), ("tile_w", C.c_int32),
                ("tile_h", C.c_int32), ("tris_per_stage", C.c_int32), ("flags", C.c_int32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "bg"}
        d["bg"] = tuple(self.bg)
        return d


class TsMap(C.Structure):
    _fields_ = [("px", C.c_void_p), ("py", C.c_void_p), ("pz", C.c_void_p), ("cr", C.c_void_p), ("cg", C.c_void_p),
                ("cb", C.c_void_p), ("op", C.c_void_p), ("faces", C.c_void_p), ("n_vertices", C.c_int64),
                ("n_faces", C.c_int64), ("sigma", C.c_void_p)]


class TsMapGrad(C.Structure):
    _fields_ = [("gpx", C.c_void_p), ("gpy", C.c_void_p), ("gpz", C.c_void_p), ("gcr", C.c_void_p),
                ("gcg", C.c_void_p), ("gcb", C.c_void_p), ("gop", C.c_void_p), ("gsigma", C.c_void_p)]


class TsPlan(C.Structure):
    _fields_ = [("opaque", C.c_uint64 * (TS_PLAN_BYTES // 8))]


class TsCounters(C.Structure):
    _fields_ = [("n_pairs", C.c_uint64), ("pair_capacity", C.c_uint64), ("n_visible", C.c_uint64),
                ("fwd_contrib", C.c_uint64), ("bwd_contrib", C.c_uint64), ("error_bits", C.c_uint32),
                ("reserved", C.c_uint32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


# name -> (restype, argtypes); mirrors include/ts_api.h
_vp, _i32, _i64, _sz, _st = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t, C.c_int
SIGNATURES = {
    "ts_default_params": (None, [C.POINTER(TsRasterParams)]),
    "ts_plan_init": (_st, [C.POINTER(TsPlan), C.POINTER(TsCamera), _i32, _i64, C.POINTER(TsRasterParams), _i64]),
    "ts_workspace_size": (_sz, [C.POINTER(TsPlan)]),
    "ts_workspace_init": (_st, [C.POINTER(TsPlan), _vp, _sz, _vp]),
    "ts_project": (_st, [C.POINTER(TsPlan), C.POINTER(TsMap), _vp, _vp, _sz, _vp]),
    "ts_bin": (_st, [C.POINTER(TsPlan), _vp, _vp]),
    "ts_render_fwd": (_st, [C.POINTER(TsPlan), _vp, _vp, _vp, _vp, _vp]),
    "ts_render_fwd_n": (_st, [C.POINTER(TsPlan), _vp, _vp, _vp, _vp, _vp, _vp]),
    "ts_render_bwd_n": (_st, [C.POINTER(TsPlan), _vp, _vp, _vp, _vp, _vp, C.POINTER(TsMapGrad), _vp]),
    "ts_face_stats": (_st, [C.POINTER(TsPlan), _vp, _vp, _vp, _vp, _vp, _vp]),
    "ts_covisibility": (_st, [C.POINTER(TsPlan), _vp, _vp, _vp]),
    "ts_normal_loss": (_st, [C.POINTER(TsPlan), _vp, _vp, _vp, C.c_float, _vp, _vp, _vp]),
    "ts_render_bwd": (_st, [C.POINTER(TsPlan), _vp, _vp, _vp, _vp, C.POINTER(TsMapGrad), _vp]),
    "ts_render_step_l1": (_st, [C.POINTER(TsPlan), _vp, _vp, _vp, C.c_float, _vp, _vp, _vp, _vp, _vp, _vp,
                                C.POINTER(TsMapGrad), _vp]),
    "ts_pose_grad": (_st, [C.POINTER(TsPlan), _vp, _vp, _vp]),
    "ts_l1_loss": (_st, [C.POINTER(TsPlan), _vp, _vp, _vp, _vp, _vp, C.c_float, _vp, _vp, _vp, _vp]),
    "ts_pose_apply": (_st, [C.POINTER(TsPlan), _vp, _vp, _vp]),
    "ts_equilateral": (_st, [C.POINTER(TsPlan), C.POINTER(TsMap), _vp, C.c_size_t, C.c_float, _vp,
                             C.POINTER(TsMapGrad), _vp]),
    "ts_pho_loss": (_st, [C.POINTER(TsPlan), _vp, _vp, _vp, _vp, _vp, C.c_float, C.c_float, _vp, _vp, _vp, _vp]),
    "ts_l1_loss_noalloc": (_st, [C.POINTER(TsCamera), _i32, _vp, _vp, _vp, _vp, C.c_float, _vp, _vp, _vp, _vp]),
    "ts_pose_adam": (_st, [C.POINTER(TsPlan), _vp, _vp, _vp, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float,
                           _vp]),
    "ts_sync_status": (_st, [C.POINTER(TsPlan), _vp, _vp, C.POINTER(TsCounters)]),
    "ts_plan_layout": (_st, [C.POINTER(TsPlan), _vp, _vp, _vp, _vp]),
    "ts_debug_copy": (_st, [C.POINTER(TsPlan), _vp, _i32, _vp, _sz, _vp]),
    "ts_set_stage_events": (_st, [C.POINTER(TsPlan), _vp]),
    "ts_debug_timeout_probe": (_st, [C.POINTER(TsPlan), _vp, C.c_uint32, _vp]),
    "ts_status_string": (C.c_char_p, [_st]),
}

_lib = None


def lib():
    """The loaded libts (raises ImportError if the in-tree library is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libts.so is not built at {LIB_PATH}; run `python -c 'import __graft_entry__ as g; "
                              f"g.build()'` (no CPU fallback exists)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int, what: str):
    if status != 0:
        raise TsError(status, what)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return int(t.data_ptr())


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ----------------------------------------------------------------------------- host-side calls
def ts_default_params(**overrides) -> TsRasterParams:
    p = TsRasterParams()
    lib().ts_default_params(C.byref(p))
    for k, v in overrides.items():
        if k == "bg":
            p.bg = (C.c_float * 3)(*v)
        else:
            setattr(p, k, v)
    return p


def cameras(cams) -> "C.Array":
    """ts_camera array from an array [V, 6] of fx, fy, cx, cy, W, H."""
    cams = np.asarray(cams, np.float64)
    arr = (TsCamera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = TsCamera(float(c[0]), float(c[1]), float(c[2]), float(c[3]), int(c[4]), int(c[5]))
    return arr


def ts_plan_init(cams, n_faces: int, params: TsRasterParams, pair_capacity: int = 0) -> TsPlan:
    plan = TsPlan()
    arr = cameras(cams)
    _check(lib().ts_plan_init(C.byref(plan), arr, len(arr), int(n_faces), C.byref(params), int(pair_capacity)),
           "ts_plan_init")
    return plan


def ts_workspace_size(plan: TsPlan) -> int:
    return int(lib().ts_workspace_size(C.byref(plan)))


def ts_plan_layout(plan: TsPlan, n_views: int):
    pix = np.zeros(n_views + 1, np.int64)
    tiles = np.zeros(n_views + 1, np.int64)
    tx = np.zeros(n_views, np.int32)
    ty = np.zeros(n_views, np.int32)
    _check(lib().ts_plan_layout(C.byref(plan), pix.ctypes.data, tiles.ctypes.data, tx.ctypes.data, ty.ctypes.data),
           "ts_plan_layout")
    return dict(pix_off=pix, tile_off=tiles, tiles_x=tx, tiles_y=ty)


def ts_status_string(s: int) -> str:
    return lib().ts_status_string(s).decode()


# ----------------------------------------------------------------------------- device calls
def make_map(pos, col, opa, faces=None, sigma=None) -> TsMap:
    """TsMap over structure-of-arrays tensors: pos [3, N], col [3, N], opa [N] (float32, CUDA,
    contiguous), faces int32 [M, 3] or None (soup), sigma [M] per-face exponents or None."""
    n = pos.shape[1]
    m = faces.shape[0] if faces is not None else n // 3
    s = pos.stride(0) * pos.element_size()
    sc = col.stride(0) * col.element_size()
    b, c = pos.data_ptr(), col.data_ptr()
    return TsMap(b, b + s, b + 2 * s, c, c + sc, c + 2 * sc, opa.data_ptr(), _ptr(faces), n, m, _ptr(sigma))


def make_grad(gpos=None, gcol=None, gopa=None, gsigma=None) -> TsMapGrad:
    g = TsMapGrad()
    if gsigma is not None:
        g.gsigma = gsigma.data_ptr()
    if gpos is not None:
        s = gpos.stride(0) * gpos.element_size()
        g.gpx, g.gpy, g.gpz = gpos.data_ptr(), gpos.data_ptr() + s, gpos.data_ptr() + 2 * s
    if gcol is not None:
        s = gcol.stride(0) * gcol.element_size()
        g.gcr, g.gcg, g.gcb = gcol.data_ptr(), gcol.data_ptr() + s, gcol.data_ptr() + 2 * s
    if gopa is not None:
        g.gop = gopa.data_ptr()
    return g


def ts_workspace_init(plan, ws, stream=None):
    _check(lib().ts_workspace_init(C.byref(plan), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)),
           "ts_workspace_init")


def ts_project(plan, tsmap: TsMap, poses, ws, stream=None):
    _check(lib().ts_project(C.byref(plan), C.byref(tsmap), _ptr(poses), _ptr(ws), ws.numel() * ws.element_size(),
                            _stream(stream)), "ts_project")


def ts_bin(plan, ws, stream=None):
    _check(lib().ts_bin(C.byref(plan), _ptr(ws), _stream(stream)), "ts_bin")


def ts_render_fwd(plan, ws, color, depth, alpha, stream=None):
    _check(lib().ts_render_fwd(C.byref(plan), _ptr(ws), _ptr(color), _ptr(depth), _ptr(alpha), _stream(stream)),
           "ts_render_fwd")


def ts_render_fwd_n(plan, ws, color, depth, alpha, normal, stream=None):
    _check(lib().ts_render_fwd_n(C.byref(plan), _ptr(ws), _ptr(color), _ptr(depth), _ptr(alpha), _ptr(normal),
                                 _stream(stream)), "ts_render_fwd_n")


def ts_render_bwd_n(plan, ws, dC, dD, dA, dN, grad: Optional[TsMapGrad], stream=None):
    g = grad if grad is not None else TsMapGrad()
    _check(lib().ts_render_bwd_n(C.byref(plan), _ptr(ws), _ptr(dC), _ptr(dD), _ptr(dA), _ptr(dN), C.byref(g),
                                 _stream(stream)), "ts_render_bwd_n")


def ts_face_stats(plan, ws, coverage=None, area=None, visible=None, n_visible=None, stream=None):
    _check(lib().ts_face_stats(C.byref(plan), _ptr(ws), _ptr(coverage), _ptr(area), _ptr(visible), _ptr(n_visible),
                               _stream(stream)), "ts_face_stats")


def ts_covisibility(plan, visible, iou, stream=None):
    _check(lib().ts_covisibility(C.byref(plan), _ptr(visible), _ptr(iou), _stream(stream)), "ts_covisibility")


def ts_normal_loss(plan, ws, normal, tgt_normal, weight, loss, dN, stream=None):
    _check(lib().ts_normal_loss(C.byref(plan), _ptr(ws), _ptr(normal), _ptr(tgt_normal), float(weight), _ptr(loss),
                                _ptr(dN), _stream(stream)), "ts_normal_loss")


def ts_render_bwd(plan, ws, dC, dD, dA, grad: Optional[TsMapGrad], stream=None):
    g = grad if grad is not None else TsMapGrad()
    _check(lib().ts_render_bwd(C.byref(plan), _ptr(ws), _ptr(dC), _ptr(dD), _ptr(dA), C.byref(g), _stream(stream)),
           "ts_render_bwd")


def ts_render_step_l1(plan, ws, tgt_color, tgt_depth, lambda_dep, color, depth, alpha, loss, dC, dD,
                      grad: Optional[TsMapGrad], stream=None):
    g = grad if grad is not None else TsMapGrad()
    _check(lib().ts_render_step_l1(C.byref(plan), _ptr(ws), _ptr(tgt_color), _ptr(tgt_depth), float(lambda_dep),
                                   _ptr(color), _ptr(depth), _ptr(alpha), _ptr(loss), _ptr(dC), _ptr(dD), C.byref(g),
                                   _stream(stream)), "ts_render_step_l1")


def ts_equilateral(plan, tsmap: TsMap, ws, weight, loss, grad: Optional[TsMapGrad] = None, stream=None):
    _check(lib().ts_equilateral(C.byref(plan), C.byref(tsmap), _ptr(ws), ws.numel() * ws.element_size(),
                                float(weight), _ptr(loss), C.byref(grad) if grad is not None else None,
                                _stream(stream)), "ts_equilateral")


def ts_pose_grad(plan, ws, dtau, stream=None):
    _check(lib().ts_pose_grad(C.byref(plan), _ptr(ws), _ptr(dtau), _stream(stream)), "ts_pose_grad")


def ts_l1_loss(plan, ws, color, depth, tgt_color, tgt_depth, lambda_dep, loss, dC, dD, stream=None):
    _check(lib().ts_l1_loss(C.byref(plan), _ptr(ws), _ptr(color), _ptr(depth), _ptr(tgt_color), _ptr(tgt_depth),
                            float(lambda_dep), _ptr(loss), _ptr(dC), _ptr(dD), _stream(stream)), "ts_l1_loss")


def ts_pho_loss(plan, ws, color, depth, tgt_color, tgt_depth, lambda_ssim, lambda_dep, loss, dC, dD, stream=None):
    _check(lib().ts_pho_loss(C.byref(plan), _ptr(ws), _ptr(color), _ptr(depth), _ptr(tgt_color), _ptr(tgt_depth),
                             float(lambda_ssim), float(lambda_dep), _ptr(loss), _ptr(dC), _ptr(dD), _stream(stream)),
           "ts_pho_loss")


def check_noalloc_args(cams, color, depth, tgt_color, tgt_depth, loss, dC, dD):
    """Host-side checks of ts_l1_loss_noalloc's tensors, before anything is launched.

    The entry point has no plan that fixes the image sizes: the cameras alone set how far its
    kernels read and write.  So every tensor must be float32, contiguous and on one CUDA device,
    with 3 * sum(W * H) elements for the colour images, sum(W * H) for the depth images and
    n_views for the loss.  Raises ValueError otherwise."""
    arr = cameras(cams)
    P = int(sum(int(c.width) * int(c.height) for c in arr))
    want = {"color": 3 * P, "depth": P, "tgt_color": 3 * P, "tgt_depth": P, "loss": len(arr), "dC": 3 * P, "dD": P}
    ts = dict(color=color, depth=depth, tgt_color=tgt_color, tgt_depth=tgt_depth, loss=loss, dC=dC, dD=dD)
    for name, t in ts.items():
        if t is None:
            raise ValueError(f"ts_l1_loss_noalloc: {name} is required")
        if str(t.dtype) != "torch.float32" or not t.is_contiguous():
            raise ValueError(f"ts_l1_loss_noalloc: {name} must be a contiguous float32 tensor")
        if t.numel() != want[name]:
            raise ValueError(f"ts_l1_loss_noalloc: {name} has {t.numel()} elements, the cameras need {want[name]}")
    dev = None
    for name, t in ts.items():
        if t.device.type != "cuda":
            raise ValueError(f"ts_l1_loss_noalloc: {name} must be on a CUDA device")
        if dev is not None and t.device != dev:
            raise ValueError("ts_l1_loss_noalloc: all tensors must be on one device")
        dev = t.device
    return arr, dev


def ts_l1_loss_noalloc(cams, color, depth, tgt_color, tgt_depth, lambda_dep, loss, dC, dD, stream=None):
    """The L1 loss without a plan or workspace (static device scratch); see include/ts_api.h.
    The call runs with the tensors' device current, so that the scratch array and the default
    stream are that device's."""
    import torch
    arr, dev = check_noalloc_args(cams, color, depth, tgt_color, tgt_depth, loss, dC, dD)
    with torch.cuda.device(dev):
        _check(lib().ts_l1_loss_noalloc(arr, len(arr), _ptr(color), _ptr(depth), _ptr(tgt_color), _ptr(tgt_depth),
                                        float(lambda_dep), _ptr(loss), _ptr(dC), _ptr(dD), _stream(stream)),
               "ts_l1_loss_noalloc")


def ts_pose_adam(plan, poses, dtau, state, lr_rho, lr_theta, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().ts_pose_adam(C.byref(plan), _ptr(poses), _ptr(dtau), _ptr(state), float(lr_rho), float(lr_theta),
                              float(beta1), float(beta2), float(eps), _stream(stream)), "ts_pose_adam")


def ts_pose_apply(plan, poses, step, stream=None):
    _check(lib().ts_pose_apply(C.byref(plan), _ptr(poses), _ptr(step), _stream(stream)), "ts_pose_apply")


def ts_sync_status(plan, ws, stream=None, raise_on_error: bool = True) -> dict:
    c = TsCounters()
    s = lib().ts_sync_status(C.byref(plan), _ptr(ws), _stream(stream), C.byref(c))
    d = c.as_dict()
    d["status"] = STATUS.get(s, s)
    if raise_on_error:
        _check(s, "ts_sync_status")
    return d


def ts_debug_copy(plan, ws, what: str, dst, stream=None):
    _check(lib().ts_debug_copy(C.byref(plan), _ptr(ws), DEBUG[what], _ptr(dst), dst.numel() * dst.element_size(),
                               _stream(stream)), f"ts_debug_copy({what})")


def ts_debug_timeout_probe(plan, ws, limit_us: int, stream=None):
    _check(lib().ts_debug_timeout_probe(C.byref(plan), _ptr(ws), int(limit_us), _stream(stream)),
           "ts_debug_timeout_probe")


def ts_set_stage_events(plan, events: Optional[Sequence]):
    """events: 2 * len(STAGES) torch.cuda.Event(enable_timing=True) objects, or None."""
    if events is None:
        _check(lib().ts_set_stage_events(C.byref(plan), None), "ts_set_stage_events")
        return
    arr = (C.c_void_p * len(events))(*[e.cuda_event for e in events])
    _check(lib().ts_set_stage_events(C.byref(plan), C.cast(arr, C.c_void_p)), "ts_set_stage_events")
