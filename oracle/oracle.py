"""Python binding of the CPU oracle (``ts_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``.  The product package never
imports this module.

The oracle follows Triangle Splatting SLAM Eq. 1-4 and their adjoint (see the
header of ``ts_oracle.cpp``).  Inputs are plain numpy arrays from ``ts_synth``;
everything is passed to C as float64 so that finite differences can perturb
inputs below float32 resolution.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ts_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle (or its k-th planted-mistake variant) and return the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    name = "libts_oracle.so" if mutant == 0 else f"libts_oracle_m{mutant}.so"
    out = os.path.join(_BUILD, name)
    with _lock:
        if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
            tmp = out + f".tmp{os.getpid()}"
            cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                   "-shared", "-fPIC", f"-DORACLE_MUTANT={mutant}", _SRC, "-o", tmp]
            subprocess.run(cmd, check=True)
            os.replace(tmp, out)
    return out


class _Params(C.Structure):
    _fields_ = [("sigma", C.c_double), ("alpha_min", C.c_double), ("alpha_max", C.c_double),
                ("T_min", C.c_double), ("z_near", C.c_double), ("r_min", C.c_double),
                ("bg", C.c_double * 3), ("tile_w", C.c_int32), ("tile_h", C.c_int32),
                ("fp64", C.c_int32), ("n_threads", C.c_int32), ("min_opacity", C.c_int32)]


class _Scene(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("col", C.c_void_p), ("opa", C.c_void_p), ("faces", C.c_void_p),
                ("n_vertices", C.c_int64), ("n_faces", C.c_int64), ("cams", C.c_void_p),
                ("poses", C.c_void_p), ("n_views", C.c_int32), ("sigma_face", C.c_void_p)]


@dataclass
class Params:
    """Rasterization parameters.  sigma = 0.5 is Table S5; the rest are readings (see ts_oracle.cpp)."""
    sigma: float = 0.5
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    T_min: float = 1e-4
    z_near: float = 0.01
    r_min: float = 0.01
    bg: Sequence[float] = (0.0, 0.0, 0.0)
    tile_w: int = 16
    tile_h: int = 16
    fp64: bool = False
    n_threads: int = 0
    min_opacity: bool = False

    def c(self) -> _Params:
        p = _Params()
        for k in ("sigma", "alpha_min", "alpha_max", "T_min", "z_near", "r_min"):
            setattr(p, k, float(getattr(self, k)))
        p.bg = (C.c_double * 3)(*[float(b) for b in self.bg])
        p.tile_w, p.tile_h = int(self.tile_w), int(self.tile_h)
        p.fp64 = 1 if self.fp64 else 0
        p.n_threads = int(self.n_threads)
        p.min_opacity = 1 if self.min_opacity else 0
        return p


@dataclass
class SceneArrays:
    """float64 copies of a scene that stay alive while the C side reads them."""
    pos: np.ndarray
    col: np.ndarray
    opa: np.ndarray
    faces: Optional[np.ndarray]
    cams: np.ndarray
    poses: np.ndarray
    sigma: Optional[np.ndarray] = None
    keep: list = field(default_factory=list)

    @staticmethod
    def of(scene, pos=None, col=None, opa=None, poses=None, sigma=None) -> "SceneArrays":
        f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
        faces = None if scene.faces is None else np.ascontiguousarray(scene.faces, dtype=np.int32)
        sig = sigma if sigma is not None else getattr(scene, "sigma", None)
        return SceneArrays(f64(scene.pos if pos is None else pos), f64(scene.col if col is None else col),
                           f64(scene.opa if opa is None else opa), faces, f64(scene.cams),
                           f64(scene.poses if poses is None else poses), None if sig is None else f64(sig))

    def c(self) -> _Scene:
        s = _Scene()
        s.pos, s.col, s.opa = self.pos.ctypes.data, self.col.ctypes.data, self.opa.ctypes.data
        s.faces = None if self.faces is None else self.faces.ctypes.data
        s.n_vertices = len(self.pos)
        s.n_faces = len(self.faces) if self.faces is not None else len(self.pos) // 3
        s.cams, s.poses = self.cams.ctypes.data, self.poses.ctypes.data
        s.n_views = len(self.cams)
        s.sigma_face = None if self.sigma is None else self.sigma.ctypes.data
        return s

    @property
    def n_faces(self) -> int:
        return len(self.faces) if self.faces is not None else len(self.pos) // 3

    def pix_offsets(self) -> np.ndarray:
        hw = [int(c[4]) * int(c[5]) for c in self.cams]
        return np.concatenate([[0], np.cumsum(hw)]).astype(np.int64)


def _ptr(a):
    return None if a is None else a.ctypes.data


class Oracle:
    """Handle on one build of the oracle library (``mutant`` > 0 loads a planted-mistake variant)."""

    def __init__(self, mutant: int = 0):
        self.mutant = mutant
        self.lib = C.CDLL(build(mutant))
        L = self.lib
        vp, i64, i32, d = C.c_void_p, C.c_int64, C.c_int32, C.c_double
        L.oracle_project.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.oracle_bin.argtypes = [vp, vp, vp, vp, i64, vp]
        L.oracle_bin.restype = i64
        L.oracle_total_tiles.argtypes = [vp, vp]
        L.oracle_total_tiles.restype = i64
        L.oracle_forward.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
        L.oracle_pixel_trace.argtypes = [vp, vp, i32, i32, i32, vp, vp, vp, i32, vp]
        L.oracle_pixel_trace.restype = i32
        L.oracle_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.oracle_backward_ex.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.oracle_normal_loss.argtypes = [vp, vp, vp, d, vp, vp]
        L.oracle_normal_loss.restype = d
        L.oracle_l1_loss.argtypes = [vp, vp, vp, vp, vp, d, vp, vp, vp]
        L.oracle_l1_loss.restype = d
        L.oracle_pho_loss.argtypes = [vp, vp, vp, vp, vp, d, d, vp, vp, vp, vp, vp]
        L.oracle_pho_loss.restype = d
        L.oracle_face_stats.argtypes = [vp, vp, vp, vp]
        L.oracle_equilateral.argtypes = [vp, vp]
        L.oracle_equilateral.restype = d
        L.oracle_window.argtypes = [vp, d, d, d, vp]
        L.oracle_window.restype = d
        L.oracle_se3_exp.argtypes = [vp, vp]
        L.oracle_pose_left_update.argtypes = [vp, vp, vp]
        assert L.oracle_mutant() == mutant

    # -- Eq. 1 projection and culling ---------------------------------------------------
    def project(self, sa: SceneArrays, prm: Params):
        VM = len(sa.cams) * sa.n_faces
        rect = np.empty((VM, 4), np.int32)
        pix = np.empty((VM, 4), np.int32)
        zbits = np.empty(VM, np.uint32)
        count = np.empty(VM, np.uint32)
        uvz = np.empty((VM, 9), np.float64)
        sc, p = sa.c(), prm.c()
        self.lib.oracle_project(C.byref(sc), C.byref(p), _ptr(rect), _ptr(pix), _ptr(zbits), _ptr(count), _ptr(uvz))
        return dict(rect=rect, pix=pix, zbits=zbits, count=count, uvz=uvz)

    # -- depth-sorted tile lists -------------------------------------------------------
    def bin(self, sa: SceneArrays, prm: Params):
        sc, p = sa.c(), prm.c()
        n_tiles = self.lib.oracle_total_tiles(C.byref(sc), C.byref(p))
        n = self.lib.oracle_bin(C.byref(sc), C.byref(p), None, None, 0, None)
        keys = np.empty(max(n, 1), np.uint64)
        ids = np.empty(max(n, 1), np.uint32)
        ranges = np.empty((n_tiles, 2), np.int64)
        self.lib.oracle_bin(C.byref(sc), C.byref(p), _ptr(keys), _ptr(ids), n, _ptr(ranges))
        return dict(keys=keys[:n], ids=ids[:n], ranges=ranges, n_tiles=n_tiles)

    # -- Eq. 4 forward -------------------------------------------------------------------
    def forward(self, sa: SceneArrays, prm: Params):
        off = sa.pix_offsets()
        P = int(off[-1])
        color, normal = np.empty(3 * P), np.empty(3 * P)
        depth, alpha, T = np.empty(P), np.empty(P), np.empty(P)
        n_last = np.empty(P, np.int32)
        sc, p = sa.c(), prm.c()
        self.lib.oracle_forward(C.byref(sc), C.byref(p), _ptr(color), _ptr(depth), _ptr(alpha), _ptr(T), _ptr(n_last),
                                _ptr(normal))
        return dict(color=color, depth=depth, alpha=alpha, T_final=T, n_last=n_last, normal=normal, pix_off=off)

    def face_stats(self, sa: SceneArrays, prm: Params):
        """Per (view, face): pixel coverage of the forward walk and projected area (Sec. 3.4)."""
        VM = len(sa.cams) * sa.n_faces
        cov = np.zeros(VM, np.uint32)
        area = np.zeros(VM)
        sc, p = sa.c(), prm.c()
        self.lib.oracle_face_stats(C.byref(sc), C.byref(p), _ptr(cov), _ptr(area))
        return dict(coverage=cov, area=area)

    def pixel_trace(self, sa: SceneArrays, prm: Params, view: int, x: int, y: int, cap: int = 4096):
        faces = np.empty(cap, np.int32)
        alphas, Tb = np.empty(cap), np.empty(cap)
        Tf = C.c_double()
        sc, p = sa.c(), prm.c()
        n = self.lib.oracle_pixel_trace(C.byref(sc), C.byref(p), view, x, y, _ptr(faces), _ptr(alphas), _ptr(Tb), cap,
                                        C.byref(Tf))
        n = min(n, cap)
        return dict(faces=faces[:n], alpha=alphas[:n], T_before=Tb[:n], T_final=Tf.value)

    # -- adjoint ---------------------------------------------------------------------------
    def backward(self, sa: SceneArrays, prm: Params, dC, dD=None, dA=None, dN=None):
        N = len(sa.pos)
        dpos, dcol = np.zeros((N, 3)), np.zeros((N, 3))
        dopa = np.zeros(N)
        dtau = np.zeros((len(sa.cams), 6))
        dtau_abs = np.zeros((len(sa.cams), 6))
        dsigma = np.zeros(sa.n_faces) if sa.sigma is not None else None
        f = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
        dC, dD, dA, dN = f(dC), f(dD), f(dA), f(dN)
        sc, p = sa.c(), prm.c()
        self.lib.oracle_backward_ex(C.byref(sc), C.byref(p), _ptr(dC), _ptr(dD), _ptr(dA), _ptr(dN), _ptr(dpos),
                                    _ptr(dcol), _ptr(dopa), _ptr(dtau), _ptr(dtau_abs), _ptr(dsigma))
        return dict(dpos=dpos, dcol=dcol, dopa=dopa, dtau=dtau, dtau_abs=dtau_abs, dsigma=dsigma)

    def l1_loss(self, sa: SceneArrays, color, depth, tgt_color, tgt_depth, lambda_dep: float = 0.05):
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
        color, depth, tgt_color, tgt_depth = f(color), f(depth), f(tgt_color), f(tgt_depth)
        V = len(sa.cams)
        loss_v = np.empty(V)
        dC, dD = np.empty_like(color), np.empty_like(depth)
        sc = sa.c()
        tot = self.lib.oracle_l1_loss(C.byref(sc), _ptr(color), _ptr(depth), _ptr(tgt_color), _ptr(tgt_depth),
                                      float(lambda_dep), _ptr(loss_v), _ptr(dC), _ptr(dD))
        return dict(loss=tot, loss_v=loss_v, dC=dC, dD=dD)

    def pho_loss(self, sa: SceneArrays, color, depth, tgt_color, tgt_depth, lambda_ssim: float = 0.2,
                 lambda_dep: float = 0.05, grads: bool = True):
        """Eq. 8-10: (1 - lambda) L1 + lambda D-SSIM colour terms plus the L1 depth term, per view."""
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
        color, depth, tgt_color, tgt_depth = f(color), f(depth), f(tgt_color), f(tgt_depth)
        V = len(sa.cams)
        loss_v = np.empty(V)
        dC = np.empty_like(color) if grads else None
        dD = np.empty_like(depth) if grads else None
        dC_abs = np.empty_like(color) if grads else None
        smap = np.empty_like(color)
        sc = sa.c()
        tot = self.lib.oracle_pho_loss(C.byref(sc), _ptr(color), _ptr(depth), _ptr(tgt_color), _ptr(tgt_depth),
                                       float(lambda_ssim), float(lambda_dep), _ptr(loss_v), _ptr(dC), _ptr(dD),
                                       _ptr(smap), _ptr(dC_abs))
        return dict(loss=tot, loss_v=loss_v, dC=dC, dD=dD, ssim_map=smap, dC_abs=dC_abs)

    def normal_loss(self, sa: SceneArrays, normal, tgt_normal, weight: float = 1.0):
        """Eq. 12: sum over pixels with a sensor normal of (1 - N . Nbar) / HW, per view; dN of weight x that."""
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
        normal, tgt_normal = f(normal), f(tgt_normal)
        loss_v = np.empty(len(sa.cams))
        dN = np.empty_like(normal)
        sc = sa.c()
        tot = self.lib.oracle_normal_loss(C.byref(sc), _ptr(normal), _ptr(tgt_normal), float(weight), _ptr(loss_v),
                                          _ptr(dN))
        return dict(loss=tot, loss_v=loss_v, dN=dN)

    def equilateral(self, sa: SceneArrays, grads: bool = True):
        """Eq. 14: mean over faces of the mean squared deviation of the angle cosines from 0.5."""
        dpos = np.zeros((len(sa.pos), 3)) if grads else None
        sc = sa.c()
        e = self.lib.oracle_equilateral(C.byref(sc), _ptr(dpos))
        return dict(loss=e, dpos=dpos)

    # -- small pieces used by the pins ---------------------------------------------------
    def window(self, tri2d, sigma: float, px: float, py: float):
        q = np.ascontiguousarray(np.asarray(tri2d, np.float64).reshape(6))
        lam = np.empty(3)
        I = self.lib.oracle_window(_ptr(q), float(sigma), float(px), float(py), _ptr(lam))
        return I, lam

    def se3_exp(self, tau) -> np.ndarray:
        t = np.ascontiguousarray(tau, np.float64)
        out = np.empty(12)
        self.lib.oracle_se3_exp(_ptr(t), _ptr(out))
        return out

    def pose_left_update(self, tau, pose) -> np.ndarray:
        t = np.ascontiguousarray(tau, np.float64)
        p = np.ascontiguousarray(pose, np.float64)
        out = np.empty(12)
        self.lib.oracle_pose_left_update(_ptr(t), _ptr(p), _ptr(out))
        return out


def pack_targets(scene) -> tuple:
    """Targets of a ts_synth scene packed like the images (colour [3][H][W] per view, back to back)."""
    tc = np.concatenate([t.reshape(-1) for t in scene.tgt_color]).astype(np.float64)
    td = np.concatenate([t.reshape(-1) for t in scene.tgt_depth]).astype(np.float64)
    return tc, td
