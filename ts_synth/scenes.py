"""Seeded synthetic scenes, cameras, poses and targets (numpy, PCG64).

Conventions shared by every consumer:

* vertices are float32 structure-of-arrays: ``pos[N,3]`` (world metres),
  ``col[N,3]`` (RGB), ``opa[N]`` (vertex opacity in [0, 1]);
* ``faces`` is ``int32[M,3]`` or ``None``; ``None`` means triangle-soup mode,
  where face ``m`` uses vertices ``3m, 3m+1, 3m+2`` (the map layout used while
  a triangle-splatting map is being optimised, Sec. 3.4 "Densification");
* ``cams[V,6]`` holds ``fx, fy, cx, cy, W, H`` of a pinhole camera;
* ``poses[V,12]`` holds the world-to-camera transform T_CW as a row-major
  rotation followed by the translation, so that ``v_C = R v_W + t``; the camera
  looks along +z with +x right and +y down.

Nothing here evaluates the rasterizer: the arrays are inputs only.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class Scene:
    pos: np.ndarray
    col: np.ndarray
    opa: np.ndarray
    faces: Optional[np.ndarray]
    cams: np.ndarray
    poses: np.ndarray
    tgt_color: List[np.ndarray] = field(default_factory=list)
    tgt_depth: List[np.ndarray] = field(default_factory=list)
    sigma: Optional[np.ndarray] = None  # per-face window exponents (learnable-sigma variant), [M]

    @property
    def n_faces(self) -> int:
        return len(self.faces) if self.faces is not None else len(self.pos) // 3

    @property
    def n_views(self) -> int:
        return len(self.cams)

    def pixels(self) -> int:
        return int(sum(int(c[4]) * int(c[5]) for c in self.cams))

    def subset_views(self, idx) -> "Scene":
        idx = list(idx)
        return Scene(self.pos, self.col, self.opa, self.faces,
                     self.cams[idx].copy(), self.poses[idx].copy(),
                     [self.tgt_color[i] for i in idx] if self.tgt_color else [],
                     [self.tgt_depth[i] for i in idx] if self.tgt_depth else [])


# --------------------------------------------------------------------------
# small helpers (random geometry)
# --------------------------------------------------------------------------

def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random rotations (Shoemake's quaternion method), float64 [n,3,3]."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    q = np.stack([np.sqrt(1 - u1) * np.sin(2 * np.pi * u2),
                  np.sqrt(1 - u1) * np.cos(2 * np.pi * u2),
                  np.sqrt(u1) * np.sin(2 * np.pi * u3),
                  np.sqrt(u1) * np.cos(2 * np.pi * u3)], axis=1)
    x, y, z, w = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _triangle_sides(rng: np.random.Generator, n: int, lo: float, hi: float) -> np.ndarray:
    """Side lengths ~U[lo, hi], kept only if each side is < (1/1.1) x the sum of the others."""
    out = np.empty((0, 3))
    while len(out) < n:
        s = rng.uniform(lo, hi, size=(2 * (n - len(out)) + 16, 3))
        a, b, c = s.T
        ok = (a + b > 1.1 * c) & (b + c > 1.1 * a) & (a + c > 1.1 * b)
        out = np.concatenate([out, s[ok]])
    return out[:n]


def _flat_triangles(sides: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Planar triangles with the given sides, centroid at 0, rotated in-plane by psi. [n,3,2]"""
    a, b, c = sides.T
    cos_a = np.clip((b * b + c * c - a * a) / (2 * b * c), -1.0, 1.0)
    sin_a = np.sqrt(1.0 - cos_a * cos_a)
    P = np.zeros((len(sides), 3, 2))
    P[:, 1, 0] = c
    P[:, 2, 0] = b * cos_a
    P[:, 2, 1] = b * sin_a
    P -= P.mean(axis=1, keepdims=True)
    cp, sp = np.cos(psi), np.sin(psi)
    rot = np.stack([np.stack([cp, -sp], 1), np.stack([sp, cp], 1)], 1)  # [n,2,2]
    return np.einsum('nij,nkj->nki', rot, P)


def _tangent_basis(nrm: np.ndarray):
    """Two unit tangents orthogonal to each (unit) normal."""
    helper = np.where(np.abs(nrm[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    t1 = np.cross(nrm, helper)
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    t2 = np.cross(nrm, t1)
    return t1, t2


def look_at(eye, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """World-to-camera pose [12] (row-major R | t) of a camera at ``eye`` looking at ``target``."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    right = np.cross(f, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    R = np.stack([right, down, f])          # rows: camera axes in world coordinates
    t = -R @ eye
    return np.concatenate([R.reshape(-1), t]).astype(np.float32)


def _cams(n: int, W: int, H: int, fx: float, fy: float, cx: float, cy: float) -> np.ndarray:
    return np.tile(np.array([[fx, fy, cx, cy, W, H]], np.float64), (n, 1))


def noise_targets(seed: int, cams: np.ndarray, depth_lo: float = 0.5, depth_hi: float = 4.0):
    """Per-view target colour ~U[0,1] per pixel and channel, target depth ~U[lo,hi]."""
    rng = np.random.default_rng(seed)
    tc, td = [], []
    for c in cams:
        W, H = int(c[4]), int(c[5])
        tc.append(rng.random((3, H, W), dtype=np.float32))
        td.append(rng.uniform(depth_lo, depth_hi, size=(H, W)).astype(np.float32))
    return tc, td



def loss_images(seed: int, cams: np.ndarray, shift: int = 2, noise: float = 0.05, flat: float = 0.25,
                invalid: float = 0.1):
    """Packed per-view image pairs for the loss: a "render" C of smooth noise (per channel, the
    clamp to [0, 1] of 0.5 + 0.5 * a sum of 4 random sinusoids in x, y) with a ``flat`` fraction of
    8 x 8 blocks set to a constant colour (the flat regions of real renders), and a target Cbar =
    C shifted by ``shift`` pixels plus N(0, noise), clamped to [0, 1]; depth D ~ U[0.5, 4] and
    Dbar = D (1 + 0.01 N(0, 1)) with an ``invalid`` fraction of zeros.  Returns float32 flat arrays
    (C [3P], D [P], Cbar [3P], Dbar [P]) in the library's packing."""
    rng = np.random.default_rng(seed)
    Cs, Ds, tCs, tDs = [], [], [], []
    for c in cams:
        W, H = int(c[4]), int(c[5])
        yy, xx = np.mgrid[0:H + shift, 0:W + shift].astype(np.float64)
        img = np.empty((3, H + shift, W + shift))
        for ch in range(3):
            acc = np.zeros_like(xx)
            for _ in range(4):
                w = rng.uniform(0.05, 0.5, size=2)
                acc += np.sin(w[0] * xx + w[1] * yy + rng.uniform(0, 2 * np.pi))
            img[ch] = np.clip(0.5 + 0.5 * acc / 2.0, 0.0, 1.0)
        for by in range(0, H + shift, 8):
            for bx in range(0, W + shift, 8):
                if rng.random() < flat:
                    img[:, by:by + 8, bx:bx + 8] = rng.random((3, 1, 1))
        C = img[:, :H, :W]
        tC = np.clip(img[:, shift:, shift:] + rng.normal(0.0, noise, size=(3, H, W)), 0.0, 1.0)
        D = rng.uniform(0.5, 4.0, size=(H, W))
        tD = D * (1.0 + 0.01 * rng.normal(size=(H, W)))
        tD[rng.random((H, W)) < invalid] = 0.0
        Cs.append(C.ravel()); tCs.append(tC.ravel()); Ds.append(D.ravel()); tDs.append(tD.ravel())
    f = lambda xs: np.concatenate(xs).astype(np.float32)  # noqa: E731
    return f(Cs), f(Ds), f(tCs), f(tDs)


def sensor_normals(seed: int, cams: np.ndarray, invalid: float = 0.1) -> np.ndarray:
    """Packed per-view sensor normal maps [3][H][W] (float32, flat): unit vectors drawn uniformly on
    the hemisphere facing the camera (negative z), with an ``invalid`` fraction of pixels set to
    the zero vector (no normal)."""
    rng = np.random.default_rng(seed)
    out = []
    for c in cams:
        HW = int(c[4]) * int(c[5])
        n = rng.normal(size=(3, HW))
        n /= np.linalg.norm(n, axis=0)
        n[2] = -np.abs(n[2])
        n[:, rng.random(HW) < invalid] = 0.0
        out.append(n.ravel())
    return np.concatenate(out).astype(np.float32)

# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def random_triangles_scene(seed: int = 1, n_faces: int = 2000, W: int = 160, H: int = 120,
                           f: float = 150.0, z_lo: float = 0.5, z_hi: float = 4.0,
                           side_lo: float = 0.02, side_hi: float = 0.10,
                           opa_lo: float = 0.3, opa_hi: float = 1.0,
                           target_seed: Optional[int] = 2) -> Scene:
    """Random triangle soup in front of one camera at the identity pose.

    Centroids sit at a uniform pixel and a uniform depth, back-projected through
    the pinhole; sides are uniform with a 10% triangle-inequality margin and each
    triangle gets a uniform random 3D orientation.
    """
    rng = np.random.default_rng(seed)
    cx, cy = W / 2.0, H / 2.0
    u = rng.uniform(0, W, n_faces)
    v = rng.uniform(0, H, n_faces)
    z = rng.uniform(z_lo, z_hi, n_faces)
    centre = np.stack([(u - cx) * z / f, (v - cy) * z / f, z], 1)
    sides = _triangle_sides(rng, n_faces, side_lo, side_hi)
    flat = _flat_triangles(sides, rng.uniform(0, 2 * np.pi, n_faces))
    R = _random_rotations(rng, n_faces)
    pts = centre[:, None, :] + flat[..., 0:1] * R[:, None, :, 0] + flat[..., 1:2] * R[:, None, :, 1]
    pos = pts.reshape(-1, 3).astype(np.float32)
    col = rng.random((3 * n_faces, 3), dtype=np.float32)
    opa = rng.uniform(opa_lo, opa_hi, 3 * n_faces).astype(np.float32)
    cams = _cams(1, W, H, f, f, cx, cy)
    poses = np.array([[1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0]], np.float32)
    sc = Scene(pos, col, opa, None, cams, poses)
    if target_seed is not None:
        sc.tgt_color, sc.tgt_depth = noise_targets(target_seed, cams)
    return sc


ROOM_MIN = np.array([-3.0, -2.5, 0.0])
ROOM_MAX = np.array([3.0, 2.5, 3.0])


def _room_surfaces(rng: np.random.Generator, n_objects: int = 40):
    """Planar quads (corner, edge1, edge2, normal) and spheres (centre, radius)."""
    quads = []
    lo, hi = ROOM_MIN, ROOM_MAX
    ext = hi - lo
    # six walls, normals pointing into the room
    for axis in range(3):
        a1, a2 = [k for k in range(3) if k != axis]
        for side, sgn in ((lo, 1.0), (hi, -1.0)):
            corner = lo.copy()
            corner[axis] = side[axis]
            e1 = np.zeros(3); e1[a1] = ext[a1]
            e2 = np.zeros(3); e2[a2] = ext[a2]
            n = np.zeros(3); n[axis] = sgn
            quads.append((corner, e1, e2, n))
    spheres = []
    for _ in range(n_objects):
        if rng.random() < 0.5:
            size = rng.uniform(0.2, 1.0, 3)
            c = np.array([rng.uniform(lo[0] + 0.6, hi[0] - 0.6), rng.uniform(lo[1] + 0.6, hi[1] - 0.6),
                          size[2] / 2 + rng.uniform(0.0, 1.0) * (rng.random() < 0.3)])
            bmin, bmax = c - size / 2, c + size / 2
            for axis in range(3):
                a1, a2 = [k for k in range(3) if k != axis]
                for sgn in (-1.0, 1.0):
                    if axis == 2 and sgn < 0 and bmin[2] <= 1e-6:
                        continue  # resting on the floor: bottom face hidden
                    corner = bmin.copy()
                    corner[axis] = bmax[axis] if sgn > 0 else bmin[axis]
                    e1 = np.zeros(3); e1[a1] = size[a1]
                    e2 = np.zeros(3); e2[a2] = size[a2]
                    n = np.zeros(3); n[axis] = sgn
                    quads.append((corner, e1, e2, n))
        else:
            r = rng.uniform(0.1, 0.5)
            c = np.array([rng.uniform(lo[0] + r, hi[0] - r), rng.uniform(lo[1] + r, hi[1] - r),
                          rng.uniform(r, hi[2] - r)])
            spheres.append((c, r))
    return quads, spheres


def _smooth_noise_colour(rng: np.random.Generator, pts: np.ndarray) -> np.ndarray:
    """Per-channel sum of four random plane waves, mapped into [0, 1]."""
    out = np.empty((len(pts), 3), np.float32)
    for ch in range(3):
        omega = rng.normal(0.0, 2.5, size=(4, 3))
        phase = rng.uniform(0, 2 * np.pi, 4)
        s = np.sin(pts @ omega.T + phase).sum(axis=1)
        out[:, ch] = np.clip(0.5 + 0.125 * s, 0.0, 1.0)
    return out


def room_map(seed: int, n_faces: int, side_lo: float = 0.01, side_hi: float = 0.05,
             opa_lo: float = 0.5, opa_hi: float = 1.0, jitter_deg: float = 10.0):
    """Triangle soup on a 6 x 5 x 3 m room with 40 random boxes and spheres.

    Face centres are area-weighted uniform samples on the surfaces; each face
    lies in the tangent plane with its normal jittered by up to ``jitter_deg``
    and a random in-plane rotation.  Returns (pos, col, opa) float32.
    """
    rng = np.random.default_rng(seed)
    quads, spheres = _room_surfaces(rng)
    areas = [np.linalg.norm(np.cross(e1, e2)) for (_, e1, e2, _) in quads]
    areas += [4 * np.pi * r * r for (_, r) in spheres]
    areas = np.asarray(areas)
    which = rng.choice(len(areas), size=n_faces, p=areas / areas.sum())
    centre = np.empty((n_faces, 3))
    nrm = np.empty((n_faces, 3))
    nq = len(quads)
    for k in range(len(areas)):
        sel = np.nonzero(which == k)[0]
        if len(sel) == 0:
            continue
        if k < nq:
            corner, e1, e2, n = quads[k]
            s, t = rng.random(len(sel)), rng.random(len(sel))
            centre[sel] = corner + s[:, None] * e1 + t[:, None] * e2
            nrm[sel] = n
        else:
            c, r = spheres[k - nq]
            d = rng.normal(size=(len(sel), 3))
            d /= np.linalg.norm(d, axis=1, keepdims=True)
            centre[sel] = c + r * d
            nrm[sel] = d
    # jitter the normal direction by up to jitter_deg
    t1, t2 = _tangent_basis(nrm)
    ang = np.deg2rad(rng.uniform(0, jitter_deg, n_faces))
    phi = rng.uniform(0, 2 * np.pi, n_faces)
    nrm = (np.cos(ang)[:, None] * nrm
           + np.sin(ang)[:, None] * (np.cos(phi)[:, None] * t1 + np.sin(phi)[:, None] * t2))
    t1, t2 = _tangent_basis(nrm)
    sides = _triangle_sides(rng, n_faces, side_lo, side_hi)
    flat = _flat_triangles(sides, rng.uniform(0, 2 * np.pi, n_faces))
    pts = centre[:, None, :] + flat[..., 0:1] * t1[:, None, :] + flat[..., 1:2] * t2[:, None, :]
    pos = pts.reshape(-1, 3).astype(np.float32)
    col = _smooth_noise_colour(rng, pos.astype(np.float64))
    opa = rng.uniform(opa_lo, opa_hi, 3 * n_faces).astype(np.float32)
    return pos, col, opa


def trajectory_poses(seed: int, n: int, radius: float = 1.5, height: float = 1.5) -> np.ndarray:
    """``n`` poses on a circle around the room centre, each looking across the room at a jittered point."""
    rng = np.random.default_rng(seed)
    out = np.empty((n, 12), np.float32)
    for i in range(n):
        th = 2 * np.pi * i / max(n, 1) + rng.uniform(-0.1, 0.1)
        eye = np.array([radius * np.cos(th), radius * np.sin(th), height])
        target = np.array([-2.4 * np.cos(th), -2.0 * np.sin(th), rng.uniform(0.6, 2.2)])
        target[:2] += rng.normal(0, 0.3, 2)
        out[i] = look_at(eye, target)
    return out


def room_scene(seed: int, n_faces: int, n_views: int, W: int, H: int, f: float,
               target_seed: Optional[int] = None) -> Scene:
    """Room map seen by ``n_views`` cameras of one resolution on a seeded trajectory."""
    pos, col, opa = room_map(seed, n_faces)
    cams = _cams(n_views, W, H, f, f, W / 2.0, H / 2.0)
    poses = trajectory_poses(seed + 1000, n_views)
    sc = Scene(pos, col, opa, None, cams, poses)
    if target_seed is not None:
        sc.tgt_color, sc.tgt_depth = noise_targets(target_seed, cams)
    return sc


def mixed_keyframe_cameras(per_res: int = 4) -> np.ndarray:
    """Keyframes of uneven resolution: 320x240 (f=262.5), 640x480 (f=525), 1200x680 (f=600)."""
    rows = []
    for (W, H, f) in ((320, 240, 262.5), (640, 480, 525.0), (1200, 680, 600.0)):
        rows.append(_cams(per_res, W, H, f, f, W / 2.0, H / 2.0))
    return np.concatenate(rows)


def tiny_scene(seed: int, n_faces: int = 6, W: int = 16, H: int = 16, f: float = 20.0,
               opa_lo: float = 0.3, opa_hi: float = 0.9, indexed: bool = False) -> Scene:
    """A handful of large triangles in front of a small camera (finite-difference tests)."""
    rng = np.random.default_rng(seed)
    sc = random_triangles_scene(seed, n_faces, W, H, f, z_lo=1.0, z_hi=3.0,
                                side_lo=0.5, side_hi=1.5, opa_lo=opa_lo, opa_hi=opa_hi,
                                target_seed=seed + 7)
    if indexed:
        # share vertices between consecutive faces: face m = (m, m+1, m+2) over a strip
        n_vert = n_faces + 2
        sc.pos = sc.pos[:n_vert].copy()
        sc.col = sc.col[:n_vert].copy()
        sc.opa = sc.opa[:n_vert].copy()
        sc.faces = np.stack([np.arange(n_faces), np.arange(n_faces) + 1, np.arange(n_faces) + 2], 1).astype(np.int32)
    del rng
    return sc


def perturb_pose(pose: np.ndarray, rng: np.random.Generator, trans: float = 0.05, rot_deg: float = 3.0) -> np.ndarray:
    """Left-multiply T_CW by a random rigid motion: translation ~U(+-trans) per axis,
    rotation ~U(+-rot_deg) about a uniform random axis (Rodrigues' formula)."""
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    ang = np.deg2rad(rng.uniform(-rot_deg, rot_deg))
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    Rd = np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * (K @ K)
    td = rng.uniform(-trans, trans, 3)
    R = pose[:9].astype(np.float64).reshape(3, 3)
    t = pose[9:].astype(np.float64)
    return np.concatenate([(Rd @ R).reshape(-1), Rd @ t + td]).astype(np.float32)


def request_stream(seed: int, rate: float, duration: float,
                   resolutions=((256, 256, 256.0), (640, 480, 525.0), (1200, 680, 600.0)),
                   n_poses: int = 64, track_fraction: float = 0.5):
    """Poisson arrivals: list of dicts {t, kind ('render'|'track'), W, H, f, pose_index}."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        W, H, f = resolutions[rng.integers(len(resolutions))]
        out.append(dict(t=t, kind='track' if rng.random() < track_fraction else 'render',
                        W=int(W), H=int(H), f=float(f), pose_index=int(rng.integers(n_poses))))
    return out
