"""Pins of the CPU oracle: checks against what the paper and the mathematics fix.

Every function takes an ``Oracle`` handle and raises ``AssertionError`` when the
oracle disagrees with a closed form, a brute-force computation, a library
routine or finite differences.  ``test_oracle_pins.py`` runs them on the real
oracle; ``test_oracle_mutants.py`` runs them on builds with a planted mistake
and requires each mistake to fail at least one of them.
"""
from __future__ import annotations

import json
import os
from fractions import Fraction

import numpy as np
import scipy.linalg

from oracle.oracle import Oracle, Params, SceneArrays
from ts_synth.scenes import Scene, random_triangles_scene, tiny_scene

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _single_face_scene(verts, cols, opas, cam=(1.0, 1.0, 0.0, 0.0, 32, 32), pose=None):
    pos = np.asarray(verts, np.float32).reshape(-1, 3)
    col = np.asarray(cols, np.float32).reshape(-1, 3)
    opa = np.asarray(opas, np.float32).reshape(-1)
    cams = np.asarray([cam], np.float64)
    poses = np.asarray([pose if pose is not None else [1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0]], np.float32)
    return Scene(pos, col, opa, None, cams, poses)


def _bary_solve(tri, px, py):
    """Barycentric coordinates by solving the 3x3 affine system (numpy)."""
    A = np.array([[tri[0], tri[2], tri[4]], [tri[1], tri[3], tri[5]], [1.0, 1.0, 1.0]])
    return np.linalg.solve(A, np.array([px, py, 1.0]))


def _dist_edges(tri, px, py):
    """Signed distances (positive inside) from p to the three edge lines of a 2D triangle."""
    P = np.asarray(tri, np.float64).reshape(3, 2)
    area2 = (P[1, 0] - P[0, 0]) * (P[2, 1] - P[0, 1]) - (P[2, 0] - P[0, 0]) * (P[1, 1] - P[0, 1])
    out = []
    for i in range(3):
        a, b = P[i], P[(i + 1) % 3]
        e = b - a
        cross = e[0] * (py - a[1]) - e[1] * (px - a[0])
        out.append(np.sign(area2) * cross / np.hypot(*e))
    return np.array(out)


# ---------------------------------------------------------------------------------------------
# Eq. 3 window: golden closed form on the 3-4-5 triangle
# ---------------------------------------------------------------------------------------------
def pin_window_closed_form(o: Oracle):
    g = _golden("window_345.json")
    tri = g["triangle"]
    for sigma in g["sigmas"]:
        for case in g["cases"]:
            px, py = case["p"]
            expect = max(case["d_min"], 0.0) ** sigma if case["d_min"] > 0 else 0.0
            for t in (tri, [tri[0], tri[1], tri[4], tri[5], tri[2], tri[3]]):  # both windings
                I, _ = o.window(t, sigma, px, py)
                assert abs(I - expect) < 1e-12, (sigma, case, I, expect)
    # random triangles: window = (nearest-edge distance / inradius)^sigma inside, 0 outside,
    # exactly 1 at the incentre
    rng = np.random.default_rng(11)
    for _ in range(50):
        tri = rng.uniform(-5, 5, 6)
        P = tri.reshape(3, 2)
        lens = np.array([np.hypot(*(P[(i + 1) % 3] - P[i])) for i in range(3)])
        area = 0.5 * abs((P[1, 0] - P[0, 0]) * (P[2, 1] - P[0, 1]) - (P[2, 0] - P[0, 0]) * (P[1, 1] - P[0, 1]))
        if area < 0.5:
            continue
        r = 2 * area / lens.sum()
        s = (lens[1] * P[0] + lens[2] * P[1] + lens[0] * P[2]) / lens.sum()
        I, _ = o.window(tri, 0.5, *s)
        assert abs(I - 1.0) < 1e-9, I
        for _ in range(10):
            p = rng.uniform(-6, 6, 2)
            d = _dist_edges(tri, *p)
            expect = (d.min() / r) ** 0.5 if d.min() > 0 else 0.0
            I, _ = o.window(tri, 0.5, *p)
            assert abs(I - expect) < 1e-9, (I, expect)


# ---------------------------------------------------------------------------------------------
# Sec. 3.1 barycentric interpolation: partition of unity, vertex values, numpy solve
# ---------------------------------------------------------------------------------------------
def pin_barycentric(o: Oracle):
    rng = np.random.default_rng(12)
    for _ in range(40):
        tri = rng.uniform(-5, 5, 6)
        for _ in range(5):
            p = rng.uniform(-5, 5, 2)
            _, lam = o.window(tri, 0.5, *p)
            ref = _bary_solve(tri, *p)
            assert np.allclose(lam, ref, atol=1e-9), (lam, ref)
            assert abs(lam.sum() - 1) < 1e-9
        for k in range(3):
            _, lam = o.window(tri, 0.5, tri[2 * k], tri[2 * k + 1])
            assert np.allclose(lam, np.eye(3)[k], atol=1e-9)


# ---------------------------------------------------------------------------------------------
# Eq. 1 projection: special points of a pinhole under a non-symmetric rotation; culling
# ---------------------------------------------------------------------------------------------
def pin_projection(o: Oracle):
    # R = rotation of +90 deg about z (row-major), t = (0, 0, 2): (x, y, z) -> (-y, x, z + 2)
    pose = [0, -1, 0, 1, 0, 0, 0, 0, 1, 0, 0, 2]
    fx, fy, cx, cy = 100.0, 80.0, 50.0, 40.0
    verts = [[0, 0, 1], [1, 0, 0], [0, 1, 2]]
    # camera points: (0, 0, 3), (0, 1, 2), (-1, 0, 4)
    sc = _single_face_scene(verts, [[0.5] * 3] * 3, [1, 1, 1], cam=(fx, fy, cx, cy, 100, 80), pose=pose)
    pr = o.project(SceneArrays.of(sc), Params(r_min=0.0))
    uvz = pr["uvz"][0]
    expect_u = [cx, cx, cx - fx / 4]
    expect_v = [cy, cy + fy / 2, cy]
    expect_z = [3, 2, 4]
    assert np.allclose(uvz[0:3], expect_u) and np.allclose(uvz[3:6], expect_v) and np.allclose(uvz[6:9], expect_z), uvz
    # a vertex behind the near plane culls the face; so does a face outside the image
    behind = _single_face_scene([[0, 0, 1], [1, 0, 1], [0, 1, -0.5]], [[0.5] * 3] * 3, [1, 1, 1], cam=(10, 10, 16, 16, 32, 32))
    assert o.project(SceneArrays.of(behind), Params())["count"][0] == 0
    off = _single_face_scene([[5, 5, 1], [6, 5, 1], [5, 6, 1]], [[0.5] * 3] * 3, [1, 1, 1], cam=(10, 10, 16, 16, 32, 32))
    assert o.project(SceneArrays.of(off), Params())["count"][0] == 0


# ---------------------------------------------------------------------------------------------
# Eq. 4 single triangle: C = alpha c(p) + (1 - alpha) bg, D = alpha z(p), A = alpha
# ---------------------------------------------------------------------------------------------
def pin_single_triangle(o: Oracle):
    bg = (0.1, 0.2, 0.3)
    cols = [[0.9, 0.1, 0.2], [0.2, 0.8, 0.3], [0.1, 0.3, 0.7]]
    opas = [0.2, 0.5, 0.8]
    # tilted triangle: vertex depths differ, camera 40x32 with f = 20
    verts = [[-0.6, -0.5, 1.5], [0.8, -0.3, 2.5], [-0.1, 0.7, 2.0]]
    sc = _single_face_scene(verts, cols, opas, cam=(20.0, 20.0, 20.0, 16.0, 40, 32))
    for sigma in (0.5, 1.0):
        prm = Params(sigma=sigma, bg=bg, alpha_min=0.0)
        sa = SceneArrays.of(sc)
        pr = o.project(sa, prm)
        uvz = pr["uvz"][0]
        tri = [uvz[0], uvz[3], uvz[1], uvz[4], uvz[2], uvz[5]]
        zs = uvz[6:9]
        P = tri
        lens = [np.hypot(P[2 * ((i + 1) % 3)] - P[2 * i], P[2 * ((i + 1) % 3) + 1] - P[2 * i + 1]) for i in range(3)]
        area = 0.5 * abs((P[2] - P[0]) * (P[5] - P[1]) - (P[4] - P[0]) * (P[3] - P[1]))
        r = 2 * area / sum(lens)
        oF = float(sa.opa.sum()) / 3.0
        colv = sa.col  # float32 vertex colours as the oracle sees them
        f = o.forward(sa, prm)
        W, H = 40, 32
        HW = W * H
        n_in = 0
        for y in range(H):
            for x in range(W):
                px, py = x + 0.5, y + 0.5
                d = _dist_edges(tri, px, py)
                i = y * W + x
                if d.min() > 0:
                    I = (d.min() / r) ** sigma
                    a = min(0.99, oF * I)
                    lam = _bary_solve(tri, px, py)
                    c = lam @ colv
                    z = lam @ zs
                    n_in += 1
                else:
                    a, c, z = 0.0, np.zeros(3), 0.0
                for ch in range(3):
                    assert abs(f["color"][ch * HW + i] - (a * c[ch] + (1 - a) * bg[ch])) < 1e-9, (x, y, ch)
                assert abs(f["depth"][i] - a * z) < 1e-9, (x, y)
                assert abs(f["alpha"][i] - a) < 1e-9
                assert abs(f["T_final"][i] - (1 - a)) < 1e-9
        assert n_in > 50


# ---------------------------------------------------------------------------------------------
# Coverage of one opaque triangle equals an exact point-in-triangle test at pixel centres
# ---------------------------------------------------------------------------------------------
def pin_coverage_bruteforce(o: Oracle):
    rng = np.random.default_rng(13)
    for trial in range(6):
        verts = np.c_[rng.uniform(-0.8, 0.8, (3, 2)), np.full(3, 1.0)] * rng.uniform(1, 3)
        sc = _single_face_scene(verts, [[1, 1, 1]] * 3, [1, 1, 1], cam=(12.0, 12.0, 12.0, 12.0, 24, 24))
        sa = SceneArrays.of(sc)
        prm = Params(alpha_min=0.0)
        uvz = o.project(sa, prm)["uvz"][0]
        if np.isnan(uvz[0]):
            continue
        q = [(Fraction(float(uvz[k])), Fraction(float(uvz[3 + k]))) for k in range(3)]
        f = o.forward(sa, prm)

        def orient(a, b, p):
            return (b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0])

        for y in range(24):
            for x in range(24):
                p = (Fraction(2 * x + 1, 2), Fraction(2 * y + 1, 2))
                s = [orient(q[i], q[(i + 1) % 3], p) for i in range(3)]
                inside = all(v > 0 for v in s) or all(v < 0 for v in s)
                covered = f["alpha"][y * 24 + x] > 0
                assert inside == covered, (trial, x, y, s)


# ---------------------------------------------------------------------------------------------
# A fronto-parallel triangle renders its plane depth: D / A = z
# ---------------------------------------------------------------------------------------------
def pin_fronto_parallel_depth(o: Oracle):
    for z0 in (0.7, 1.9, 3.3):
        verts = [[-0.5 * z0, -0.4 * z0, z0], [0.6 * z0, -0.2 * z0, z0], [0.0, 0.6 * z0, z0]]
        sc = _single_face_scene(verts, [[0.3, 0.6, 0.9]] * 3, [0.6, 0.7, 0.8], cam=(20.0, 20.0, 16.0, 16.0, 32, 32))
        f = o.forward(SceneArrays.of(sc), Params())
        m = f["alpha"] > 0
        assert m.sum() > 50
        assert np.allclose(f["depth"][m] / f["alpha"][m], float(np.float32(z0)), rtol=1e-12, atol=0)


# ---------------------------------------------------------------------------------------------
# Transmittance: T_n = prod_{k<n} (1 - alpha_k), T_final = prod (1 - alpha), A = 1 - T_final
# ---------------------------------------------------------------------------------------------
def pin_transmittance_product(o: Oracle):
    sc = random_triangles_scene(seed=5, n_faces=400, W=48, H=40, f=45.0, side_lo=0.1, side_hi=0.4)
    sa = SceneArrays.of(sc)
    prm = Params()
    f = o.forward(sa, prm)
    rng = np.random.default_rng(3)
    multi = 0
    for _ in range(60):
        x, y = int(rng.integers(48)), int(rng.integers(40))
        tr = o.pixel_trace(sa, prm, 0, x, y)
        a = tr["alpha"]
        prefix = np.concatenate([[1.0], np.cumprod(1 - a)])
        assert np.allclose(tr["T_before"], prefix[:-1], rtol=1e-12)
        assert abs(tr["T_final"] - prefix[-1]) < 1e-12
        i = y * 48 + x
        assert abs(f["T_final"][i] - prefix[-1]) < 1e-12
        assert abs(f["alpha"][i] - (1 - prefix[-1])) < 1e-12
        multi += len(a) >= 2
    assert multi >= 5


# ---------------------------------------------------------------------------------------------
# Termination and depth order on a stack of identical-footprint faces (closed form)
# ---------------------------------------------------------------------------------------------
def pin_termination_stack(o: Oracle):
    # 2D triangle (10,10), (20,10), (10,17.5): a 3-4-5 triangle scaled by 2.5, incentre (12.5, 12.5)
    # = centre of pixel (12, 12), where I = 1.  Copies at depths 8, 4, 2, 1, 0.5, 16 (world
    # coordinates scaled by depth, so every copy projects to the same 2D triangle with f = 1, c = 0).
    depths = [8.0, 4.0, 2.0, 1.0, 0.5, 16.0, 0.25]
    tri2 = [(10.0, 10.0), (20.0, 10.0), (10.0, 17.5)]
    verts = [[u * z, v * z, z] for z in depths for (u, v) in tri2]
    cols = [[0.25 * (1 + k % 3), 0.5, 0.125 * k] for k in range(len(depths)) for _ in range(3)]
    sc = _single_face_scene(verts, cols, [0.8] * (3 * len(depths)), cam=(1.0, 1.0, 0.0, 0.0, 32, 32))
    sa = SceneArrays.of(sc)
    prm = Params()
    tr = o.pixel_trace(sa, prm, 0, 12, 12)
    order = np.argsort(depths)
    # alpha = 0.8 per face; T: 1, .2, .04, .008, .0016, .00032; the 6th would give 6.4e-5 < T_min
    assert list(tr["faces"]) == list(order[:5]), (tr["faces"], order)
    a = float(np.float32(0.8))  # the vertex opacity as stored (float32); I = 1 at the incentre
    assert np.allclose(tr["alpha"], a, atol=1e-12)
    assert abs(tr["T_final"] - (1 - a) ** 5) < 1e-12
    f = o.forward(sa, prm)
    i = 12 * 32 + 12
    assert f["n_last"][i] == 5
    w = a * (1 - a) ** np.arange(5)
    d = np.asarray(depths)[order[:5]]
    assert abs(f["depth"][i] - (w * d).sum()) < 1e-12
    c = sa.col[3 * order[:5]]
    assert np.allclose(f["color"][[i, 1024 + i, 2048 + i]], (w[:, None] * c).sum(0), atol=1e-12)


# ---------------------------------------------------------------------------------------------
# The alpha_max clamp of the compositing (alpha = min(alpha_max, o_F I)): an opaque face at its
# incentre, where I = 1, has alpha = alpha_max exactly and passes no gradient through alpha
# ---------------------------------------------------------------------------------------------
_TRI_345 = [(10.0, 10.0), (20.0, 10.0), (10.0, 17.5)]  # 3-4-5 triangle x 2.5; incentre (12.5, 12.5)


def pin_alpha_max_clamp(o: Oracle):
    z = 2.0
    verts = [[u * z, v * z, z] for (u, v) in _TRI_345]  # fronto-parallel: projects to _TRI_345 (f = 1, c = 0)
    cols = [[0.9, 0.1, 0.2], [0.2, 0.8, 0.3], [0.1, 0.3, 0.7]]
    bg = (0.1, 0.2, 0.3)
    sc = _single_face_scene(verts, cols, [1.0, 1.0, 1.0], cam=(1.0, 1.0, 0.0, 0.0, 32, 32))
    sa = SceneArrays.of(sc)
    i = 12 * 32 + 12  # pixel (12, 12) samples the incentre
    tri = [c for q in _TRI_345 for c in q]
    cp = _bary_solve(tri, 12.5, 12.5) @ sa.col  # vertex colours as stored (float32)
    for T_min in (1e-4, 0.0):
        prm = Params(bg=bg, T_min=T_min)
        f = o.forward(sa, prm)
        assert abs(f["alpha"][i] - 0.99) < 1e-12, f["alpha"][i]
        assert abs(f["T_final"][i] - 0.01) < 1e-12, f["T_final"][i]
        assert abs(f["depth"][i] - 0.99 * z) < 1e-12
        for ch in range(3):
            assert abs(f["color"][ch * 1024 + i] - (0.99 * cp[ch] + 0.01 * bg[ch])) < 1e-12, ch
        assert o.pixel_trace(sa, prm, 0, 12, 12)["alpha"].tolist() == [0.99]
        # a loss on the clamped pixel alone: alpha is constant there, so the opacities get nothing
        # while the colours get alpha * lambda_k per channel
        dC = np.zeros(3 * 1024)
        dC[i] = 1.0
        g = o.backward(sa, prm, dC)
        assert np.all(g["dopa"] == 0.0), g["dopa"]
        lam = _bary_solve(tri, 12.5, 12.5)
        assert np.allclose(g["dcol"][:, 0], 0.99 * lam, atol=1e-12), g["dcol"]


# ---------------------------------------------------------------------------------------------
# Termination: the walk STOPS before the face that would take T below T_min; a later face that
# would keep T above T_min is not blended either
# ---------------------------------------------------------------------------------------------
def pin_stop_at_tmin(o: Oracle):
    # six faces of opacity 0.8 at depths 1..6 (the sixth would take T = 0.2^6 = 6.4e-5 below 1e-4),
    # then a face of opacity 0.01 at depth 7 (T 0.2^5 * 0.99 = 3.2e-4 would stay above T_min)
    depths = [1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 7.0]
    opas = [0.8] * 6 + [0.01]
    verts = [[u * z, v * z, z] for z in depths for (u, v) in _TRI_345]
    cols = [[0.1 * k, 0.5, 1.0 - 0.1 * k] for k in range(len(depths)) for _ in range(3)]
    sc = _single_face_scene(verts, cols, [o_ for o_ in opas for _ in range(3)], cam=(1.0, 1.0, 0.0, 0.0, 32, 32))
    sa = SceneArrays.of(sc)
    prm = Params()
    tr = o.pixel_trace(sa, prm, 0, 12, 12)
    assert list(tr["faces"]) == [0, 1, 2, 3, 4], tr["faces"]
    a = float(np.float32(0.8))
    assert abs(tr["T_final"] - (1 - a) ** 5) < 1e-15
    f = o.forward(sa, prm)
    i = 12 * 32 + 12
    assert f["n_last"][i] == 5, f["n_last"][i]
    assert abs(f["T_final"][i] - (1 - a) ** 5) < 1e-15
    w = a * (1 - a) ** np.arange(5)
    assert abs(f["depth"][i] - (w * np.asarray(depths[:5])).sum()) < 1e-12
    # with T_min = 0 every face blends, the last one included
    tr0 = o.pixel_trace(sa, Params(T_min=0.0), 0, 12, 12)
    assert list(tr0["faces"]) == list(range(7)), tr0["faces"]


# ---------------------------------------------------------------------------------------------
# Binning: per-tile depth-sorted lists by brute force over tiles x faces
# ---------------------------------------------------------------------------------------------
def pin_binning_bruteforce(o: Oracle):
    sc = random_triangles_scene(seed=6, n_faces=300, W=72, H=40, f=60.0)
    for tw, th in ((16, 16), (8, 4), (32, 8)):
        prm = Params(tile_w=tw, tile_h=th)
        sa = SceneArrays.of(sc)
        pr = o.project(sa, prm)
        b = o.bin(sa, prm)
        W, H = 72, 40
        TX, TY = -(-W // tw), -(-H // th)
        assert b["n_tiles"] == TX * TY
        pix = pr["pix"]
        zb = pr["zbits"]
        uvz = pr["uvz"]
        for m in range(sc.n_faces):
            if pr["count"][m] == 0:
                continue
            u, v = uvz[m, 0:3].astype(np.float32), uvz[m, 3:6].astype(np.float32)
            x0 = max(0, int(np.ceil(np.float32(u.min()) - np.float32(0.5))))
            x1 = min(W - 1, int(np.floor(np.float32(u.max()) - np.float32(0.5))))
            y0 = max(0, int(np.ceil(np.float32(v.min()) - np.float32(0.5))))
            y1 = min(H - 1, int(np.floor(np.float32(v.max()) - np.float32(0.5))))
            assert list(pix[m]) == [x0, y0, x1, y1]
            zk = np.float32(np.float32(np.float32(uvz[m, 6]) + np.float32(uvz[m, 7])) + np.float32(uvz[m, 8])) / np.float32(3)
            assert np.float32(zk).view(np.uint32) == zb[m]
        for ty in range(TY):
            for tx in range(TX):
                t = ty * TX + tx
                want = []
                for m in range(sc.n_faces):
                    if pr["count"][m] == 0:
                        continue
                    x0, y0, x1, y1 = pix[m]
                    if x0 <= tx * tw + tw - 1 and x1 >= tx * tw and y0 <= ty * th + th - 1 and y1 >= ty * th:
                        want.append((int(zb[m]), m))
                want.sort()
                s, e = b["ranges"][t]
                got = list(b["ids"][s:e]) if e > s else []
                assert got == [m for _, m in want], (tw, th, tx, ty)
                for k in range(s, e):
                    assert int(b["keys"][k]) >> 32 == t


def pin_sort_ties(o: Oracle):
    verts = [[-0.5, -0.5, 2.0], [0.5, -0.4, 2.0], [0.0, 0.5, 2.0]] * 3
    sc = _single_face_scene(verts, [[0.5] * 3] * 9, [0.5] * 9, cam=(20.0, 20.0, 16.0, 16.0, 32, 32))
    b = o.bin(SceneArrays.of(sc), Params())
    for t in range(b["n_tiles"]):
        s, e = b["ranges"][t]
        if e > s:
            assert list(b["ids"][s:e]) == [0, 1, 2]


# ---------------------------------------------------------------------------------------------
# Loss (R11): mean L1 colour + lambda_dep * masked mean L1 depth; gradient signs
# ---------------------------------------------------------------------------------------------
def pin_l1_loss(o: Oracle):
    sc = random_triangles_scene(seed=7, n_faces=10, W=12, H=10, f=10.0)
    sa = SceneArrays.of(sc)
    rng = np.random.default_rng(1)
    C = rng.random(3 * 120)
    D = rng.random(120) * 3
    tC = rng.random(3 * 120)
    tD = rng.random(120) * 3
    tD[::7] = 0.0
    r = o.l1_loss(sa, C, D, tC, tD, 0.05)
    valid = tD > 0
    expect = np.abs(C - tC).mean() + 0.05 * np.abs(D - tD)[valid].sum() / 120
    assert abs(r["loss"] - expect) < 1e-12
    assert np.allclose(r["dC"], np.sign(C - tC) / 360)
    assert np.allclose(r["dD"], 0.05 * np.sign(D - tD) * valid / 120)


# ---------------------------------------------------------------------------------------------
# D-SSIM (Eq. 8, R15-R17): scipy's Gaussian filter, closed forms, finite differences
# ---------------------------------------------------------------------------------------------
SSIM_C1, SSIM_C2 = 0.01 ** 2, 0.03 ** 2


def _loss_cams(sizes):
    """SceneArrays carrying only cameras of the given (W, H) sizes (the loss needs no faces)."""
    sc = random_triangles_scene(seed=3, n_faces=4, W=sizes[0][0], H=sizes[0][1], f=10.0)
    cams = np.asarray([[10.0, 10.0, W / 2, H / 2, W, H] for W, H in sizes], np.float64)
    poses = np.repeat(sc.poses[:1], len(sizes), axis=0)
    return SceneArrays.of(Scene(sc.pos, sc.col, sc.opa, None, cams, poses))


def ssim_map_scipy(x, y):
    """Per-pixel SSIM of two HxW images, local statistics by scipy.ndimage.gaussian_filter
    (sigma 1.5, radius 5, zero padding)."""
    import scipy.ndimage as ndi

    g = lambda a: ndi.gaussian_filter(a, sigma=1.5, truncate=5.0 / 1.5, mode="constant", cval=0.0)  # noqa: E731
    mx, my = g(x), g(y)
    sxx, syy, sxy = g(x * x) - mx * mx, g(y * y) - my * my, g(x * y) - mx * my
    return ((2 * mx * my + SSIM_C1) * (2 * sxy + SSIM_C2)) / ((mx * mx + my * my + SSIM_C1) * (sxx + syy + SSIM_C2))


def pin_ssim_scipy(o: Oracle):
    sizes = [(23, 17), (8, 13)]
    sa = _loss_cams(sizes)
    rng = np.random.default_rng(31)
    P = sum(W * H for W, H in sizes)
    C, tC = rng.random(3 * P), rng.random(3 * P)
    tC[: 3 * 23 * 17] = np.clip(C[: 3 * 23 * 17] + 0.1 * rng.normal(size=3 * 23 * 17), 0, 1)  # correlated view
    D, tD = rng.random(P), rng.random(P)
    r = o.pho_loss(sa, C, D, tC, tD, lambda_ssim=0.2, lambda_dep=0.05, grads=False)
    off = 0
    for v, (W, H) in enumerate(sizes):
        HW = W * H
        ref = np.concatenate([ssim_map_scipy(C[3 * off + c * HW:3 * off + (c + 1) * HW].reshape(H, W),
                                             tC[3 * off + c * HW:3 * off + (c + 1) * HW].reshape(H, W)).ravel()
                              for c in range(3)])
        got = r["ssim_map"][3 * off:3 * off + 3 * HW]
        assert np.abs(got - ref).max() < 1e-12, (v, np.abs(got - ref).max())
        l1 = np.abs(C[3 * off:3 * off + 3 * HW] - tC[3 * off:3 * off + 3 * HW]).mean()
        dep = np.abs(D[off:off + HW] - tD[off:off + HW]).sum() / HW
        expect = 0.8 * l1 + 0.2 * (1 - ref.mean()) + 0.05 * dep
        assert abs(r["loss_v"][v] - expect) < 1e-12, (v, r["loss_v"][v], expect)
        off += HW


def pin_ssim_closed_forms(o: Oracle):
    # identical images: SSIM = 1 everywhere, and x = y is a stationary point (zero gradient)
    sa = _loss_cams([(19, 14)])
    rng = np.random.default_rng(32)
    C = rng.random(3 * 19 * 14)
    D = rng.random(19 * 14)
    r = o.pho_loss(sa, C, D, C.copy(), D.copy(), lambda_ssim=0.2, lambda_dep=0.05)
    assert np.abs(r["ssim_map"] - 1).max() < 1e-12
    assert abs(r["loss"]) < 1e-12
    assert np.abs(r["dC"]).max() < 1e-12
    # constant images a, b: SSIM = (2ab + C1) / (a^2 + b^2 + C1) wherever the window lies inside
    W, H = 21, 16
    sa = _loss_cams([(W, H)])
    for a, b in ((0.3, 0.7), (0.9, 0.05), (0.5, 0.5)):
        C = np.full(3 * W * H, a)
        tC = np.full(3 * W * H, b)
        r = o.pho_loss(sa, C, np.ones(W * H), tC, np.ones(W * H), grads=False)
        smap = r["ssim_map"].reshape(3, H, W)[:, 5:H - 5, 5:W - 5]
        assert np.abs(smap - (2 * a * b + SSIM_C1) / (a * a + b * b + SSIM_C1)).max() < 1e-12


def pin_pho_fd(o: Oracle):
    sizes = [(9, 7), (6, 5)]
    sa = _loss_cams(sizes)
    rng = np.random.default_rng(33)
    P = sum(W * H for W, H in sizes)
    tC = rng.random(3 * P)
    # keep |C - Cbar| >= 0.05 so that the L1 term is differentiable at every entry
    C = np.clip(tC + rng.choice([-1, 1], size=3 * P) * rng.uniform(0.05, 0.4, size=3 * P), -0.5, 1.5)
    D, tD = rng.random(P) + 1, rng.random(P) + 1
    lam = 0.35
    an = o.pho_loss(sa, C, D, tC, tD, lambda_ssim=lam, lambda_dep=0.05)
    h = 1e-6
    scale = np.abs(an["dC"]).max()
    for i in range(3 * P):
        cp, cm = C.copy(), C.copy()
        cp[i] += h
        cm[i] -= h
        fd = (o.pho_loss(sa, cp, D, tC, tD, lam, 0.05, grads=False)["loss"] -
              o.pho_loss(sa, cm, D, tC, tD, lam, 0.05, grads=False)["loss"]) / (2 * h)
        assert abs(fd - an["dC"][i]) <= 1e-7 * scale + 1e-5 * abs(fd), (i, fd, an["dC"][i])


# ---------------------------------------------------------------------------------------------
# Rendered normal map (Eq. 12, R20-R22): plane normals in camera space, winding, the loss
# ---------------------------------------------------------------------------------------------
def _rot(axis, deg):
    a = np.asarray(axis, np.float64) / np.linalg.norm(axis)
    th = np.radians(deg)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K


def pin_normal_closed_forms(o: Oracle):
    prm = Params(alpha_min=0.0)
    # fronto-parallel face at z = 2 under the identity pose: N = A (0, 0, -1) (towards the camera)
    sc = _single_face_scene([[-0.6, -0.5, 2.0], [0.7, -0.4, 2.0], [0.0, 0.6, 2.0]], [[0.5] * 3] * 3, [0.9, 0.6, 0.8],
                            cam=(20.0, 20.0, 16.0, 16.0, 32, 32))
    f = o.forward(SceneArrays.of(sc), prm)
    P = 32 * 32
    N = f["normal"].reshape(3, P)
    assert f["alpha"].max() > 0.5
    assert np.abs(N[0]).max() < 1e-12 and np.abs(N[1]).max() < 1e-12
    assert np.abs(N[2] + f["alpha"]).max() < 1e-12
    # a tilted face under a rotated, translated camera: N = A n_C, n_C = R n_W turned to the camera
    R = _rot([0.3, -1.0, 0.4], 25.0)
    t = np.array([0.1, -0.2, 2.5])
    n_w = np.array([0.2, 0.5, -1.0]) / np.linalg.norm([0.2, 0.5, -1.0])
    b1 = np.cross(n_w, [1.0, 0.0, 0.0]); b1 /= np.linalg.norm(b1)
    b2 = np.cross(n_w, b1)
    c_w = R.T @ (np.array([0.05, 0.0, 2.6]) - t)  # a point in front of the camera
    verts = [c_w + 0.8 * b1, c_w - 0.5 * b1 + 0.7 * b2, c_w - 0.4 * b1 - 0.8 * b2]
    pose = np.concatenate([R.reshape(-1), t]).astype(np.float32)
    for order in ((0, 1, 2), (0, 2, 1)):  # both windings give the same map
        sc = _single_face_scene([verts[i] for i in order], [[0.5] * 3] * 3, [0.9, 0.6, 0.8],
                                cam=(24.0, 24.0, 16.0, 16.0, 32, 32), pose=pose)
        sa = SceneArrays.of(sc)
        f = o.forward(sa, prm)
        # the plane's normal carried into the camera frame (R rounded to float32 is orthonormal to
        # ~1e-8, hence the tolerance), turned towards the camera centre
        n_c = R @ n_w
        if n_c @ (R @ c_w + t) > 0:
            n_c = -n_c
        A = f["alpha"]
        assert A.max() > 0.5
        N = f["normal"].reshape(3, P)
        assert np.abs(N - n_c[:, None] * A[None, :]).max() < 1e-7, order


def pin_normal_loss(o: Oracle):
    sizes = [(9, 7), (5, 4)]
    sa = _loss_cams(sizes)
    rng = np.random.default_rng(51)
    P = sum(W * H for W, H in sizes)
    N = rng.normal(size=3 * P)
    Nb = rng.normal(size=(3, P))
    Nb /= np.linalg.norm(Nb, axis=0)
    Nb[:, ::4] = 0.0  # no sensor normal at every fourth pixel
    Nb = Nb.reshape(-1)
    r = o.normal_loss(sa, N, Nb, weight=0.05)
    off = 0
    for v, (W, H) in enumerate(sizes):
        HW = W * H
        n = N[3 * off:3 * off + 3 * HW].reshape(3, HW)
        nb = Nb[3 * off:3 * off + 3 * HW].reshape(3, HW)
        valid = np.abs(nb).sum(0) > 0
        expect = (1 - (n * nb).sum(0))[valid].sum() / HW
        assert abs(r["loss_v"][v] - expect) < 1e-12
        assert np.allclose(r["dN"][3 * off:3 * off + 3 * HW].reshape(3, HW), -0.05 * nb * valid / HW, atol=1e-15)
        off += HW


# ---------------------------------------------------------------------------------------------
# Min-opacity variant (Mesh Splatting, R24): alpha scales by min(o) / mean(o); FD of dopa
# ---------------------------------------------------------------------------------------------
def pin_min_opacity_variant(o: Oracle):
    verts = [[-0.6, -0.5, 2.0], [0.7, -0.4, 2.3], [0.0, 0.6, 1.8]]
    opas = [0.5, 0.2, 0.35]
    sc = _single_face_scene(verts, [[0.5] * 3] * 3, opas, cam=(20.0, 20.0, 16.0, 16.0, 32, 32))
    sa = SceneArrays.of(sc)
    a_mean = o.forward(sa, Params(alpha_min=0.0))["alpha"]
    a_min = o.forward(sa, Params(alpha_min=0.0, min_opacity=True))["alpha"]
    cov = a_mean > 0
    assert cov.sum() > 20
    ratio = sa.opa.min() / sa.opa.mean()
    assert np.abs(a_min[cov] - ratio * a_mean[cov]).max() < 1e-12
    # finite differences of the opacity gradient: only the minimal vertex receives one
    sc = tiny_scene(23, n_faces=5)
    base = SceneArrays.of(sc)
    prm = Params(alpha_min=0.0, T_min=0.0, fp64=True, min_opacity=True, sigma=1.0)
    P = int(base.pix_offsets()[-1])
    rng = np.random.default_rng(123)
    wC, wD, wA = rng.normal(size=3 * P), rng.normal(size=P), rng.normal(size=P)
    an = o.backward(base, prm, wC, wD, wA)
    opa3 = base.opa.reshape(-1, 3)
    is_min = np.zeros_like(opa3, bool)
    is_min[np.arange(len(opa3)), np.argmin(opa3, axis=1)] = True
    assert np.all(an["dopa"].reshape(-1, 3)[~is_min] == 0)
    h = 1e-6
    scale = np.abs(an["dopa"]).max() + 1e-12
    for i in range(len(base.opa)):
        xp, xm = base.opa.copy(), base.opa.copy()
        xp[i] += h
        xm[i] -= h
        f = lambda x: _linear_functional(SceneArrays.of(sc, opa=x), prm, o, wC, wD, wA, np.zeros(3 * P))  # noqa
        fd = (f(xp) - f(xm)) / (2 * h)
        assert abs(fd - an["dopa"][i]) <= 2e-5 * scale + 1e-4 * abs(fd), (i, fd, an["dopa"][i])


# ---------------------------------------------------------------------------------------------
# Learnable per-face sigma (R25): reduces to the global exponent; finite differences in sigma_F
# ---------------------------------------------------------------------------------------------
def pin_face_sigma_variant(o: Oracle):
    sc = tiny_scene(24, n_faces=5)
    M = sc.n_faces
    prm = Params(alpha_min=0.0, T_min=0.0, fp64=True, sigma=0.5)
    ref = o.forward(SceneArrays.of(sc), prm)
    same = o.forward(SceneArrays.of(sc, sigma=np.full(M, 0.5)), prm)
    for k in ("color", "depth", "alpha", "normal"):
        assert np.array_equal(ref[k], same[k]), k
    sig = np.random.default_rng(25).uniform(0.6, 1.5, size=M)
    base = SceneArrays.of(sc, sigma=sig)
    P = int(base.pix_offsets()[-1])
    rng = np.random.default_rng(125)
    wC, wD, wA, wN = rng.normal(size=3 * P), rng.normal(size=P), rng.normal(size=P), rng.normal(size=3 * P)
    an = o.backward(base, prm, wC, wD, wA, wN)
    h = 1e-6

    def J(**kw):
        return _linear_functional(SceneArrays.of(sc, sigma=kw.pop("sigma", sig), **kw), prm, o, wC, wD, wA, wN)

    scale = np.abs(an["dsigma"]).max()
    assert scale > 0
    for i in range(M):
        sp, sm = sig.copy(), sig.copy()
        sp[i] += h
        sm[i] -= h
        fd = (J(sigma=sp) - J(sigma=sm)) / (2 * h)
        assert abs(fd - an["dsigma"][i]) <= 2e-5 * scale + 1e-4 * abs(fd), (i, fd, an["dsigma"][i])
    scale = np.abs(an["dpos"]).max()
    for idx in list(np.ndindex(base.pos.shape))[::4]:
        xp, xm = base.pos.copy(), base.pos.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (J(pos=xp) - J(pos=xm)) / (2 * h)
        assert abs(fd - an["dpos"][idx]) <= 2e-5 * scale + 1e-4 * abs(fd), (idx, fd, an["dpos"][idx])


# ---------------------------------------------------------------------------------------------
# Map statistics (Sec. 3.4, R23): coverage by brute force, projected area in closed form
# ---------------------------------------------------------------------------------------------
def pin_face_stats(o: Oracle):
    # one face of low opacity: its rim pixels have alpha < alpha_min and must not count
    verts = [[-0.6, -0.5, 2.0], [0.7, -0.4, 2.0], [0.0, 0.6, 2.0]]
    opas = [0.01, 0.012, 0.011]
    sc = _single_face_scene(verts, [[0.5] * 3] * 3, opas, cam=(20.0, 20.0, 16.0, 16.0, 32, 32))
    sa = SceneArrays.of(sc)
    prm = Params()
    st = o.face_stats(sa, prm)
    pr = o.project(sa, prm)
    uvz = pr["uvz"][0]
    tri = [uvz[0], uvz[3], uvz[1], uvz[4], uvz[2], uvz[5]]
    P = np.asarray(tri).reshape(3, 2)
    lens = [np.hypot(*(P[(i + 1) % 3] - P[i])) for i in range(3)]
    area2 = (P[1, 0] - P[0, 0]) * (P[2, 1] - P[0, 1]) - (P[2, 0] - P[0, 0]) * (P[1, 1] - P[0, 1])
    r = abs(area2) / sum(lens)
    oF = sa.opa.sum() / 3
    inside = counted = 0
    for y in range(32):
        for x in range(32):
            d = _dist_edges(tri, x + 0.5, y + 0.5)
            if d.min() > 0:
                inside += 1
                if min(prm.alpha_max, oF * (d.min() / r) ** prm.sigma) >= prm.alpha_min:
                    counted += 1
    assert 0 < counted < inside
    assert int(st["coverage"][0]) == counted
    # projected area: a fronto-parallel face at depth z scales its world area by (f / z)^2
    world = 0.5 * abs(np.cross(np.subtract(verts[1], verts[0]), np.subtract(verts[2], verts[0]))[2])
    assert abs(st["area"][0] - world * (20.0 / 2.0) ** 2) < 1e-4 * st["area"][0]
    # a culled face (behind the camera) has no area and no coverage
    behind = _single_face_scene([[0, 0, -1], [1, 0, -1], [0, 1, -1]], [[0.5] * 3] * 3, [1, 1, 1],
                                cam=(20.0, 20.0, 16.0, 16.0, 32, 32))
    st2 = o.face_stats(SceneArrays.of(behind), prm)
    assert st2["area"][0] == 0 and st2["coverage"][0] == 0


# ---------------------------------------------------------------------------------------------
# Equilateral regulariser (Eq. 14, R19): closed forms, invariances, finite differences
# ---------------------------------------------------------------------------------------------
def _soup(tris, seed=0):
    tris = np.asarray(tris, np.float64).reshape(-1, 3)
    n = len(tris)
    return SceneArrays.of(Scene(tris.astype(np.float32), np.full((n, 3), 0.5, np.float32), np.full(n, 0.8, np.float32),
                                None, np.array([[10.0, 10.0, 5.0, 5.0, 10, 10]]),
                                np.array([[1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0]], np.float32)), pos=tris)


def pin_equilateral_closed_forms(o: Oracle):
    s3 = np.sqrt(3.0)
    # equilateral: every cosine is 0.5
    r = o.equilateral(_soup([[0, 0, 1], [2, 0, 1], [1, s3, 1]]))
    assert abs(r["loss"]) < 1e-15 and np.abs(r["dpos"]).max() < 1e-12
    # 3-4-5 right triangle: cosines 0, 4/5, 3/5 -> (0.25 + 0.09 + 0.01) / 3 = 7/60
    assert abs(o.equilateral(_soup([[0, 0, 0], [4, 0, 0], [0, 3, 0]]))["loss"] - 7.0 / 60.0) < 1e-15
    # right isosceles: cosines 0, 1/sqrt2, 1/sqrt2
    c = 1 / np.sqrt(2.0)
    expect = (0.25 + 2 * (c - 0.5) ** 2) / 3
    assert abs(o.equilateral(_soup([[0, 0, 0], [1, 0, 0], [0, 1, 0]]))["loss"] - expect) < 1e-15
    # the mean over faces, with a degenerate face (zero-length edge) adding 0 but counting
    r = o.equilateral(_soup([[0, 0, 0], [4, 0, 0], [0, 3, 0], [1, 1, 1], [1, 1, 1], [2, 0, 0]]))
    assert abs(r["loss"] - 7.0 / 120.0) < 1e-15
    assert np.all(r["dpos"][3:] == 0)


def pin_equilateral_invariance_and_fd(o: Oracle):
    rng = np.random.default_rng(41)
    tris = rng.normal(size=(30, 3, 3))
    base = o.equilateral(_soup(tris.reshape(-1, 3)))
    # similarity transforms leave every angle unchanged
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    moved = 2.7 * tris.reshape(-1, 3) @ Q.T + np.array([0.3, -1.0, 4.0])
    assert abs(o.equilateral(_soup(moved))["loss"] - base["loss"]) < 1e-13
    # central differences of every coordinate
    flat = tris.reshape(-1, 3)
    h = 1e-6
    for idx in np.ndindex(flat.shape):
        xp, xm = flat.copy(), flat.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (o.equilateral(_soup(xp), grads=False)["loss"] - o.equilateral(_soup(xm), grads=False)["loss"]) / (2 * h)
        assert abs(fd - base["dpos"][idx]) <= 1e-8 + 1e-5 * abs(fd), (idx, fd, base["dpos"][idx])


# ---------------------------------------------------------------------------------------------
# SE(3) exponential against scipy's matrix exponential of the twist
# ---------------------------------------------------------------------------------------------
def twist_expm(tau):
    rho, th = np.asarray(tau[:3], np.float64), np.asarray(tau[3:], np.float64)
    X = np.zeros((4, 4))
    X[:3, :3] = [[0, -th[2], th[1]], [th[2], 0, -th[0]], [-th[1], th[0], 0]]
    X[:3, 3] = rho
    return scipy.linalg.expm(X)


def pin_se3_exp(o: Oracle):
    rng = np.random.default_rng(14)
    for scale in (1e-9, 1e-4, 0.3, 2.5):
        for _ in range(5):
            tau = rng.normal(size=6) * scale
            E = twist_expm(tau)
            T = o.se3_exp(tau)
            assert np.allclose(T[:9].reshape(3, 3), E[:3, :3], atol=1e-12)
            assert np.allclose(T[9:], E[:3, 3], atol=1e-12)


# ---------------------------------------------------------------------------------------------
# Adjoint vs central finite differences (FP64 mode) on tiny scenes
# ---------------------------------------------------------------------------------------------
def _linear_functional(sa, prm, o, wC, wD, wA, wN):
    f = o.forward(sa, prm)
    return float(wC @ f["color"] + wD @ f["depth"] + wA @ f["alpha"] + wN @ f["normal"])


def pin_fd_gradients(o: Oracle, seeds=(21, 22), sigmas=(1.0, 0.5)):
    for seed in seeds:
        for sigma in sigmas:
            for indexed in (False, True):
                sc = tiny_scene(seed, n_faces=5, indexed=indexed)
                base = SceneArrays.of(sc)
                prm = Params(sigma=sigma, alpha_min=0.0, T_min=0.0, fp64=True, bg=(0.2, 0.1, 0.3))
                rng = np.random.default_rng(seed + 100)
                P = int(base.pix_offsets()[-1])
                wC, wD, wA = rng.normal(size=3 * P), rng.normal(size=P), rng.normal(size=P)
                wN = rng.normal(size=3 * P)
                an = o.backward(base, prm, wC, wD, wA, wN)
                h = 1e-6

                def J(**kw):
                    return _linear_functional(SceneArrays.of(sc, **kw), prm, o, wC, wD, wA, wN)

                for name, arr, key in (("pos", base.pos, "dpos"), ("col", base.col, "dcol"), ("opa", base.opa, "dopa")):
                    g = an[key]
                    scale = np.abs(g).max() + 1e-12
                    for idx in np.ndindex(arr.shape):
                        xp, xm = arr.copy(), arr.copy()
                        xp[idx] += h
                        xm[idx] -= h
                        fd = (J(**{name: xp}) - J(**{name: xm})) / (2 * h)
                        tol = 2e-5 * scale + 1e-4 * abs(fd) + (1e-4 * scale if sigma < 1 else 0.0)
                        assert abs(fd - g[idx]) <= tol, (seed, sigma, indexed, name, idx, fd, g[idx])
                # pose: left perturbation Exp(tau) o T with the exponential from scipy
                pose = base.poses[0]
                T0 = np.eye(4)
                T0[:3, :3] = pose[:9].reshape(3, 3)
                T0[:3, 3] = pose[9:]
                scale = np.abs(an["dtau"]).max() + 1e-12
                for k in range(6):
                    vals = []
                    for s in (+1, -1):
                        tau = np.zeros(6)
                        tau[k] = s * h
                        T = twist_expm(tau) @ T0
                        p = np.concatenate([T[:3, :3].reshape(-1), T[:3, 3]])[None, :]
                        vals.append(J(poses=p))
                    fd = (vals[0] - vals[1]) / (2 * h)
                    tol = 2e-5 * scale + 1e-4 * abs(fd) + (1e-4 * scale if sigma < 1 else 0.0)
                    assert abs(fd - an["dtau"][0, k]) <= tol, (seed, sigma, "tau", k, fd, an["dtau"][0, k])


ALL_PINS = [pin_window_closed_form, pin_barycentric, pin_projection, pin_single_triangle, pin_coverage_bruteforce,
            pin_fronto_parallel_depth, pin_transmittance_product, pin_termination_stack, pin_alpha_max_clamp,
            pin_stop_at_tmin, pin_binning_bruteforce,
            pin_sort_ties, pin_l1_loss, pin_ssim_scipy, pin_ssim_closed_forms, pin_pho_fd,
            pin_normal_closed_forms, pin_normal_loss, pin_min_opacity_variant, pin_face_sigma_variant,
            pin_face_stats,
            pin_equilateral_closed_forms,
            pin_equilateral_invariance_and_fd,
            pin_se3_exp, pin_fd_gradients]
