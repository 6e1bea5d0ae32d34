"""Tracking through the pose gradient (Sec. 3.3, Eq. 5-10) on the GPU.

* the device Adam + Exp(-step) o T update against numpy Adam and scipy's matrix exponential;
* many hypotheses tracked by replaying a captured CUDA graph converge toward the true pose on a
  target rendered by the oracle, and the graph replay equals eager execution;
* the autograd pose gradient (RenderFunction with tau) against the oracle and against central
  finite differences of the GPU forward pass.
"""
import numpy as np
import pytest

from harness import assert_pose_grad, params_pair
from oracle_pins import twist_expm
from ts_synth.scenes import Scene, perturb_pose, room_map, trajectory_poses

pytestmark = pytest.mark.gpu


def _adam_reference(pose, g, state, lr_rho, lr_theta, b1=0.9, b2=0.999, eps=1e-8):
    m, v, t = state[:6].copy(), state[6:12].copy(), state[12] + 1
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    lr = np.array([lr_rho] * 3 + [lr_theta] * 3)
    step = lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    T = np.eye(4)
    T[:3, :3] = pose[:9].reshape(3, 3)
    T[:3, 3] = pose[9:]
    T2 = twist_expm(-step) @ T
    return np.concatenate([T2[:3, :3].reshape(-1), T2[:3, 3]]), np.concatenate([m, v, [t]])


def test_pose_adam_matches_reference():
    import torch
    import paper_2605_31419_gb300 as ts
    rng = np.random.default_rng(0)
    V = 5
    plan = ts.ts_plan_init(np.tile([[100.0, 100.0, 50, 40, 100, 80]], (V, 1)), 1, ts.ts_default_params())
    poses = trajectory_poses(7, V).astype(np.float64)
    state = np.zeros((V, 13))
    P = torch.tensor(poses, dtype=torch.float32, device="cuda")
    S = torch.zeros(V, 13, device="cuda")
    for it in range(3):
        g = rng.normal(size=(V, 6))
        ts.ts_pose_adam(plan, P, torch.tensor(g, dtype=torch.float32, device="cuda"), S, 0.001, 0.003)
        for v in range(V):
            poses[v], state[v] = _adam_reference(poses[v], g[v], state[v], 0.001, 0.003)
    torch.cuda.synchronize()
    assert np.allclose(P.cpu().numpy(), poses, atol=2e-6)
    assert np.allclose(S.cpu().numpy(), state, rtol=1e-5, atol=1e-7)


def _tracking_scene(n_faces=60000, W=160, H=120, f=131.25):
    # faces large enough to cover the room's surfaces, so the photometric signal is a continuous
    # image rather than a speckle of isolated triangles
    pos, col, opa = room_map(3, n_faces, side_lo=0.05, side_hi=0.12, opa_lo=0.8)
    cams = np.array([[f, f, W / 2, H / 2, W, H]])
    gt = trajectory_poses(1003, 3)[1]
    return Scene(pos, col, opa, None, cams, gt[None, :])


@pytest.mark.parametrize("lambda_ssim", [0.2, 0.0])
def test_tracking_converges_with_graph_replay(oracle, lambda_ssim):
    import torch
    import paper_2605_31419_gb300 as ts
    from oracle.oracle import SceneArrays
    sc = _tracking_scene()
    p, po = params_pair()
    f = oracle.forward(SceneArrays.of(sc), po)  # target rendered by the oracle at the true pose
    W, H = 160, 120
    rng = np.random.default_rng(5)
    tc = (f["color"].reshape(3, H, W) + rng.normal(0, 0.02, (3, H, W))).astype(np.float32)
    td = (f["depth"].reshape(H, W) * (1 + 0.01 * rng.normal(size=(H, W)))).astype(np.float32)
    gt = sc.poses[0]
    init = np.stack([perturb_pose(gt, rng, trans=0.03, rot_deg=1.5) for _ in range(8)])
    m = ts.Map.from_numpy(sc.pos, sc.col, sc.opa)
    trk = ts.Tracker(m, sc.cams[0], tc, td, init, p, lambda_ssim=lambda_ssim)
    trk.run(100, use_graph=True)
    torch.cuda.synchronize()
    err0 = ts.pose_error(init, np.tile(gt, (8, 1)))
    err1 = ts.pose_error(trk.poses.cpu().numpy(), np.tile(gt, (8, 1)))
    assert np.median(err1[:, 0]) < 0.5 * np.median(err0[:, 0]), (err0, err1)
    assert np.median(err1[:, 1]) < 0.5 * np.median(err0[:, 1]), (err0, err1)
    # a graph replay computes what eager execution computes: the same (deterministic) loss and the
    # same pose gradient up to the order of its atomic sums.  (Poses are not compared: Adam's
    # first steps are +-lr per component, so a near-zero gradient component whose last bits
    # differ between two runs can flip its step.)
    a = ts.Tracker(m, sc.cams[0], tc, td, init, p, lambda_ssim=lambda_ssim)
    a.run(1, use_graph=True)
    b = ts.Tracker(m, sc.cams[0], tc, td, init, p, lambda_ssim=lambda_ssim)
    b.run(1, use_graph=False)
    torch.cuda.synchronize()
    assert np.array_equal(a.loss().cpu().numpy(), b.loss().cpu().numpy())
    ga, gb = a.rast.dtau.cpu().numpy(), b.rast.dtau.cpu().numpy()
    assert np.allclose(ga, gb, rtol=1e-4, atol=1e-6 * np.abs(gb).max())


def _crop_scene():
    # a 32 x 24 camera on 40 faces at well-separated depths: finite differences of the composite
    # need faces whose depth order does not swap under the step (dense maps have overlapping faces
    # at nearly equal depth, where the order -- and so the image -- jumps)
    from ts_synth.scenes import random_triangles_scene
    sc = random_triangles_scene(seed=12, n_faces=40, W=32, H=24, f=30.0, z_lo=1.0, z_hi=3.0, side_lo=0.3,
                                side_hi=0.8, opa_lo=0.3, opa_hi=0.8, target_seed=None)
    return sc  # identity pose


def test_autograd_pose_gradient_vs_oracle_and_fd(oracle):
    import torch
    import paper_2605_31419_gb300 as ts
    from oracle.oracle import SceneArrays
    # sigma = 1 keeps the window's derivative bounded at the edges, so central differences of the
    # FP32 forward can follow it; sigma = 0.5 is checked against the oracle in the parity tests
    sc = _crop_scene()
    p, po = params_pair(alpha_min=0.0, T_min=0.0, sigma=1.0)
    rng = np.random.default_rng(2)
    P = 32 * 24
    wC, wD = rng.normal(size=3 * P), rng.normal(size=P)
    rast = ts.Rasterizer(sc.cams, sc.n_faces, p)
    m = ts.Map.from_numpy(sc.pos, sc.col, sc.opa)
    poses = ts.poses_tensor(sc.poses)
    tau = torch.zeros(1, 6, device="cuda", requires_grad=True)
    C, D, A = ts.render(rast, m, poses, tau)
    J = (C.double() * torch.as_tensor(wC, device="cuda")).sum() + (D.double() * torch.as_tensor(wD, device="cuda")).sum()
    J.backward()
    g = tau.grad.cpu().numpy()[0].astype(np.float64)
    r = oracle.backward(SceneArrays.of(sc), po, wC, wD, None)
    assert_pose_grad(g, r["dtau"][0], r["dtau_abs"][0])

    def J_at(pose):
        C, D, _ = rast.forward(m, ts.poses_tensor(pose[None, :]))
        return float((C.double().cpu().numpy() * wC).sum() + (D.double().cpu().numpy() * wD).sum())

    T0 = np.eye(4)
    T0[:3, :3] = sc.poses[0][:9].reshape(3, 3)
    T0[:3, 3] = sc.poses[0][9:]
    # the composite is strongly curved at the scale of 1e-3 rad (faces slide over pixels): the
    # oracle's own differences agree with its adjoint at 1e-5 and not at 1e-3
    h = 1e-5
    fd = np.zeros(6)
    for k in range(6):
        vals = []
        for s in (1, -1):
            e = np.zeros(6)
            e[k] = s * h
            T = twist_expm(e) @ T0
            vals.append(J_at(np.concatenate([T[:3, :3].reshape(-1), T[:3, 3]]).astype(np.float32)))
        fd[k] = (vals[0] - vals[1]) / (2 * h)
    assert np.allclose(g, fd, rtol=0.05, atol=0.05 * np.abs(fd).max()), (g, fd)
