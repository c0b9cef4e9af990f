"""Pins of the mini bundle adjustment oracle (CPU): the analytic Jacobian
against FP64 central differences, the robust cost against hand values, the
outlier rule against planted outliers, and convergence to the synthetic truth
(reprojection, and the scale-free geometry)."""
import math

import numpy as np

from oracle import mini_ba as B
from oracle import oracle as O


def test_jacobian_matches_central_differences():
    rng = np.random.default_rng(0)
    gt, obs, cx, cy, _ = B.synthetic_problem(rng, F=4, P=6)
    params = {"fl": gt["fl"] * 1.05, "R": gt["R"].copy(), "t": gt["t"] + 0.01, "X": gt["X"] * 1.1}
    Jm = B.jacobian(params, cx, cy)
    n = Jm.shape[1]
    h = 1e-6
    for j in range(n):
        d = np.zeros(n)
        d[j] = h
        rp = B.residuals(B.apply_step(params, d), obs, cx, cy).reshape(-1)
        rm = B.residuals(B.apply_step(params, -d), obs, cx, cy).reshape(-1)
        np.testing.assert_allclose(Jm[:, j], (rp - rm) / (2 * h), rtol=1e-5, atol=1e-6 * np.abs(Jm).max())


def test_robust_cost_hand_values():
    e = np.array([0.5, 2.0, 5.0, 100.0])
    mask = np.array([True, True, True, False])
    assert abs(B.robust_cost(e, mask, 2.0) - (0.125 + 2.0 + 2.0 * (5.0 - 1.0))) < 1e-12
    # lower median / MAD rule: 9 small errors and one large
    e = np.array([1.0, 1.1, 0.9, 1.2, 0.8, 1.05, 0.95, 1.15, 0.85, 40.0])
    m = B.inlier_mask(e)
    assert not m[-1] and m[:-1].all()


def test_lm_converges_from_a_perturbed_truth_and_rejects_outliers():
    """0.5 px noise and 3% gross outliers, start 1-3% off the truth: after 30
    iterations every planted outlier is excluded, the inlier reprojection RMS
    is at the noise level, and the robust cost is no higher than that of the
    true parameters on the same observations (a short forward path leaves focal
    length and depth weakly separable, so the truth is not the minimiser under
    noise)."""
    rng = np.random.default_rng(1)
    F, P = 6, 80
    gt, obs, cx, cy, out = B.synthetic_problem(rng, F=F, P=P, outlier_frac=0.03, noise_px=0.5)
    params = {"fl": gt["fl"] * 1.03, "R": gt["R"].copy(), "t": gt["t"].copy(),
              "X": gt["X"] * (1 + rng.normal(0, 0.02, gt["X"].shape))}
    for f in range(1, F):
        params["R"][f], params["t"][f] = O.retract_pose(gt["R"][f], gt["t"][f], rng.normal(0, 0.01, 6))
    lam = 1e-5
    costs = []
    for _ in range(30):
        params, lam, info = B.lm_iteration(params, lam, obs, cx, cy)
        costs.append(min(info["cost"], info["trial_cost"]))
    e = np.linalg.norm(B.residuals(params, obs, cx, cy), axis=2)
    mask = B.inlier_mask(e)
    assert not (mask & out).any()
    assert math.sqrt(np.mean(e[~out] ** 2)) < 0.7
    e_gt = np.linalg.norm(B.residuals(gt, obs, cx, cy), axis=2)
    assert B.robust_cost(e, mask, 2.0) <= B.robust_cost(e_gt, mask, 2.0)


def test_accepted_costs_never_increase_from_the_bootstrap_start():
    """From the App. A.1 start (focal 0.7 W, identity poses, depth-1 points) the
    accepted robust cost never increases (each comparison uses the same
    observation set) and falls well below its start."""
    rng = np.random.default_rng(3)
    F, P = 8, 60
    gt, obs, cx, cy, _ = B.synthetic_problem(rng, F=F, P=P, noise_px=0.5)
    params = B.bootstrap_init(obs, F, 640, cx, cy)
    lam = 1e-5
    first = None
    for _ in range(40):
        params, lam, info = B.lm_iteration(params, lam, obs, cx, cy)
        first = info["cost"] if first is None else first
        if info["accepted"]:
            assert info["trial_cost"] < info["cost"]
    assert info["cost"] < 0.05 * first


def test_rejected_step_keeps_parameters():
    """At the exact solution no step lowers the cost: the parameters stay and
    lam doubles."""
    rng = np.random.default_rng(2)
    gt, obs, cx, cy, _ = B.synthetic_problem(rng, F=3, P=10)
    p2, lam, info = B.lm_iteration(gt, 1e-3, obs, cx, cy)
    assert not info["accepted"] and lam == 2e-3
    assert p2 is gt


def test_pose_jacobian_matches_central_differences():
    rng = np.random.default_rng(7)
    R, t, X, obs, cx, cy, _ = B.synthetic_pose_problem(rng, M=8)
    R0, t0 = O.retract_pose(R, t, rng.normal(0, 0.05, 6))
    Jm = B.pose_jacobian(500.0, R0, t0, X)
    h = 1e-6
    for j in range(6):
        d = np.zeros(6)
        d[j] = h
        Rp, tp = O.retract_pose(R0, t0, d)
        Rm, tm = O.retract_pose(R0, t0, -d)
        fd = (B.project(500.0, cx, cy, Rp, tp, X) - B.project(500.0, cx, cy, Rm, tm, X)).reshape(-1) / (2 * h)
        np.testing.assert_allclose(Jm[:, j], fd, rtol=1e-5, atol=1e-6 * np.abs(Jm).max())
    # the pose columns equal the frame's columns of the full bundle adjustment Jacobian
    params = {"fl": 500.0, "R": np.stack([np.eye(3), R0]), "t": np.stack([np.zeros(3), t0]), "X": X}
    full = B.jacobian(params, cx, cy)
    rows = np.concatenate([np.arange(2 * (2 * m + 1), 2 * (2 * m + 1) + 2) for m in range(8)])
    np.testing.assert_allclose(full[rows, :6], Jm, rtol=1e-12, atol=1e-12)


def test_pose_refinement_recovers_the_pose_and_rejects_outliers():
    """0.5 px noise and 10% gross outliers, start 27 mrad / several cm off:
    after 20 iterations (the paper's count) the pose is within 1 mrad and 5 mm,
    every planted outlier is excluded, and the robust cost is at most the true
    pose's on the same observation set."""
    rng = np.random.default_rng(5)
    R, t, X, obs, cx, cy, out = B.synthetic_pose_problem(rng, M=400, noise_px=0.5, outlier_frac=0.1)
    Rc, tc = O.retract_pose(R, t, rng.normal(0, 0.02, 6))
    lam = 1e-5
    for _ in range(20):
        Rc, tc, lam, info = B.pose_lm_iteration(Rc, tc, lam, X, obs, 500.0, cx, cy)
    ang = math.acos(min(1.0, max(-1.0, (np.trace(Rc @ R.T) - 1) / 2)))
    assert ang < 1e-3 and np.linalg.norm(tc - t) < 5e-3
    e = np.linalg.norm(B.project(500.0, cx, cy, Rc, tc, X) - obs, axis=1)
    m = B.inlier_mask(e)
    assert not m[out].any() and m[~out].mean() > 0.98
    e_gt = np.linalg.norm(B.project(500.0, cx, cy, R, t, X) - obs, axis=1)
    assert B.robust_cost(e, m, 2.0) <= B.robust_cost(e_gt, m, 2.0)


def test_pose_rejected_step_keeps_the_pose():
    """Noise-free observations at the true pose: no step lowers the cost, so
    the pose stays and lam grows by nu; lam never exceeds 1e10."""
    rng = np.random.default_rng(8)
    R, t, X, obs, cx, cy, _ = B.synthetic_pose_problem(rng, M=30)
    R2, t2, lam, info = B.pose_lm_iteration(R, t, 1e-3, X, obs, 500.0, cx, cy)
    assert not info["accepted"] and lam == 2e-3 and R2 is R and t2 is t
    _, _, lam, _ = B.pose_lm_iteration(R, t, 8e9, X, obs, 500.0, cx, cy)
    assert lam == 1e10
