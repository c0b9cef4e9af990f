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
