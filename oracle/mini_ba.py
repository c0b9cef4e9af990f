"""FP64 oracle of the mini bundle adjustment of the initial pose estimation
(Sec. 4.1 bootstrapping, App. A.1): Levenberg-Marquardt over a shared focal
length, the poses of frames 1..F-1 (frame 0 is held fixed: the gauge) and P
3-D points, each point observed in all F frames (the fixed-size layout).

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).

Model: pixel of point p in frame f = (fl x / z + cx, fl y / z + cy) with
(x, y, z) = R_f X_p + t_f; residual r_pf = pixel - observed (2-vector). Per
iteration: residual norms e_pf; observations with e > median + 4 MAD (lower
median, MAD = lower median of |e - median|) are discarded; the rest are
weighted by Huber with threshold delta (weight 1 inside, delta / e outside;
cost 0.5 e^2 inside, delta (e - delta / 2) outside). The step solves
(H + lam diag(H) + 1e-9 I) d = -g with H = J^T W J and g = J^T W r over the
parameters
(pose tangents of frames 1..F-1 as left perturbations T <- exp(d^) T, the
focal length, the points), written out as the dense normal equations. A step
is accepted when the robust cost over the same observation set decreases: then
lam /= nu, else the parameters stay and lam *= nu; lam stays within
[1e-12, 1e10].
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def project(fl, cx, cy, R, t, X):
    """Pixels [P][2] of points X [P][3] in a camera (R, t)."""
    q = X @ R.T + t
    return np.stack([fl * q[:, 0] / q[:, 2] + cx, fl * q[:, 1] / q[:, 2] + cy], 1)


def residuals(params, obs, cx, cy):
    """r [P][F][2] for params = dict(fl, R [F][3][3], t [F][3], X [P][3])."""
    F = obs.shape[1]
    return np.stack([project(params["fl"], cx, cy, params["R"][f], params["t"][f], params["X"]) - obs[:, f]
                     for f in range(F)], 1)


def lower_median(a):
    a = np.sort(np.asarray(a, np.float64).reshape(-1))
    return a[(a.size - 1) // 2]


def inlier_mask(e):
    """Observations kept: e <= median + 4 MAD (App. A.1)."""
    med = lower_median(e)
    mad = lower_median(np.abs(e - med))
    return e <= med + 4.0 * mad


def robust_cost(e, mask, delta):
    e = np.where(mask, e, 0.0)
    return float(np.where(e <= delta, 0.5 * e * e, delta * (e - 0.5 * delta)).sum())


def jacobian(params, cx, cy):
    """Dense Jacobian [P*F*2][6(F-1) + 1 + 3P] of the residuals with respect to
    (pose tangents of frames 1.., focal length, points), each column by its
    analytic derivative: for q = R X + t, d pixel / d q = fl / z [[1, 0, -x/z],
    [0, 1, -y/z]]; a left perturbation moves q by rho + phi x q; d/dX = R."""
    fl, R, t, X = params["fl"], params["R"], params["t"], params["X"]
    P, F = X.shape[0], R.shape[0]
    nc = 6 * (F - 1) + 1
    Jm = np.zeros((P * F * 2, nc + 3 * P))
    for p in range(P):
        for f in range(F):
            q = R[f] @ X[p] + t[f]
            x, y, z = q
            dq = fl / z * np.array([[1, 0, -x / z], [0, 1, -y / z]])
            row = (p * F + f) * 2
            if f > 0:
                # d q / d (rho, phi) = [I, -q^]
                Jm[row:row + 2, 6 * (f - 1):6 * (f - 1) + 3] = dq
                Jm[row:row + 2, 6 * (f - 1) + 3:6 * f] = dq @ -O.hat(q)
            Jm[row:row + 2, nc - 1] = [x / z, y / z]
            Jm[row:row + 2, nc + 3 * p:nc + 3 * p + 3] = dq @ R[f]
    return Jm


def apply_step(params, d):
    F = params["R"].shape[0]
    P = params["X"].shape[0]
    nc = 6 * (F - 1) + 1
    out = {"fl": params["fl"] + d[nc - 1], "R": params["R"].copy(), "t": params["t"].copy(),
           "X": params["X"] + d[nc:].reshape(P, 3)}
    for f in range(1, F):
        out["R"][f], out["t"][f] = O.retract_pose(params["R"][f], params["t"][f], d[6 * (f - 1):6 * f])
    return out


def lm_iteration(params, lam, obs, cx, cy, delta=2.0, nu=2.0):
    """One Levenberg-Marquardt iteration. Returns (params, lam, info)."""
    r = residuals(params, obs, cx, cy)
    e = np.linalg.norm(r, axis=2)
    mask = inlier_mask(e)
    w = np.where(mask, np.where(e <= delta, 1.0, delta / np.maximum(e, 1e-300)), 0.0)
    Jm = jacobian(params, cx, cy)
    wr = np.repeat(w.reshape(-1), 2)
    H = Jm.T @ (wr[:, None] * Jm)
    g = Jm.T @ (wr * r.reshape(-1))
    # Marquardt damping plus an absolute floor 1e-9 on the diagonal, so a
    # parameter without any kept observation gets a zero step instead of a
    # singular system
    dg = np.diag(H)
    A = H + np.diag(lam * dg + 1e-9)
    d = np.linalg.solve(A, -g)
    trial = apply_step(params, d)
    c0 = robust_cost(e, mask, delta)
    c1 = robust_cost(np.linalg.norm(residuals(trial, obs, cx, cy), axis=2), mask, delta)
    info = dict(cost=c0, trial_cost=c1, step=d, inliers=int(mask.sum()), accepted=c1 < c0)
    # lam is kept within [1e-12, 1e10] (a converged run rejects every step)
    if c1 < c0:
        return trial, max(1e-12, lam / nu), info
    return params, min(1e10, lam * nu), info


def bootstrap_init(obs, F, width, cx, cy):
    """Initial values of App. A.1: focal length 0.7 x width, identity poses,
    points at depth 1 on their frame-0 rays."""
    fl = 0.7 * width
    uv = obs[:, 0]
    X = np.stack([(uv[:, 0] - cx) / fl, (uv[:, 1] - cy) / fl, np.ones(len(uv))], 1)
    return {"fl": fl, "R": np.tile(np.eye(3), (F, 1, 1)), "t": np.zeros((F, 3)), "X": X}


def synthetic_problem(rng, F=8, P=200, width=640, height=480, fl=500.0, noise_px=0.0, outlier_frac=0.0):
    """Seeded two-view-style bootstrapping problem: points in a box 3-8 m in
    front of frame 0, frames on a short forward path (0.1 m and 2 degrees per
    frame), observations with optional pixel noise and gross outliers (30-80 px
    off). Returns (ground truth params, obs [P][F][2], cx, cy, outlier mask)."""
    cx, cy = width / 2.0, height / 2.0
    X = np.stack([rng.uniform(-2, 2, P), rng.uniform(-1.5, 1.5, P), rng.uniform(3, 8, P)], 1)
    R = np.tile(np.eye(3), (F, 1, 1))
    t = np.zeros((F, 3))
    for f in range(1, F):
        xi = np.concatenate([rng.normal(0, 0.05, 3) + [0.1 * f, 0, 0], rng.normal(0, 0.02, 3) + [0, 0.035 * f, 0]])
        R[f], t[f] = O.retract_pose(np.eye(3), np.zeros(3), xi)
    gt = {"fl": fl, "R": R, "t": t, "X": X}
    obs = residuals(gt, np.zeros((P, F, 2)), cx, cy) + rng.normal(0, noise_px, (P, F, 2))
    out = rng.random((P, F)) < outlier_frac
    ang = rng.uniform(0, 2 * np.pi, (P, F))
    mag = rng.uniform(30, 80, (P, F))
    obs[out] += np.stack([np.cos(ang), np.sin(ang)], -1)[out] * mag[out][:, None]
    return gt, obs, cx, cy, out


# ---------------------------------------------------------------------------
# Pose refinement of a new frame (Sec. 4.1, subsequent frames): the same
# robust Levenberg-Marquardt iteration over one camera pose only, the 3-D
# points (triangulated from earlier frames) and the focal length held fixed.
# ---------------------------------------------------------------------------

def pose_jacobian(fl, R, t, X):
    """Jacobian [2M][6] of the residuals of points X [M][3] in camera (R, t)
    with respect to a left perturbation (rho, phi) of the pose: for q = R X + t,
    d pixel / d q = fl / z [[1, 0, -x/z], [0, 1, -y/z]] and d q / d(rho, phi) =
    [I, -q^]."""
    M = X.shape[0]
    Jm = np.zeros((2 * M, 6))
    for m in range(M):
        q = R @ X[m] + t
        x, y, z = q
        dq = fl / z * np.array([[1, 0, -x / z], [0, 1, -y / z]])
        Jm[2 * m:2 * m + 2, :3] = dq
        Jm[2 * m:2 * m + 2, 3:] = dq @ -O.hat(q)
    return Jm


def pose_lm_iteration(R, t, lam, X, obs, fl, cx, cy, delta=2.0, nu=2.0):
    """One Levenberg-Marquardt iteration on the pose (R, t) against obs [M][2].
    Same robust terms, damping, floor and decision as lm_iteration. Returns
    (R, t, lam, info)."""
    r = project(fl, cx, cy, R, t, X) - obs
    e = np.linalg.norm(r, axis=1)
    mask = inlier_mask(e)
    w = np.where(mask, np.where(e <= delta, 1.0, delta / np.maximum(e, 1e-300)), 0.0)
    Jm = pose_jacobian(fl, R, t, X)
    wr = np.repeat(w, 2)
    H = Jm.T @ (wr[:, None] * Jm)
    g = Jm.T @ (wr * r.reshape(-1))
    A = H + np.diag(lam * np.diag(H) + 1e-9)
    d = np.linalg.solve(A, -g)
    R1, t1 = O.retract_pose(R, t, d)
    c0 = robust_cost(e, mask, delta)
    c1 = robust_cost(np.linalg.norm(project(fl, cx, cy, R1, t1, X) - obs, axis=1), mask, delta)
    info = dict(cost=c0, trial_cost=c1, step=d, inliers=int(mask.sum()), accepted=c1 < c0)
    if c1 < c0:
        return R1, t1, max(1e-12, lam / nu), info
    return R, t, min(1e10, lam * nu), info


def synthetic_pose_problem(rng, M=500, width=640, height=480, fl=500.0, noise_px=0.0, outlier_frac=0.0):
    """Seeded 3-D to 2-D problem of a new frame: points in a box 3-8 m ahead of
    the origin, a true pose 0.3 m and a few degrees from it, observations with
    optional pixel noise and gross outliers (30-80 px off). Returns (R, t, X,
    obs, cx, cy, outlier mask)."""
    cx, cy = width / 2.0, height / 2.0
    X = np.stack([rng.uniform(-2, 2, M), rng.uniform(-1.5, 1.5, M), rng.uniform(3, 8, M)], 1)
    xi = np.concatenate([rng.normal(0, 0.05, 3) + [0.3, 0, 0], rng.normal(0, 0.02, 3) + [0, 0.05, 0]])
    R, t = O.retract_pose(np.eye(3), np.zeros(3), xi)
    obs = project(fl, cx, cy, R, t, X) + rng.normal(0, noise_px, (M, 2))
    out = rng.random(M) < outlier_frac
    ang = rng.uniform(0, 2 * np.pi, M)
    mag = rng.uniform(30, 80, M)
    obs[out] += np.stack([np.cos(ang), np.sin(ang)], -1)[out] * mag[out][:, None]
    return R, t, X, obs, cx, cy, out
