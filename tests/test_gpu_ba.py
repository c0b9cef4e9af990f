"""Mini bundle adjustment on the GPU (Sec. 4.1, App. A.1) against the FP64
oracle: one Levenberg-Marquardt iteration (step, costs, decision), a 30-iteration
run (final robust cost), determinism and CUDA-graph replay."""
import numpy as np
import pytest
import torch

from helpers import assert_close
from oracle import mini_ba as B
from oracle import oracle as O
from paper_2506_05558_gb300 import gs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2506_05558_gb300 import build
    build.build()


def problem(seed, F=6, P=200):
    """0.5 px noise, 3% outliers, start 1-3% off the truth; returns oracle state
    and its FP32 copy (the GPU starts from the same rounded values)."""
    rng = np.random.default_rng(seed)
    gt, obs, cx, cy, out = B.synthetic_problem(rng, F=F, P=P, outlier_frac=0.03, noise_px=0.5)
    params = {"fl": gt["fl"] * 1.03, "R": gt["R"].copy(), "t": gt["t"].copy(),
              "X": gt["X"] * (1 + rng.normal(0, 0.02, gt["X"].shape))}
    for f in range(1, F):
        params["R"][f], params["t"][f] = O.retract_pose(gt["R"][f], gt["t"][f], rng.normal(0, 0.01, 6))
    r32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    params = {k: r32(v) for k, v in params.items()}
    params["fl"] = float(params["fl"])
    return gt, r32(obs), cx, cy, params


def to_device(obs, params):
    P, F = obs.shape[:2]
    poses = np.concatenate([params["R"].reshape(F, 9), params["t"]], 1)
    pts = np.concatenate([params["X"], np.zeros((P, 1))], 1)
    f32 = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda").contiguous()
    return f32(obs), f32([params["fl"]]), f32(poses), f32(pts)


def from_device(fl, poses, pts):
    pz = poses.cpu().numpy().astype(np.float64)
    return {"fl": float(fl.item()), "R": pz[:, :9].reshape(-1, 3, 3), "t": pz[:, 9:12],
            "X": pts.cpu().numpy().astype(np.float64)[:, :3]}


def run_gpu(obs, params, iterations, lam0=1e-5):
    P, F = obs.shape[:2]
    ob, fl, poses, pts = to_device(obs, params)
    lam = torch.tensor([lam0], device="cuda")
    ws = gs.workspace(gs.gs_ba_workspace_size(F, P))
    hist = torch.zeros((max(iterations, 1), 3), device="cuda")
    failed = torch.zeros(1, dtype=torch.int32, device="cuda")
    gs.gs_ba_lm(ob, CX, CY, fl, poses, pts, lam, iterations, ws, failed, history=hist)
    torch.cuda.synchronize()
    assert int(failed.item()) == 0
    return from_device(fl, poses, pts), float(lam.item()), hist.cpu().numpy()


CX, CY = 320.0, 240.0


def test_one_iteration_matches_oracle():
    gt, obs, cx, cy, params = problem(11)
    assert (cx, cy) == (CX, CY)
    e = np.linalg.norm(B.residuals(params, obs, cx, cy), axis=2)
    med = B.lower_median(e)
    thr = med + 4 * B.lower_median(np.abs(e - med))
    assert np.abs(e - thr).min() > 1e-4 * thr  # no observation within FP32 reach of the rejection boundary
    ref, lam_ref, info = B.lm_iteration(params, 1e-5, obs, cx, cy)
    got, lam, hist = run_gpu(obs, params, 1)
    assert info["accepted"] and hist[0, 2] == 1.0 and abs(lam - lam_ref) < 1e-12
    assert abs(hist[0, 0] - info["cost"]) < 1e-4 * info["cost"]
    assert abs(hist[0, 1] - info["trial_cost"]) < 1e-3 * info["trial_cost"]
    assert abs(got["fl"] - ref["fl"]) < 1e-4 * ref["fl"]
    assert_close(got["X"], ref["X"], 1e-4, what="points")
    assert_close(got["R"], ref["R"], 1e-5, what="rotations")
    assert_close(got["t"], ref["t"], 1e-4, what="translations")


def test_thirty_iterations_reach_the_oracle_cost():
    gt, obs, cx, cy, params = problem(12)
    ref, lam_ref = params, 1e-5
    for _ in range(30):
        ref, lam_ref, info = B.lm_iteration(ref, lam_ref, obs, cx, cy)
    got, lam, hist = run_gpu(obs, params, 30)
    accepted = hist[:, 2] > 0
    assert accepted[:3].all() and accepted.sum() >= 4
    final = lambda prm: B.robust_cost(np.linalg.norm(B.residuals(prm, obs, cx, cy), axis=2),
                                      B.inlier_mask(np.linalg.norm(B.residuals(prm, obs, cx, cy), axis=2)), 2.0)
    c_gpu, c_ref = final(got), final(ref)
    assert abs(c_gpu - c_ref) < 1e-3 * c_ref, (c_gpu, c_ref)
    # accepted costs never increase
    acc_costs = hist[accepted, 1]
    assert (np.diff(acc_costs) <= 1e-6 * acc_costs[0]).all()


def test_deterministic_and_graph_replay():
    gt, obs, cx, cy, params = problem(13, F=8, P=500)
    P, F = obs.shape[:2]
    a, _, ha = run_gpu(obs, params, 10)
    b, _, hb = run_gpu(obs, params, 10)
    assert np.array_equal(ha, hb) and np.array_equal(a["X"], b["X"])
    # the same 10 iterations captured into one CUDA graph
    ob, fl, poses, pts = to_device(obs, params)
    lam = torch.tensor([1e-5], device="cuda")
    ws = gs.workspace(gs.gs_ba_workspace_size(F, P))
    hist = torch.zeros((10, 3), device="cuda")
    failed = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        gs.gs_ba_lm(ob, CX, CY, fl, poses, pts, lam, 1, ws, failed, stream=stream)  # warm-up (attributes)
    torch.cuda.synchronize()
    ob, fl, poses, pts = to_device(obs, params)
    lam.fill_(1e-5)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        gs.gs_ba_lm(ob, CX, CY, fl, poses, pts, lam, 10, ws, failed, history=hist, stream=stream)
    g.replay()
    torch.cuda.synchronize()
    c = from_device(fl, poses, pts)
    assert np.array_equal(hist.cpu().numpy(), ha) and np.array_equal(c["X"], a["X"])


def test_invalid_arguments():
    ob = torch.zeros((10, 9, 2), device="cuda")
    f = torch.zeros(1, device="cuda")
    ws = gs.workspace(1024)
    failed = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(RuntimeError):
        gs.gs_ba_lm(ob, 0, 0, f, torch.zeros((9, 12), device="cuda"), torch.zeros((10, 4), device="cuda"), f, 1, ws,
                    failed)  # 9 frames > 8
    assert gs.gs_ba_workspace_size(9, 10) == 0 and gs.gs_ba_workspace_size(1, 10) == 0
    assert gs.gs_ba_workspace_size(8, 0) == 0 and gs.gs_ba_workspace_size(8, 1 << 24) == 0  # over 2^26 observations


def test_large_problem_cost_and_threshold():
    """96,000 observations (12,000 points x 8 frames): the first iteration's cost
    is the robust cost under the oracle's median + 4 MAD set, bracketed by the
    costs at thresholds 1e-4 below and above it (FP32 norms may move an
    observation that close to the boundary)."""
    rng = np.random.default_rng(77)
    F, P = 8, 12000
    gt, obs, cx, cy, _ = B.synthetic_problem(rng, F=F, P=P, outlier_frac=0.03, noise_px=0.5)
    obs = np.asarray(obs, np.float32).astype(np.float64)
    params = {"fl": float(np.float32(gt["fl"] * 1.02)), "R": gt["R"].astype(np.float32).astype(np.float64),
              "t": gt["t"].astype(np.float32).astype(np.float64),
              "X": (gt["X"] * (1 + rng.normal(0, 0.01, gt["X"].shape))).astype(np.float32).astype(np.float64)}
    e = np.linalg.norm(B.residuals(params, obs, cx, cy), axis=2)
    med = B.lower_median(e)
    thr = med + 4 * B.lower_median(np.abs(e - med))
    lo = B.robust_cost(e, e <= thr * (1 - 1e-4), 2.0)
    hi = B.robust_cost(e, e <= thr * (1 + 1e-4), 2.0)
    _, _, hist = run_gpu(obs, params, 1)
    assert lo * (1 - 1e-4) <= hist[0, 0] <= hi * (1 + 1e-4)
    assert B.robust_cost(e, e <= thr, 2.0) > 0 and hist[0, 1] > 0


# ---------------------------------------------------------------------------
# pose refinement of a new frame (points and focal length fixed)
# ---------------------------------------------------------------------------

def pose_problem(seed, M=500):
    rng = np.random.default_rng(seed)
    R, t, X, obs, cx, cy, out = B.synthetic_pose_problem(rng, M=M, noise_px=0.5, outlier_frac=0.1)
    R0, t0 = O.retract_pose(R, t, rng.normal(0, 0.02, 6))
    r32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    return (R, t), r32(X), r32(obs), cx, cy, r32(R0), r32(t0), out


def run_pose_gpu(X, obs, R0, t0, iterations, fl=500.0, lam0=1e-5, graph=False):
    M = X.shape[0]
    f32 = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda").contiguous()
    pts = f32(np.concatenate([X, np.zeros((M, 1))], 1))
    ob = f32(obs)
    flt = f32([fl])
    pose = f32(np.concatenate([R0.reshape(9), t0]))
    lam = f32([lam0])
    ws = gs.workspace(gs.gs_ba_pose_workspace_size(M))
    hist = torch.zeros((max(iterations, 1), 3), device="cuda")
    failed = torch.zeros(1, dtype=torch.int32, device="cuda")
    if graph:
        gs.gs_ba_pose_lm(pts, ob, flt, CX, CY, pose.clone(), lam.clone(), 1, ws, failed)  # set-up outside capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        with torch.cuda.graph(g, stream=s):
            gs.gs_ba_pose_lm(pts, ob, flt, CX, CY, pose, lam, iterations, ws, failed, history=hist, stream=s)
        g.replay()
    else:
        gs.gs_ba_pose_lm(pts, ob, flt, CX, CY, pose, lam, iterations, ws, failed, history=hist)
    torch.cuda.synchronize()
    assert int(failed.item()) == 0
    pz = pose.cpu().numpy().astype(np.float64)
    return pz[:9].reshape(3, 3), pz[9:], float(lam.item()), hist.cpu().numpy()


def test_pose_one_iteration_matches_oracle():
    _, X, obs, cx, cy, R0, t0, _ = pose_problem(21)
    assert (cx, cy) == (CX, CY)
    e = np.linalg.norm(B.project(500.0, cx, cy, R0, t0, X) - obs, axis=1)
    med = B.lower_median(e)
    thr = med + 4 * B.lower_median(np.abs(e - med))
    assert np.abs(e - thr).min() > 1e-4 * thr
    R1, t1, lam_ref, info = B.pose_lm_iteration(R0, t0, 1e-5, X, obs, 500.0, cx, cy)
    R, t, lam, hist = run_pose_gpu(X, obs, R0, t0, 1)
    assert info["accepted"] and hist[0, 2] == 1.0 and abs(lam - lam_ref) < 1e-12
    assert abs(hist[0, 0] - info["cost"]) < 1e-4 * info["cost"]
    assert abs(hist[0, 1] - info["trial_cost"]) < 1e-3 * info["trial_cost"]
    assert np.abs(R - R1).max() < 2e-6 and np.abs(t - t1).max() < 2e-6


def test_pose_twenty_iterations_recover_the_pose():
    (Rt, tt), X, obs, cx, cy, R0, t0, _ = pose_problem(22, M=2000)
    R, t, lam, hist = run_pose_gpu(X, obs, R0, t0, 20)
    Rr, tr, lr = R0, t0, 1e-5
    for _ in range(20):
        Rr, tr, lr, info = B.pose_lm_iteration(Rr, tr, lr, X, obs, 500.0, cx, cy)
    for Ra, ta in ((R, t), (Rr, tr)):
        ang = np.arccos(np.clip((np.trace(Ra @ Rt.T) - 1) / 2, -1, 1))
        assert ang < 1e-3 and np.linalg.norm(ta - tt) < 5e-3
    assert abs(hist[-1, 0] - info["cost"]) < 1e-2 * info["cost"]


def test_pose_graph_replay_is_bit_exact():
    _, X, obs, cx, cy, R0, t0, _ = pose_problem(23, M=6144)
    a = run_pose_gpu(X, obs, R0, t0, 20)
    b = run_pose_gpu(X, obs, R0, t0, 20, graph=True)
    c = run_pose_gpu(X, obs, R0, t0, 20)
    for x, y, z in zip(a, b, c):
        assert np.array_equal(np.asarray(x), np.asarray(y)) and np.array_equal(np.asarray(x), np.asarray(z))


def test_pose_invalid_arguments():
    assert gs.gs_ba_pose_workspace_size(0) == 0 and gs.gs_ba_pose_workspace_size(1 << 27) == 0
    pts = torch.zeros((10, 4), device="cuda")
    ob = torch.zeros((10, 2), device="cuda")
    f = torch.ones(1, device="cuda")
    pose = torch.zeros(12, device="cuda")
    failed = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = gs.workspace(gs.gs_ba_pose_workspace_size(10))
    with pytest.raises(RuntimeError):
        gs.gs_ba_pose_lm(pts, ob, f, 0, 0, pose, f, 1, ws, failed, nu=1.0)
    with pytest.raises(RuntimeError):
        gs.gs_ba_pose_lm(pts, ob, f, 0, 0, pose, f, 1, ws[:16], failed)  # workspace too small
