"""Shared test helpers: tolerance checks and oracle/GPU plumbing."""
from __future__ import annotations

import numpy as np


def assert_close(got, ref, rtol, mask=None, what=""):
    """Per-tensor check |x_gpu - x_ref| <= rtol * (|x_ref| + rms(x_ref)),
    elementwise, over the entries selected by mask."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    if mask is not None:
        got = got[mask]
        ref = ref[mask]
    if ref.size == 0:
        return
    rms = float(np.sqrt(np.mean(ref * ref)))
    err = np.abs(got - ref)
    lim = rtol * (np.abs(ref) + rms)
    bad = ~(err <= lim)
    if bad.any():
        i = np.argmax(np.where(bad, err / np.maximum(lim, 1e-300), 0))
        raise AssertionError(f"{what}: {int(bad.sum())} of {ref.size} entries exceed rtol={rtol} "
                             f"(worst got={got.flat[i]!r} ref={ref.flat[i]!r}, rms={rms:.3e})")


def tile_pixel_mask(bad_tiles: np.ndarray, width: int, height: int, tile: int) -> np.ndarray:
    """Pixel mask [H, W] of the pixels lying in flagged tiles."""
    m = np.repeat(np.repeat(bad_tiles, tile, 0), tile, 1)
    return m[:height, :width]


def assert_within(got, ref, rtol, bound=None, mask=None, what=""):
    """|x_gpu - x_ref| <= rtol * (|x_ref| + rms(x_ref)) + bound, elementwise over
    the entries selected by mask (rms over those entries). bound [same shape,
    >= 0] is the oracle's own estimate of how far an FP32 evaluation may
    legitimately move the value (decisions within their margin taking the
    other branch, rounding). Returns (worst ratio of error to allowance,
    median share of bound / (rtol * (|x_ref| + rms)))."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    bound = np.zeros_like(ref) if bound is None else np.broadcast_to(np.asarray(bound, np.float64), ref.shape)
    if mask is not None:
        got, ref, bound = got[mask], ref[mask], bound[mask]
    if ref.size == 0:
        return 0.0, 0.0
    rms = float(np.sqrt(np.mean(ref * ref)))
    tol = rtol * (np.abs(ref) + rms)
    lim = tol + bound
    err = np.abs(got - ref)
    bad = ~(err <= lim)
    if bad.any():
        i = np.argmax(np.where(bad, err / np.maximum(lim, 1e-300), 0))
        raise AssertionError(f"{what}: {int(bad.sum())} of {ref.size} entries exceed rtol={rtol} + bound "
                             f"(worst got={got.flat[i]!r} ref={ref.flat[i]!r} bound={bound.flat[i]!r}, rms={rms:.3e})")
    return float((err / np.maximum(lim, 1e-300)).max()), float(np.median(bound / np.maximum(tol, 1e-300)))


def workload_gradients(oracle, scene, cams, cfg, views, synth, seed=0):
    """dL/dC of the joint optimisation's L1 loss for each view: the oracle's
    render at the training pose against a target rendered from the same
    scene at a pose perturbed by N(0, 0.01) rad / m (the training poses of the
    benchmark workload are off by that much), sign(C - target) / (3 H W)."""
    rng = np.random.default_rng(seed)
    out = []
    for view, cam in zip(views, cams):
        R, t = synth.perturb_pose(rng, np.asarray(cam["R"], np.float64), np.asarray(cam["t"], np.float64))
        cam2 = dict(cam, R=R.astype(np.float32), t=t.astype(np.float32))
        target = oracle.render_view(scene, cam2, cfg)["color"]
        out.append(np.sign(view["color"] - target) / view["color"].size)
    return out
