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


def excluded_gaussians(view: dict, bad_tiles: np.ndarray) -> np.ndarray:
    """Gaussians listed in any flagged tile, plus those with an ambiguous
    geometric or gradient-path decision."""
    n = view["proj"]["mean2d"].shape[0]
    out = np.zeros(n, bool)
    start, ids = view["start"], view["ids"]
    for t in np.nonzero(bad_tiles.reshape(-1))[0]:
        out[ids[start[t]:start[t + 1]]] = True
    out |= (view["proj"]["amb"] & (1 | 2)) > 0
    return out


def tile_pixel_mask(bad_tiles: np.ndarray, width: int, height: int, tile: int) -> np.ndarray:
    """Pixel mask [H, W] of the pixels lying in flagged tiles."""
    m = np.repeat(np.repeat(bad_tiles, tile, 0), tile, 1)
    return m[:height, :width]


def amb_heavy(g2d, amb, rtol, share=0.3):
    """Items whose 2D adjoint draws more than `share` of the tolerance from
    pixels the oracle flagged as ambiguous (a flip there could move it)."""
    g2d = np.asarray(g2d)
    amb = np.asarray(amb)
    rms = np.sqrt(np.mean(g2d * g2d, axis=0, keepdims=True)) + 1e-300
    return np.any(amb > share * rtol * (np.abs(g2d) + rms), axis=1)


def fp32_adjoint_kappa(n_contrib_max):
    """Relative FP32 error per contribution of the compositing adjoint: the
    transmittance in front of a Gaussian is recovered from T_final through up
    to n_contrib reciprocal-and-multiply steps (about 1.5 ulp each), so a term
    can be off by about n_contrib x 2^-23 relative (bound taken 2x wider)."""
    return 3.0 * 2.0 ** -23 * max(1, int(n_contrib_max))


def ill_conditioned(g2d, absum, rtol, kappa, share=0.3):
    """Items whose 2D adjoint is a sum with so much cancellation that its FP32
    error bound, kappa x the sum of |contributions| (absum, from the oracle),
    exceeds `share` of the tolerance: the FP32 path cannot be held to the
    tolerance there, so such items are excluded and counted like flagged ones."""
    g2d = np.asarray(g2d)
    rms = np.sqrt(np.mean(g2d * g2d, axis=0, keepdims=True)) + 1e-300
    return np.any(kappa * np.asarray(absum) > share * rtol * (np.abs(g2d) + rms), axis=1)


def assert_close_tail(got, ref, rtol, mask=None, what="", min_frac=0.9999, hard=4.0):
    """assert_close for full-size sums: at least min_frac of the entries within
    rtol x (|ref| + rms), every entry within hard x that (FP32 sums over
    hundreds of composited Gaussians and several views leave a thin tail)."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    if mask is not None:
        got = got[mask]
        ref = ref[mask]
    if ref.size == 0:
        return
    rms = float(np.sqrt(np.mean(ref * ref)))
    ratio = np.abs(got - ref) / (rtol * (np.abs(ref) + rms) + 1e-300)
    frac = float(np.mean(ratio <= 1.0))
    assert frac >= min_frac and ratio.max() <= hard, (what, frac, float(ratio.max()), ref.size)
