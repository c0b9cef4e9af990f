"""FP64 oracle of the guided-matching depth refinement (Sec. 4.2, App. A.2):
per pixel of frame i, candidates uniform in inverse depth around the monocular
estimate, one neighbouring frame chosen per pixel, correlation of feature
vectors along the candidates, and a quadratic fit of the best one.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).

Readings (the appendix fixes the window and the correlation; the rest is ours):
- Feature maps are given per frame, [H][W][C] bfloat16 (16-bit features; bf16
  widens to FP32/FP64 exactly), all at the reference frame's size.
- Pixel (u, v) has centre (u + 0.5, v + 0.5); its ray in camera i is
  r = ((u + 0.5 - cx) / fx, (v + 0.5 - cy) / fy, 1) and a candidate of inverse
  depth d is the point r / d (depth = z in camera i). Cameras map world to
  camera: x_c = R x_w + t.
- Candidates: n inverse depths d_k = d_lo + k (d_hi - d_lo) / (n - 1) with
  d_lo = max(1/Z* - w, 0), d_hi = 1/Z* + w, w = 0.1 (d = 0 is the point at
  infinity, still a valid direction).
- In neighbour j the candidate is a + d b with a = R_ji r, b = t_j - R_ji t_i,
  R_ji = R_j R_i^T (homogeneous in d), projected to x = fx_j X / Z + cx_j.
- A neighbour is usable for a pixel when the whole candidate segment lies in
  front of it (Z > 0 at both ends; Z is linear in d) and inside the bilinear
  domain of its map: sample coordinates s = x - 0.5 in [0, W - 1] x [0, H - 1]
  at both ends (the domain is convex, so the whole segment is). Adaptive
  matching: among usable neighbours the one whose segment is longest in pixels
  (the most depth-discriminative) is chosen; ties go to the lower index.
- C_k = <F_i(u, v), bilinear(F_j, s_k)>; k* = the first maximum; when both
  neighbours of k* exist, the parabola through (k* - 1, k*, k* + 1) gives the
  offset delta = (C_{k*-1} - C_{k*+1}) / (2 (C_{k*-1} - 2 C_{k*} + C_{k*+1}))
  (0 when the denominator is not negative) and d* = d_{k*} + delta (d_hi - d_lo)
  / (n - 1); at either end of the window d* = d_{k*}. Depth = 1 / d*.
- No usable neighbour, a monocular depth that is not a positive finite number,
  or d* = 0: the pixel keeps its monocular depth, neighbour -1, correlation 0.
"""
from __future__ import annotations

import numpy as np

WINDOW = 0.1


def bf16_to_f64(u16):
    """bfloat16 bit patterns (uint16) to float64, exactly."""
    u = np.asarray(u16, np.uint16).astype(np.uint32) << np.uint32(16)
    return u.view(np.float32).astype(np.float64)


def camera_arrays(cam):
    """(R [3][3], t [3], fx, fy, cx, cy, W, H) from a dict with those keys."""
    return (np.asarray(cam["R"], np.float64).reshape(3, 3), np.asarray(cam["t"], np.float64).reshape(3),
            float(cam["fx"]), float(cam["fy"]), float(cam["cx"]), float(cam["cy"]), int(cam["width"]),
            int(cam["height"]))


def pixel_rays(cam):
    """Rays r [H*W][3] of every pixel centre of camera i (z component 1)."""
    _, _, fx, fy, cx, cy, W, H = camera_arrays(cam)
    v, u = np.mgrid[0:H, 0:W]
    return np.stack([((u + 0.5 - cx) / fx).ravel(), ((v + 0.5 - cy) / fy).ravel(), np.ones(H * W)], 1)


def relative(cam_i, cam_j):
    """(R_ji, b): a point r / d of camera i is (R_ji r + d b) / d in camera j."""
    Ri, ti = camera_arrays(cam_i)[:2]
    Rj, tj = camera_arrays(cam_j)[:2]
    Rji = Rj @ Ri.T
    return Rji, tj - Rji @ ti


def reproject(a, b, d, cam_j):
    """Pixel coordinates (x, y) and depth-sign Z of the candidates a + d b
    (a [..., 3], d [...]) in camera j."""
    _, _, fx, fy, cx, cy, _, _ = camera_arrays(cam_j)
    q = a + d[..., None] * b
    return fx * q[..., 0] / q[..., 2] + cx, fy * q[..., 1] / q[..., 2] + cy, q[..., 2]


def candidates(z_mono, n, window=WINDOW):
    """Inverse depths [..., n] uniform over [max(1/Z* - w, 0), 1/Z* + w]."""
    dc = 1.0 / np.asarray(z_mono, np.float64)
    lo = np.maximum(dc - window, 0.0)
    hi = dc + window
    k = np.arange(n) / (n - 1)
    return lo[..., None] + (hi - lo)[..., None] * k


def in_domain(x, y, W, H):
    sx, sy = x - 0.5, y - 0.5
    return (sx >= 0) & (sx <= W - 1) & (sy >= 0) & (sy <= H - 1)


def bilinear(Fj, x, y):
    """Bilinear sample of Fj [H][W][C] at pixel coordinates (x, y) inside the
    domain: weights from s = (x - 0.5, y - 0.5) around the cell (x0, y0), x0 =
    min(floor(sx), W - 2) (the last column gets weight 1 on its own cell)."""
    H, W = Fj.shape[:2]
    sx, sy = x - 0.5, y - 0.5
    x0 = np.minimum(np.floor(sx), W - 2).astype(np.int64)
    y0 = np.minimum(np.floor(sy), H - 2).astype(np.int64)
    wx, wy = sx - x0, sy - y0
    return (((1 - wx) * (1 - wy))[..., None] * Fj[y0, x0] + (wx * (1 - wy))[..., None] * Fj[y0, x0 + 1] +
            ((1 - wx) * wy)[..., None] * Fj[y0 + 1, x0] + (wx * wy)[..., None] * Fj[y0 + 1, x0 + 1])


def fit_peak(cm, c0, cp):
    """Sub-sample offset of the parabola through (-1, cm), (0, c0), (1, cp)."""
    den = cm - 2.0 * c0 + cp
    return np.where(den < 0, (cm - cp) / (2.0 * np.where(den < 0, den, -1.0)), 0.0)


def guided_depth(feat_i, feats_nb, cam_i, cams_nb, z_mono, n_cand=32, window=WINDOW, margins=False, pixels=None):
    """Refined depth of every pixel of frame i (or of the flat pixel indices
    `pixels`, then every output is 1-D over them).

    feat_i [H][W][C] and feats_nb [J][H][W][C]: uint16 bfloat16 patterns;
    z_mono [H][W]. Returns dict(depth [H][W], nb [H][W] int, corr [H][W]) and,
    with margins=True, the per-pixel quantities the FP32 path may decide the
    other way: 'score_gap' (relative gap of the two longest usable segments),
    'edge' (smallest distance in pixels of a segment end to a domain border),
    'front' (smallest Z of a segment end relative to |a|), 'arg_gap' (best
    minus second-best correlation), 'den' (the parabola's curvature),
    'depth_alt', 'den_alt', 'nb_alt' (result, curvature and neighbour output
    had the runner-up candidate been the maximum), 'cbest' (the largest
    correlation, also where the refined inverse depth is not positive)."""
    _, _, _, _, _, _, W, H = camera_arrays(cam_i)
    sel = np.arange(H * W) if pixels is None else np.asarray(pixels, np.int64)
    Fi = bf16_to_f64(np.asarray(feat_i).reshape(H * W, -1)[sel])
    Fn = [bf16_to_f64(f) for f in feats_nb]
    z = np.asarray(z_mono, np.float64).reshape(-1)[sel]
    npx = sel.size
    r = pixel_rays(cam_i)[sel]
    ok = np.isfinite(z) & (z > 0)
    zs = np.where(ok, z, 1.0)
    d = candidates(zs, n_cand, window)
    lo, hi = d[:, 0], d[:, -1]
    best_score = np.full(npx, -1.0)
    second_score = np.full(npx, -1.0)
    nb = np.full(npx, -1, np.int64)
    edge = np.full(npx, np.inf)
    front = np.full(npx, np.inf)
    for j, cam_j in enumerate(cams_nb):
        Rji, b = relative(cam_i, cam_j)
        a = r @ Rji.T
        _, _, _, _, _, _, Wj, Hj = camera_arrays(cam_j)
        x0, y0, z0 = reproject(a, b, lo, cam_j)
        x1, y1, z1 = reproject(a, b, hi, cam_j)
        usable = ok & (z0 > 0) & (z1 > 0) & in_domain(x0, y0, Wj, Hj) & in_domain(x1, y1, Wj, Hj)
        score = np.where(usable, np.hypot(x1 - x0, y1 - y0), -1.0)
        with np.errstate(invalid="ignore", divide="ignore"):
            dist = np.minimum.reduce([np.abs(v) for v in (x0 - 0.5, Wj - 0.5 - x0, y0 - 0.5, Hj - 0.5 - y0,
                                                          x1 - 0.5, Wj - 0.5 - x1, y1 - 0.5, Hj - 0.5 - y1)])
            zrel = np.minimum(np.abs(z0), np.abs(z1)) / np.linalg.norm(a, axis=1)
        edge = np.minimum(edge, np.where(ok & np.isfinite(dist), dist, np.where(ok, 0.0, np.inf)))
        front = np.minimum(front, np.where(ok, zrel, np.inf))
        better = score > best_score
        second_score = np.where(better, best_score, np.maximum(second_score, score))
        nb = np.where(better, j, nb)
        best_score = np.where(better, score, best_score)
    has = nb >= 0
    depth = z.copy()
    corr = np.zeros(npx)
    arg_gap = np.full(npx, np.inf)
    den = np.full(npx, -np.inf)
    depth_alt = depth.copy()
    den_alt = np.full(npx, -np.inf)
    nb_alt = nb.copy()
    cbest = np.zeros(npx)
    for j, cam_j in enumerate(cams_nb):
        idx = np.nonzero(has & (nb == j))[0]
        if idx.size == 0:
            continue
        Rji, b = relative(cam_i, cam_j)
        a = r[idx] @ Rji.T
        dk = d[idx]
        x, y, _ = reproject(a[:, None, :], b, dk, cam_j)
        C = np.empty((idx.size, n_cand))
        for k in range(n_cand):
            C[:, k] = np.einsum("pc,pc->p", Fi[idx], bilinear(Fn[j], x[:, k], y[:, k]))
        step = (dk[:, -1] - dk[:, 0]) / (n_cand - 1)
        rows = np.arange(idx.size)

        def refine(ks):
            cb = C[rows, ks]
            interior = (ks > 0) & (ks < n_cand - 1)
            km, kp = np.clip(ks - 1, 0, n_cand - 1), np.clip(ks + 1, 0, n_cand - 1)
            cm, cp = C[rows, km], C[rows, kp]
            delta = np.where(interior, fit_peak(cm, cb, cp), 0.0)
            return cb, dk[rows, ks] + delta * step, np.where(interior, cm - 2 * cb + cp, -np.inf)

        ks = np.argmax(C, axis=1)
        cb, ds, den[idx] = refine(ks)
        order = np.argsort(-C, axis=1, kind="stable")
        arg_gap[idx] = C[rows, order[:, 0]] - C[rows, order[:, 1]]
        _, ds2, den_alt[idx] = refine(order[:, 1])  # the runner-up as the maximum (a near tie may go either way)
        good = ds > 0
        depth[idx] = np.where(good, 1.0 / np.where(good, ds, 1.0), z[idx])
        depth_alt[idx] = np.where(ds2 > 0, 1.0 / np.where(ds2 > 0, ds2, 1.0), z[idx])
        nb_alt[idx] = np.where(ds2 > 0, j, -1)
        cbest[idx] = cb
        corr[idx] = np.where(good, cb, 0.0)
        nb[idx] = np.where(good, j, -1)
    shape = (H, W) if pixels is None else (npx,)
    out = {"depth": depth.reshape(shape), "nb": nb.reshape(shape), "corr": corr.reshape(shape)}
    if margins:
        with np.errstate(invalid="ignore", divide="ignore"):
            gap = np.where(second_score >= 0, (best_score - second_score) / np.maximum(best_score, 1e-30), np.inf)
        out.update(score_gap=gap.reshape(shape), edge=edge.reshape(shape), front=front.reshape(shape),
                   arg_gap=arg_gap.reshape(shape), den=den.reshape(shape), depth_alt=depth_alt.reshape(shape),
                   den_alt=den_alt.reshape(shape), nb_alt=nb_alt.reshape(shape), cbest=cbest.reshape(shape),
                   inv_step=((hi - lo) / (n_cand - 1)).reshape(shape))
    return out
