"""Seeded synthetic inputs shared by the CUDA path, the tests and the bench.

This module draws numbers only. It holds none of the rasterizer's arithmetic
(no projection, no SH evaluation, no compositing), so the FP64 oracle and the
CUDA path can both consume its arrays without sharing any method code.

The scene shapes follow the paper's captures (Sec. 5): ordered camera paths,
images 1200-1920 px wide, about one million small, roughly isotropic
primitives of the kind direct sampling produces (Sec. 4.2, Sec. 6.3).

Layout of a Gaussian set (float32, structure of arrays):
  mean_opa [N, 4]  world position x, y, z and the opacity logit
  scale    [N, 4]  log-scales along the three principal axes, then 0
  quat     [N, 4]  rotation quaternion (w, x, y, z), not normalised
  sh       [N, 48] SH coefficients, coefficient-major: sh[g, 3*k + c]
A camera is a dict with R (3x3 world-to-camera rotation, row-major), t (3),
fx, fy, cx, cy, width, height. The camera looks down +z.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# Standard deviation of the SH DC coefficient that spreads colours by about
# 0.2 around mid-grey (colour = 0.5 + 0.282 * DC for degree-0 SH).
DC_STD = 0.709


@dataclass
class Scene:
    mean_opa: np.ndarray
    scale: np.ndarray
    quat: np.ndarray
    sh: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.mean_opa.shape[0])


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussians(rng: np.random.Generator, n: int, lo, hi, log_scale_mu: float,
              log_scale_sd: float, sh_degree: int, band_sd: float = 0.05) -> Scene:
    """Gaussians with means uniform in the box [lo, hi]."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    mean = lo + (hi - lo) * rng.random((n, 3))
    logit = rng.standard_normal(n)
    mean_opa = np.concatenate([mean, logit[:, None]], 1).astype(np.float32)
    scale = np.zeros((n, 4), np.float32)
    scale[:, :3] = rng.normal(log_scale_mu, log_scale_sd, (n, 3))
    quat = rng.standard_normal((n, 4)).astype(np.float32)
    sh = np.zeros((n, 48), np.float32)
    sh[:, 0:3] = rng.normal(0.0, DC_STD, (n, 3))
    n_coef = (sh_degree + 1) ** 2
    if n_coef > 1:
        sh[:, 3:3 * n_coef] = rng.normal(0.0, band_sd, (n, 3 * n_coef - 3))
    return Scene(mean_opa, scale, quat, sh, sh_degree)


def frustum_gaussians(rng, n, width, height, f, zmin, zmax, log_scale_mu,
                      log_scale_sd, sh_degree) -> Scene:
    """Gaussians uniform in depth and uniform across the image at that depth."""
    z = zmin + (zmax - zmin) * rng.random(n)
    x = (rng.random(n) - 0.5) * width * z / f
    y = (rng.random(n) - 0.5) * height * z / f
    sc = gaussians(rng, n, [0, 0, 0], [1, 1, 1], log_scale_mu, log_scale_sd, sh_degree)
    sc.mean_opa[:, 0] = x
    sc.mean_opa[:, 1] = y
    sc.mean_opa[:, 2] = z
    return sc


def camera(R, t, f, width, height, fy=None, dtype=np.float32) -> dict:
    """Pinhole camera with the principal point at the image centre. Stored in
    float32 (the values both the CUDA path and the oracle consume) unless dtype
    says otherwise."""
    return dict(R=np.asarray(R, dtype).reshape(3, 3), t=np.asarray(t, dtype).reshape(3),
                fx=float(f), fy=float(f if fy is None else fy), cx=width / 2.0, cy=height / 2.0,
                width=int(width), height=int(height))


def _yaw(a: float) -> np.ndarray:
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]], np.float64)


def camera_path(rng, n_views, step_m=0.3, step_deg=5.0):
    """Camera-to-world rotations and centres along a smooth random path.

    Consecutive frames are step_m apart and turn by step_deg about the vertical
    axis; the turn direction changes sign with probability 0.25 per frame so the
    path wiggles but stays smooth. Returns a list of (R_cw, centre).
    """
    yaw = 0.0
    sign = 1.0 if rng.random() < 0.5 else -1.0
    c = np.zeros(3)
    out = []
    for k in range(n_views):
        out.append((_yaw(yaw), c.copy()))
        if rng.random() < 0.25:
            sign = -sign
        yaw += sign * math.radians(step_deg) * 0.5
        fwd = _yaw(yaw) @ np.array([0.0, 0.0, 1.0])
        c = c + step_m * fwd
        yaw += sign * math.radians(step_deg) * 0.5
    # centre the path's yaw range on the box axis
    mid = sum(math.atan2(r[0, 2], r[2, 2]) for r, _ in out) / n_views
    back = _yaw(-mid)
    return [(back @ r, back @ p) for r, p in out]


def world_to_camera(R_cw: np.ndarray, centre: np.ndarray):
    R = R_cw.T
    t = -R @ centre
    return R, t


def perturb_pose(rng, R, t, rot_sd=0.01, trans_sd=0.01):
    """Left-multiplies the world-to-camera pose by a random small rigid motion."""
    w = rng.normal(0, rot_sd, 3)
    th = float(np.linalg.norm(w))
    K = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    if th > 0:
        dR = np.eye(3) + math.sin(th) / th * K + (1 - math.cos(th)) / th ** 2 * K @ K
    else:
        dR = np.eye(3)
    dt = rng.normal(0, trans_sd, 3)
    return dR @ R, dR @ t + dt


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

def tiny_scene(seed=1000, n=1000, width=64, height=64, f=80.0, sh_degree=0):
    """Single 64x64 view, fx=fy=80, 1,000 Gaussians in the frustum at depth 2-6,
    log-scales N(-3, 0.5), random quaternions, opacity sigmoid(N(0,1)), SH0."""
    rng = _rng(seed)
    sc = frustum_gaussians(rng, n, width, height, f, 2.0, 6.0, -3.0, 0.5, sh_degree)
    cam = camera(np.eye(3), np.zeros(3), f, width, height)
    return sc, cam, rng


def view_720p_scene(seed=1001, n=200_000):
    """Single 1280x720 view, fx=fy=1000, 200k Gaussians in a 20x10x30 m box in
    front of the camera, log-scales N(-4, 0.7), SH degree 3."""
    rng = _rng(seed)
    sc = gaussians(rng, n, [-10, -5, 2], [10, 5, 32], -4.0, 0.7, 3)
    cam = camera(np.eye(3), np.zeros(3), 1000.0, 1280, 720)
    return sc, cam, rng


def multiview_scene(seed=1002, n=1_000_000, n_views=8, sizes=None, f_per_width=1500.0 / 1920.0):
    """n Gaussians (SH3) in a 30x15x50 m box and n_views cameras on a smooth path
    (0.3 m and 5 degrees between frames). sizes: list of (width, height) per view
    (default 1920x1080). The focal length keeps a 65-degree horizontal field of view."""
    rng = _rng(seed)
    sc = gaussians(rng, n, [-15, -7.5, 2], [15, 7.5, 52], -4.0, 0.7, 3)
    if sizes is None:
        sizes = [(1920, 1080)] * n_views
    cams = []
    for (R_cw, c), (w, h) in zip(camera_path(rng, n_views), sizes):
        R, t = world_to_camera(R_cw, c)
        cams.append(camera(R, t, f_per_width * w, w, h))
    return sc, cams, rng


UNEVEN_SIZES = [(640, 480), (1280, 720), (1600, 1200), (1920, 1080)]


def uneven_sizes(rng, n_views):
    idx = rng.integers(0, len(UNEVEN_SIZES), n_views)
    return [UNEVEN_SIZES[i] for i in idx]


def image(rng, width, height, lo=0.0, hi=1.0):
    return (lo + (hi - lo) * rng.random((3, height, width))).astype(np.float32)


def scene_subset(sc: Scene, idx) -> Scene:
    return Scene(sc.mean_opa[idx].copy(), sc.scale[idx].copy(), sc.quat[idx].copy(),
                 sc.sh[idx].copy(), sc.sh_degree)


def projected_items(rng, n_items, tiles_x, tiles_y, tile, max_rect=4, depth_levels=None):
    """Synthetic projected splats for testing the sort and the compositing on their
    own: random centres, conics, opacities, colours, depths and tile rects.

    Returned arrays follow the projected-buffer layout (mean2d [n,2],
    conic_opa [n,4], rgb_depth [n,4], rect [n,4] int32 tile bounds, n_tiles [n]).
    depth_levels: if given, depths are drawn from that many discrete values so
    that exact ties occur.
    """
    W, H = tiles_x * tile, tiles_y * tile
    mean2d = np.stack([rng.random(n_items) * W, rng.random(n_items) * H], 1).astype(np.float32)
    # conic from a random SPD 2x2 matrix with eigenvalues in [0.5, 30] px^2
    ang = rng.random(n_items) * math.pi
    l1 = np.exp(rng.uniform(math.log(0.5), math.log(30.0), n_items))
    l2 = np.exp(rng.uniform(math.log(0.5), math.log(30.0), n_items))
    c, s = np.cos(ang), np.sin(ang)
    a = c * c / l1 + s * s / l2
    b = c * s * (1 / l1 - 1 / l2)
    d = s * s / l1 + c * c / l2
    opa = 1.0 / (1.0 + np.exp(-rng.standard_normal(n_items)))
    conic_opa = np.stack([a, b, d, opa], 1).astype(np.float32)
    if depth_levels:
        depth = (1.0 + rng.integers(0, depth_levels, n_items)).astype(np.float32)
    else:
        depth = rng.uniform(0.5, 50.0, n_items).astype(np.float32)
    rgb = rng.random((n_items, 3)).astype(np.float32)
    rgb_depth = np.concatenate([rgb, depth[:, None]], 1).astype(np.float32)
    x0 = rng.integers(0, tiles_x, n_items)
    y0 = rng.integers(0, tiles_y, n_items)
    x1 = np.minimum(x0 + rng.integers(1, max_rect + 1, n_items), tiles_x)
    y1 = np.minimum(y0 + rng.integers(1, max_rect + 1, n_items), tiles_y)
    rect = np.stack([x0, y0, x1, y1], 1).astype(np.int32)
    # a share of culled items (empty rect)
    culled = rng.random(n_items) < 0.1
    rect[culled] = 0
    n_tiles = ((rect[:, 2] - rect[:, 0]) * (rect[:, 3] - rect[:, 1])).astype(np.int32)
    return dict(mean2d=mean2d, conic_opa=conic_opa, rgb_depth=rgb_depth, rect=rect, n_tiles=n_tiles)


def ba_problem(seed=1005, n_frames=8, n_points=6144, width=1920, fl=1500.0, noise_px=0.5, outlier_frac=0.03):
    """Seeded inputs of a bootstrapping mini bundle adjustment shaped like the
    paper's (8 initial frames, 6144 keypoints): ground-truth points in a box
    3-8 m ahead, frame poses as small tangent steps along a forward path
    (0.1 m and 2 degrees per frame, jittered), per-observation pixel noise and
    gross-outlier offsets (30-80 px on outlier_frac of the observations), and
    start-state jitters. Only random draws: the caller builds poses and
    observations from them."""
    rng = _rng(seed)
    P, F = n_points, n_frames
    X = np.stack([rng.uniform(-2, 2, P), rng.uniform(-1.5, 1.5, P), rng.uniform(3, 8, P)], 1)
    xi = np.zeros((F, 6))
    for f in range(1, F):
        xi[f] = np.concatenate([rng.normal(0, 0.05, 3) + [0.1 * f, 0, 0], rng.normal(0, 0.02, 3) + [0, 0.035 * f, 0]])
    noise = rng.normal(0, noise_px, (P, F, 2))
    out = rng.random((P, F)) < outlier_frac
    ang = rng.uniform(0, 2 * np.pi, (P, F))
    mag = rng.uniform(30, 80, (P, F))
    noise[out] += np.stack([np.cos(ang), np.sin(ang)], -1)[out] * mag[out][:, None]
    return dict(X=X, xi=xi, noise=noise, fl=fl, width=width, start_X_scale=1 + rng.normal(0, 0.02, (P, 3)),
                start_xi=rng.normal(0, 0.01, (F, 6)), start_fl=1.03)


def to_bf16(x) -> np.ndarray:
    """bfloat16 bit patterns (uint16) of x, rounded to nearest even from float32."""
    u = np.ascontiguousarray(np.asarray(x, np.float32)).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)


def guided_scene(seed=1006, width=1920, height=1080, f=1500.0, n_nb=4, channels=32, period_px=(8.0, 40.0),
                 mono_sd=0.05, mono_holes=0.01, n_boxes=4):
    """Multi-view feature maps of a synthetic room, the input of guided depth
    matching: a reference frame (the newest of a camera path, 0.3 m and 5
    degrees per frame) and n_nb earlier frames. The room is a ray-cast set of
    planes (back wall, floor, ceiling, side walls, n_boxes fronto-parallel
    rectangles 3-6 m ahead); each pixel's feature vector is a smooth random
    field of the world point it sees (random mixtures of 8 sinusoids whose
    periods span period_px pixels at 5 m), normalised to unit length and
    rounded to bfloat16. The monocular depth is the reference's true depth
    times exp(N(0, mono_sd)), with a fraction mono_holes of pixels set to 0.
    Returns dict(cams [1 + n_nb] (reference first), feats uint16
    [1 + n_nb][H][W][C], z_mono float32 [H][W], z_true float32 [H][W])."""
    rng = _rng(seed)
    path = camera_path(rng, n_nb + 1)
    order = [n_nb] + list(range(n_nb))
    cams = [camera(*world_to_camera(*path[k]), f, width, height) for k in order]
    planes = [(np.array([0.0, 0.0, 1.0]), 9.0, None), (np.array([0.0, 1.0, 0.0]), 1.6, None),
              (np.array([0.0, 1.0, 0.0]), -1.8, None), (np.array([1.0, 0.0, 0.0]), -3.5, None),
              (np.array([1.0, 0.0, 0.0]), 3.5, None)]
    for _ in range(n_boxes):
        zc, xc, yc = rng.uniform(3, 6), rng.uniform(-2, 2), rng.uniform(-1, 1)
        hw, hh = rng.uniform(0.3, 1.0), rng.uniform(0.3, 1.0)
        planes.append((np.array([0.0, 0.0, 1.0]), zc, (xc - hw, xc + hw, yc - hh, yc + hh)))
    lo_m, hi_m = (p * 5.0 / f for p in period_px)
    dirs = rng.normal(size=(8, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    omega = dirs * (2 * np.pi / rng.uniform(lo_m, hi_m, 8))[:, None]
    phase = rng.uniform(0, 2 * np.pi, 8)
    mix = rng.normal(size=(8, channels))
    feats = np.empty((n_nb + 1, height, width, channels), np.uint16)
    z_true = None
    v, u = np.mgrid[0:height, 0:width]
    for k, cam in enumerate(cams):
        R, t = cam["R"].astype(np.float64), cam["t"].astype(np.float64)
        ray = np.stack([((u + 0.5 - cam["cx"]) / cam["fx"]).ravel(), ((v + 0.5 - cam["cy"]) / cam["fy"]).ravel(),
                        np.ones(height * width)], 1)
        dw = ray @ R  # world directions R^T ray
        c = -R.T @ t
        s_best = np.full(height * width, np.inf)
        for n, off, rect in planes:
            den = dw @ n
            with np.errstate(divide="ignore", invalid="ignore"):
                s = (off - n @ c) / den
            hit = np.isfinite(s) & (s > 0.05)
            if rect is not None:
                p = c + s[:, None] * dw
                hit &= (p[:, 0] >= rect[0]) & (p[:, 0] <= rect[1]) & (p[:, 1] >= rect[2]) & (p[:, 1] <= rect[3])
            s_best = np.where(hit & (s < s_best), s, s_best)
        s_best = np.where(np.isfinite(s_best), s_best, 50.0)
        X = c + s_best[:, None] * dw
        fv = np.sin(X @ omega.T + phase) @ mix
        fv /= np.linalg.norm(fv, axis=1, keepdims=True) + 1e-12
        feats[k] = to_bf16(fv).reshape(height, width, channels)
        if k == 0:
            z_true = s_best.reshape(height, width).astype(np.float32)
    z_mono = (z_true * np.exp(rng.normal(0, mono_sd, z_true.shape))).astype(np.float32)
    z_mono[rng.random(z_true.shape) < mono_holes] = 0.0
    return dict(cams=cams, feats=feats, z_mono=z_mono, z_true=z_true)


def ba_pose_problem(seed=1007, n_obs=6144, width=1920, fl=1500.0, noise_px=0.5, outlier_frac=0.1):
    """Seeded inputs of a new frame's pose refinement (6144 keypoints matched
    to triangulated points): points in a box 3-8 m ahead, the true pose as a
    tangent step (0.3 m and a few degrees, jittered), per-observation pixel
    noise and gross outliers (30-80 px on outlier_frac of them), and the start
    pose's tangent offset (about 0.02 rad / 0.02 m, a RANSAC estimate). Only
    random draws: the caller builds the pose and the observations."""
    rng = _rng(seed)
    M = n_obs
    X = np.stack([rng.uniform(-2, 2, M), rng.uniform(-1.5, 1.5, M), rng.uniform(3, 8, M)], 1)
    xi = np.concatenate([rng.normal(0, 0.05, 3) + [0.3, 0, 0], rng.normal(0, 0.02, 3) + [0, 0.05, 0]])
    noise = rng.normal(0, noise_px, (M, 2))
    out = rng.random(M) < outlier_frac
    ang = rng.uniform(0, 2 * np.pi, M)
    mag = rng.uniform(30, 80, M)
    noise[out] += np.stack([np.cos(ang), np.sin(ang)], -1)[out] * mag[out][:, None]
    return dict(X=X, xi=xi, noise=noise, fl=fl, width=width, start_xi=rng.normal(0, 0.02, 6))


def surface_scene(seed=1008, n=120_000, n_views=10, size=(256, 144), f=200.0):
    """Gaussians on the surfaces of a room (back wall, floor, ceiling, side walls,
    four fronto-parallel boxes 5.5-7.5 m ahead; every surface stays a few metres
    from the camera path): small flat discs (in-plane scale
    3 cm, 3 mm along the normal), nearly opaque (opacity logit 4), random
    colours - so rendered images and per-Gaussian feature maps are consistent
    across views, as on real textured surfaces - seen by n_views cameras along
    the standard path (0.3 m and 5 degrees per frame). Returns (Scene, cameras)."""
    rng = _rng(seed)
    # (origin, u axis, v axis): rectangle origin + a u + b v, a, b in [0, 1]
    rects = [((-4.0, -2.2, 9.0), (8.0, 0, 0), (0, 4.0, 0)),     # back wall z = 9
             ((-4.0, 1.6, 0.5), (8.0, 0, 0), (0, 0, 8.5)),      # floor y = 1.6
             ((-4.0, -2.2, 0.5), (8.0, 0, 0), (0, 0, 8.5)),     # ceiling y = -2.2
             ((-3.5, -2.2, 0.5), (0, 3.8, 0), (0, 0, 8.5)),     # left wall x = -3.5
             ((3.5, -2.2, 0.5), (0, 3.8, 0), (0, 0, 8.5))]      # right wall x = 3.5
    for _ in range(4):
        zc, xc, yc = rng.uniform(5.5, 7.5), rng.uniform(-2, 2), rng.uniform(-1, 1)
        hw, hh = rng.uniform(0.3, 1.0), rng.uniform(0.3, 1.0)
        rects.append(((xc - hw, yc - hh, zc), (2 * hw, 0, 0), (0, 2 * hh, 0)))
    area = np.array([np.linalg.norm(np.cross(u, v)) for _, u, v in rects])
    which = rng.choice(len(rects), n, p=area / area.sum())
    ab = rng.random((n, 2))
    mean = np.empty((n, 3))
    quat = np.empty((n, 4))
    for k, (o, u, v) in enumerate(rects):
        m = which == k
        o, u, v = np.asarray(o), np.asarray(u, float), np.asarray(v, float)
        mean[m] = o + ab[m, :1] * u + ab[m, 1:] * v
        nrm = np.cross(u, v)
        nrm /= np.linalg.norm(nrm)
        # rotation taking the z axis to the normal (the disc's thin axis)
        axis = np.cross([0.0, 0.0, 1.0], nrm)
        s, c = np.linalg.norm(axis), nrm[2]
        if s < 1e-9:
            q = np.array([1.0, 0.0, 0.0, 0.0])
        else:
            ang = math.atan2(s, c)
            axis /= s
            q = np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * axis])
        quat[m] = q
    scale = np.zeros((n, 4))
    scale[:, 0] = scale[:, 1] = math.log(0.03)
    scale[:, 2] = math.log(0.003)
    sh = np.zeros((n, 48))
    sh[:, :3] = rng.normal(0, DC_STD, (n, 3))
    mean_opa = np.concatenate([mean, np.full((n, 1), 4.0)], 1)
    sc = Scene(mean_opa.astype(np.float32), scale.astype(np.float32), quat.astype(np.float32),
               sh.astype(np.float32), 0)
    path = camera_path(rng, n_views)
    cams = [camera(*world_to_camera(R, c), f, size[0], size[1]) for R, c in path]
    return sc, cams


def corridor_scene(seed=1009, n=2_000_000, n_views=100, size=(1920, 1080), f=1500.0):
    """The streaming workload at full size: Gaussians on the surfaces of a long
    room built around the standard camera path (0.3 m and 5 degrees per
    frame; drawn first, from its own seed): side walls 3 m beyond the path's
    extent either side, a floor 2 m below and a ceiling 2.5 m above the
    cameras, walls 3 m behind the start and 8 m past the end, plus 40 boxes
    along the side walls - as small flat, nearly opaque discs with random
    colours (as surface_scene). n_views cameras of the given size, fx = fy = f.
    Returns (Scene, cameras)."""
    path = camera_path(_rng(seed + 1), n_views)
    ctr = np.array([c for _, c in path])
    x0, x1 = ctr[:, 0].min() - 3.0, ctr[:, 0].max() + 3.0
    z0, z1 = ctr[:, 2].min() - 3.0, ctr[:, 2].max() + 8.0
    y0, y1 = -2.5, 2.0
    wx, wy, wz = x1 - x0, y1 - y0, z1 - z0
    rng = _rng(seed)
    rects = [((x0, y0, z1), (wx, 0, 0), (0, wy, 0)),   # end wall
             ((x0, y0, z0), (wx, 0, 0), (0, wy, 0)),   # start wall
             ((x0, y1, z0), (wx, 0, 0), (0, 0, wz)),   # floor
             ((x0, y0, z0), (wx, 0, 0), (0, 0, wz)),   # ceiling
             ((x0, y0, z0), (0, wy, 0), (0, 0, wz)),   # left wall
             ((x1, y0, z0), (0, wy, 0), (0, 0, wz))]   # right wall
    for _ in range(40):
        zc = rng.uniform(z0 + 2.0, z1 - 2.0)
        left = rng.random() < 0.5
        xc = (x0 + rng.uniform(0.3, 0.9)) if left else (x1 - rng.uniform(0.3, 0.9))
        yc = rng.uniform(0.0, 1.5)
        hw, hh = rng.uniform(0.2, 0.4), rng.uniform(0.3, 0.5)
        rects.append(((xc - hw, yc - hh, zc), (2 * hw, 0, 0), (0, 2 * hh, 0)))
    area = np.array([np.linalg.norm(np.cross(u, v)) for _, u, v in rects])
    which = rng.choice(len(rects), n, p=area / area.sum())
    ab = rng.random((n, 2))
    mean = np.empty((n, 3))
    quat = np.empty((n, 4))
    for k, (o, u, v) in enumerate(rects):
        m = which == k
        o, u, v = np.asarray(o), np.asarray(u, float), np.asarray(v, float)
        mean[m] = o + ab[m, :1] * u + ab[m, 1:] * v
        nrm = np.cross(u, v)
        nrm /= np.linalg.norm(nrm)
        axis = np.cross([0.0, 0.0, 1.0], nrm)
        s, c = np.linalg.norm(axis), nrm[2]
        if s < 1e-9:
            q = np.array([1.0, 0.0, 0.0, 0.0])
        else:
            ang = math.atan2(s, c)
            axis /= s
            q = np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * axis])
        quat[m] = q
    scale = np.zeros((n, 4))
    scale[:, 0] = scale[:, 1] = math.log(0.03)
    scale[:, 2] = math.log(0.003)
    sh = np.zeros((n, 48))
    sh[:, :3] = rng.normal(0, DC_STD, (n, 3))
    mean_opa = np.concatenate([mean, np.full((n, 1), 4.0)], 1)
    sc = Scene(mean_opa.astype(np.float32), scale.astype(np.float32), quat.astype(np.float32),
               sh.astype(np.float32), 0)
    cams = [camera(*world_to_camera(R, c), f, size[0], size[1]) for R, c in path]
    return sc, cams


def monocular_factor(width, height, seed, sd=0.25, noise=0.02):
    """Multiplicative error of a monocular-style depth estimate: exp(sd x a
    smooth random field + noise x per-pixel N(0, 1)), the field a 4 x 6 grid of
    N(0, 1) values interpolated bilinearly (corners at the image corners).
    Returns float32 [height][width]."""
    rng = _rng(seed)
    coarse = rng.standard_normal((4, 6))
    ys = np.linspace(0, 3, height)
    xs = np.linspace(0, 5, width)
    y0 = np.minimum(np.floor(ys).astype(int), 2)
    x0 = np.minimum(np.floor(xs).astype(int), 4)
    fy = (ys - y0)[:, None]
    fx = (xs - x0)[None, :]
    c00 = coarse[y0][:, x0]
    c01 = coarse[y0][:, x0 + 1]
    c10 = coarse[y0 + 1][:, x0]
    c11 = coarse[y0 + 1][:, x0 + 1]
    field = (c00 * (1 - fx) + c01 * fx) * (1 - fy) + (c10 * (1 - fx) + c11 * fx) * fy
    return np.exp(sd * field + noise * rng.standard_normal((height, width))).astype(np.float32)
