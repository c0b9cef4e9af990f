"""Python face of the FP64 oracle: ctypes calls into gs_oracle.c plus the few
steps that are plain NumPy FP64 (Adam, the L1 loss gradient, the SE(3) pose
retraction, multi-view sums).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg, never by the product path. It imports nothing
from the CUDA package; its inputs are the seeded arrays of the input
generator module.

Each function states the step of the method it follows (the paper builds its
joint optimisation, Sec. 4.3, on the 3DGS rasterizer, Sec. 5). Where the paper
is silent the reading is the one documented at the top of gs_oracle.c.
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        d, i64, i32, f32, u8 = (np.ctypeslib.ndpointer(np.float64, flags="C"),
                                np.ctypeslib.ndpointer(np.int64, flags="C"),
                                np.ctypeslib.ndpointer(np.int32, flags="C"),
                                np.ctypeslib.ndpointer(np.float32, flags="C"),
                                np.ctypeslib.ndpointer(np.uint8, flags="C"))
        _lib.or_project.restype = C.c_int64
        _lib.or_project.argtypes = [C.c_int64, d, d, d, d, d, d, d, d, d, d, d, f32, i32, i32, u8, u8]
        _lib.or_tile_lists.restype = C.c_int64
        _lib.or_tile_lists.argtypes = [C.c_int64, i32, f32, C.c_int, C.c_int, i64, i32, C.c_int64]
        _lib.or_render_fwd.restype = None
        _lib.or_render_fwd.argtypes = [d, d, i64, i32, d, d, d, d, d, d, i32, u8]
        _lib.or_render_bwd.restype = None
        _lib.or_render_bwd.argtypes = [d, d, i64, i32, d, d, d, d, d, C.c_int64, d]
        _lib.or_project_bwd.restype = None
        _lib.or_project_bwd.argtypes = [C.c_int64, d, d, d, d, d, d, d, d, d, d, d, d, d]
        _lib.or_sh_basis.restype = None
        _lib.or_sh_basis.argtypes = [C.c_int, d, d, d]
    return _lib


@dataclass
class Config:
    tile: int = 16
    sh_degree: int = 3
    near_z: float = 0.2
    dilation: float = 0.3
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    bg: tuple = (0.0, 0.0, 0.0)
    pose_grad_through_sh: int = 0
    margin_geo: float = 1e-5
    margin_alpha: float = 1e-5
    margin_T: float = 1e-4
    margin_rect_px: float = 2e-3

    def array(self) -> np.ndarray:
        return np.array([self.tile, self.sh_degree, self.near_z, self.dilation, self.alpha_min,
                         self.alpha_max, self.t_min, *self.bg, self.pose_grad_through_sh,
                         self.margin_geo, self.margin_alpha, self.margin_T, self.margin_rect_px, 0], np.float64)


def cam_array(cam: dict) -> np.ndarray:
    return np.array([*np.asarray(cam["R"], np.float64).reshape(9), *np.asarray(cam["t"], np.float64).reshape(3),
                     cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["width"], cam["height"]], np.float64)


def tiles_xy(cam, cfg: Config):
    T = cfg.tile
    return (cam["width"] + T - 1) // T, (cam["height"] + T - 1) // T


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ---------------------------------------------------------------------------
# Projection (EWA + SH), one view
# ---------------------------------------------------------------------------

def project(scene, cam, cfg: Config) -> dict:
    n = scene.n
    out = dict(mean2d=np.zeros((n, 2)), conic=np.zeros((n, 3)), opacity=np.zeros(n), rgb=np.zeros((n, 3)),
               depth=np.zeros(n), depth_key=np.zeros(n, np.float32), rect=np.zeros((n, 4), np.int32),
               n_tiles=np.zeros(n, np.int32), clamp=np.zeros(n, np.uint8), amb=np.zeros(n, np.uint8))
    vis = lib().or_project(n, _c(scene.mean_opa, np.float64), _c(scene.scale, np.float64),
                           _c(scene.quat, np.float64), _c(scene.sh, np.float64), cam_array(cam), cfg.array(),
                           out["mean2d"], out["conic"], out["opacity"], out["rgb"], out["depth"],
                           out["depth_key"], out["rect"], out["n_tiles"], out["clamp"], out["amb"])
    out["n_visible"] = int(vis)
    return out


def tile_lists(rect, depth_key, tiles_x, tiles_y):
    """Per tile, the ids whose rect holds the tile, ordered by (fp32 depth bits, id)."""
    rect = _c(rect, np.int32)
    depth_key = _c(depth_key, np.float32)
    n = rect.shape[0]
    start = np.zeros(tiles_x * tiles_y + 1, np.int64)
    total = lib().or_tile_lists(n, rect, depth_key, tiles_x, tiles_y, start, np.zeros(1, np.int32), 0)
    ids = np.zeros(max(total, 1), np.int32)
    lib().or_tile_lists(n, rect, depth_key, tiles_x, tiles_y, start, ids, total)
    return start, ids[:total]


def render_fwd(proj, start, ids, cam, cfg: Config) -> dict:
    H, W = cam["height"], cam["width"]
    out = dict(color=np.zeros((3, H, W)), t_final=np.zeros((H, W)), n_contrib=np.zeros((H, W), np.int32),
               amb=np.zeros((H, W), np.uint8))
    lib().or_render_fwd(cam_array(cam), cfg.array(), _c(start, np.int64), _c(ids, np.int32),
                        _c(proj["mean2d"], np.float64), _c(proj["conic"], np.float64),
                        _c(proj["opacity"], np.float64), _c(proj["rgb"], np.float64),
                        out["color"], out["t_final"], out["n_contrib"], out["amb"])
    return out


def render_bwd(proj, start, ids, cam, cfg: Config, dL_dcolor) -> np.ndarray:
    """Returns g2d [n, 9] = dL/d(u, v, conic a, b, c, opacity, r, g, b)."""
    n = proj["mean2d"].shape[0]
    g2d = np.zeros((n, 9))
    lib().or_render_bwd(cam_array(cam), cfg.array(), _c(start, np.int64), _c(ids, np.int32),
                        _c(proj["mean2d"], np.float64), _c(proj["conic"], np.float64),
                        _c(proj["opacity"], np.float64), _c(proj["rgb"], np.float64),
                        _c(dL_dcolor, np.float64), n, g2d)
    return g2d


def project_bwd(scene, cam, cfg: Config, g2d) -> dict:
    n = scene.n
    out = dict(mean=np.zeros((n, 3)), logit=np.zeros(n), log_scale=np.zeros((n, 3)), quat=np.zeros((n, 4)),
               sh=np.zeros((n, 48)), pose=np.zeros(6))
    lib().or_project_bwd(n, _c(scene.mean_opa, np.float64), _c(scene.scale, np.float64),
                         _c(scene.quat, np.float64), _c(scene.sh, np.float64), cam_array(cam), cfg.array(),
                         _c(g2d, np.float64), out["mean"], out["logit"], out["log_scale"], out["quat"],
                         out["sh"], out["pose"])
    return out


def sh_basis(degree, d):
    Y = np.zeros(16)
    dY = np.zeros(48)
    lib().or_sh_basis(degree, _c(d, np.float64), Y, dY)
    return Y, dY.reshape(16, 3)


# ---------------------------------------------------------------------------
# Whole views
# ---------------------------------------------------------------------------

def render_view(scene, cam, cfg: Config) -> dict:
    proj = project(scene, cam, cfg)
    tx, ty = tiles_xy(cam, cfg)
    start, ids = tile_lists(proj["rect"], proj["depth_key"], tx, ty)
    img = render_fwd(proj, start, ids, cam, cfg)
    return dict(proj=proj, start=start, ids=ids, **img)


def backward_view(scene, cam, cfg: Config, view: dict, dL_dcolor) -> dict:
    g2d = render_bwd(view["proj"], view["start"], view["ids"], cam, cfg, dL_dcolor)
    out = project_bwd(scene, cam, cfg, g2d)
    out["g2d"] = g2d
    return out


def backward_views(scene, cams, cfg, views, dL_dcolors) -> dict:
    """Parameter gradients summed over views (the joint loss is a sum over views);
    the pose gradient is per view."""
    tot = None
    poses = []
    for cam, v, g in zip(cams, views, dL_dcolors):
        b = backward_view(scene, cam, cfg, v, g)
        poses.append(b["pose"])
        if tot is None:
            tot = {k: b[k].copy() for k in ("mean", "logit", "log_scale", "quat", "sh")}
        else:
            for k in tot:
                tot[k] += b[k]
    tot["pose"] = np.stack(poses)
    return tot


def ambiguous_tiles(view: dict, cam, cfg: Config) -> np.ndarray:
    """Tiles whose list or pixels the FP32 path may legitimately compute
    differently: tiles holding an ambiguous pixel, tiles within one tile of an
    ambiguous Gaussian's rect, and tiles whose list holds two consecutive
    Gaussians with depths equal to within margin_geo (relative)."""
    tx, ty = tiles_xy(cam, cfg)
    T = cfg.tile
    bad = np.zeros((ty, tx), bool)
    H, W = cam["height"], cam["width"]
    amb_px = view["amb"]
    pad = np.zeros((ty * T, tx * T), bool)
    pad[:H, :W] = amb_px > 0
    bad |= pad.reshape(ty, T, tx, T).any(axis=(1, 3))
    proj = view["proj"]
    for i in np.nonzero(proj["amb"] & 1)[0]:
        r = proj["rect"][i]
        if r[2] > r[0] and r[3] > r[1]:
            bad[max(r[1] - 1, 0):r[3] + 1, max(r[0] - 1, 0):r[2] + 1] = True
        else:
            # culled here but may survive in FP32: mark the neighbourhood of its centre
            u, v = proj["mean2d"][i]
            if np.isfinite(u) and np.isfinite(v) and proj["depth"][i] > 0:
                cx, cy = int(np.clip(u // T, 0, tx - 1)), int(np.clip(v // T, 0, ty - 1))
                bad[max(cy - 2, 0):cy + 3, max(cx - 2, 0):cx + 3] = True
    start, ids = view["start"], view["ids"]
    z = proj["depth"]
    for t in range(tx * ty):
        seg = ids[start[t]:start[t + 1]]
        if len(seg) > 1:
            zz = z[seg]
            if np.any(np.abs(np.diff(zz)) <= cfg.margin_geo * np.abs(zz[1:])):
                bad[t // tx, t % tx] = True
    return bad


# ---------------------------------------------------------------------------
# Loss, optimiser and pose update (FP64 NumPy)
# ---------------------------------------------------------------------------

def l1_loss_grad(color, target):
    """L = mean |C - C*| over all pixels and channels; dL/dC = sign(C - C*) / n
    (sign(0) = 0)."""
    diff = np.asarray(color, np.float64) - np.asarray(target, np.float64)
    n = diff.size
    return float(np.abs(diff).sum() / n), np.sign(diff) / n


def adam_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-15, mask=None):
    """Adam (Kingma & Ba) with bias correction; rows where mask is False keep
    their parameters and moments (sparse Adam over visible Gaussians, Sec. 4.3)."""
    p = np.array(p, np.float64)
    m = np.array(m, np.float64)
    v = np.array(v, np.float64)
    g = np.asarray(g, np.float64)
    m2 = beta1 * m + (1 - beta1) * g
    v2 = beta2 * v + (1 - beta2) * g * g
    mh = m2 / (1 - beta1 ** step)
    vh = v2 / (1 - beta2 ** step)
    p2 = p - lr * mh / (np.sqrt(vh) + eps)
    if mask is not None:
        keep = ~np.asarray(mask, bool)
        p2[keep] = p[keep]
        m2[keep] = m[keep]
        v2[keep] = v[keep]
    return p2, m2, v2


def hat(w):
    return np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]], np.float64)


def se3_exp(xi):
    """exp of xi = (rho, phi) in se(3) as (R, t) (closed form, Rodrigues)."""
    rho, phi = np.asarray(xi[:3], np.float64), np.asarray(xi[3:], np.float64)
    th = float(np.linalg.norm(phi))
    K = hat(phi)
    if th < 1e-12:
        R = np.eye(3) + K
        V = np.eye(3) + 0.5 * K
    else:
        R = np.eye(3) + math.sin(th) / th * K + (1 - math.cos(th)) / th ** 2 * K @ K
        V = np.eye(3) + (1 - math.cos(th)) / th ** 2 * K + (th - math.sin(th)) / th ** 3 * K @ K
    return R, V @ rho


def retract_pose(R, t, xi):
    """T_cw <- exp(xi^) T_cw."""
    dR, dt = se3_exp(xi)
    return dR @ np.asarray(R, np.float64), dR @ np.asarray(t, np.float64) + dt


def perturbed_cam(cam, xi):
    R, t = retract_pose(cam["R"], cam["t"], xi)
    c = dict(cam)
    c["R"], c["t"] = R, t
    return c
