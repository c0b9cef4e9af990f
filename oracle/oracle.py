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
import dataclasses
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
        _lib.or_project.argtypes = [C.c_int64, d, d, d, d, d, d, d, d, d, d, d, f32, i32, i32, u8, u8, u8]
        _lib.or_tile_lists.restype = C.c_int64
        _lib.or_tile_lists.argtypes = [C.c_int64, i32, f32, C.c_int, C.c_int, i64, i32, C.c_int64]
        _lib.or_render_fwd.restype = None
        dn = np.ctypeslib.ndpointer(np.float64, flags="C")
        opt = C.c_void_p  # optional double array
        _lib.or_render_fwd.argtypes = [d, d, i64, i32, d, d, d, d, opt, d, d, i32, u8, u8, i32]
        _lib.or_render_bwd.restype = None
        _lib.or_render_bwd.argtypes = [d, d, i64, i32, d, d, d, d, opt, d, C.c_int64, d, opt, opt]
        _lib.or_project_bwd.restype = None
        _lib.or_project_bwd.argtypes = [C.c_int64, d, d, d, d, d, d, d, d, d, d, d, d, d]
        _lib.or_project_bwd_abs.restype = None
        _lib.or_project_bwd_abs.argtypes = [C.c_int64, d, d, d, d, d, d, d, opt, d, d, d, d, d, d, d]
        _lib.or_pose_jacobian.restype = None
        _lib.or_pose_jacobian.argtypes = [C.c_int64, d, d, d, d, d, d, d]
        _lib.or_render_bwd_bounds.restype = None
        _lib.or_render_bwd_bounds.argtypes = [d, d, i64, i32, d, d, d, d, opt, f32, d, C.c_int64, i64, C.c_int64,
                                              opt, opt, d, d, d, d]
        _lib.or_sh_basis.restype = None
        _lib.or_sh_basis.argtypes = [C.c_int, d, d, d]
        u32 = np.ctypeslib.ndpointer(np.uint32, flags="C")
        _lib.or_philox4x32_10.restype = None
        _lib.or_philox4x32_10.argtypes = [u32, u32, u32]
        _lib.or_philox_uniforms.restype = None
        _lib.or_philox_uniforms.argtypes = [C.c_int64, C.c_uint32, C.c_uint32, C.c_uint64, d]
        _lib.or_log_kernel.restype = C.c_int
        _lib.or_log_kernel.argtypes = [C.c_double, d]
        _lib.or_spawn_maps.restype = None
        _lib.or_spawn_maps.argtypes = [d, opt, C.c_int, C.c_int, C.c_double, C.c_uint64, C.c_uint32, C.c_double,
                                       d, d, d, d, u8, u8]
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
    margin_depth: float = 1e-6
    mip_filter: int = 0
    alpha_rect: int = 1

    def array(self) -> np.ndarray:
        return np.array([self.tile, self.sh_degree, self.near_z, self.dilation, self.alpha_min,
                         self.alpha_max, self.t_min, *self.bg, self.pose_grad_through_sh,
                         self.margin_geo, self.margin_alpha, self.margin_T, self.margin_rect_px,
                         self.margin_depth, self.mip_filter, self.alpha_rect], np.float64)


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
               n_tiles=np.zeros(n, np.int32), clamp=np.zeros(n, np.uint8), amb=np.zeros(n, np.uint8),
               edge_side=np.zeros(n, np.uint8))
    vis = lib().or_project(n, _c(scene.mean_opa, np.float64), _c(scene.scale, np.float64),
                           _c(scene.quat, np.float64), _c(scene.sh, np.float64), cam_array(cam), cfg.array(),
                           out["mean2d"], out["conic"], out["opacity"], out["rgb"], out["depth"],
                           out["depth_key"], out["rect"], out["n_tiles"], out["clamp"], out["amb"],
                           out["edge_side"])
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


def _depth_arg(proj):
    """Depth array (keeps a reference alive) and its address, or (None, None)."""
    if proj.get("depth") is None:
        return None, None
    z = _c(proj["depth"], np.float64)
    return z, z.ctypes.data


def render_fwd(proj, start, ids, cam, cfg: Config) -> dict:
    H, W = cam["height"], cam["width"]
    n = proj["mean2d"].shape[0]
    out = dict(color=np.zeros((3, H, W)), t_final=np.zeros((H, W)), n_contrib=np.zeros((H, W), np.int32),
               amb=np.zeros((H, W), np.uint8), amb_gauss=np.zeros(max(n, 1), np.uint8),
               n_composited=np.zeros((H, W), np.int32))
    z, zp = _depth_arg(proj)
    lib().or_render_fwd(cam_array(cam), cfg.array(), _c(start, np.int64), _c(ids, np.int32),
                        _c(proj["mean2d"], np.float64), _c(proj["conic"], np.float64),
                        _c(proj["opacity"], np.float64), _c(proj["rgb"], np.float64), zp,
                        out["color"], out["t_final"], out["n_contrib"], out["amb"], out["amb_gauss"],
                        out["n_composited"])
    out["amb_gauss"] = out["amb_gauss"][:n]
    return out


def render_depth(proj, start, ids, cam, cfg: Config) -> np.ndarray:
    """Depth integral per pixel, sum_i alpha_i T_i z_i over the composited
    Gaussians (expected depth times 1 - T_final): the compositing of render_fwd
    with every Gaussian's colour replaced by its camera depth and a black
    background (the weights alpha_i T_i do not depend on the colours)."""
    import dataclasses
    p2 = dict(proj)
    p2["rgb"] = np.repeat(np.asarray(proj["depth"], np.float64)[:, None], 3, 1)
    return render_fwd(p2, start, ids, cam, dataclasses.replace(cfg, bg=(0.0, 0.0, 0.0)))["color"][0]


def render_bwd(proj, start, ids, cam, cfg: Config, dL_dcolor, with_amb=False, amb_pixels=None):
    """Returns g2d [n, 9] = dL/d(u, v, conic a, b, c, opacity, r, g, b); with
    with_amb also the [n, 9] bound on contributions from ambiguous pixels
    (those the oracle flags, plus amb_pixels [H, W] when given)."""
    n = proj["mean2d"].shape[0]
    g2d = np.zeros((n, 9))
    amb = np.zeros((n, 9))
    z, zp = _depth_arg(proj)
    extra = None if amb_pixels is None else _c(amb_pixels, np.uint8)
    lib().or_render_bwd(cam_array(cam), cfg.array(), _c(start, np.int64), _c(ids, np.int32),
                        _c(proj["mean2d"], np.float64), _c(proj["conic"], np.float64),
                        _c(proj["opacity"], np.float64), _c(proj["rgb"], np.float64), zp,
                        _c(dL_dcolor, np.float64), n, g2d, amb.ctypes.data if with_amb else None,
                        None if extra is None else extra.ctypes.data)
    return (g2d, amb) if with_amb else g2d


def project_bwd(scene, cam, cfg: Config, g2d) -> dict:
    n = scene.n
    out = dict(mean=np.zeros((n, 3)), logit=np.zeros(n), log_scale=np.zeros((n, 3)), quat=np.zeros((n, 4)),
               sh=np.zeros((n, 48)), pose=np.zeros(6))
    lib().or_project_bwd(n, _c(scene.mean_opa, np.float64), _c(scene.scale, np.float64),
                         _c(scene.quat, np.float64), _c(scene.sh, np.float64), cam_array(cam), cfg.array(),
                         _c(g2d, np.float64), out["mean"], out["logit"], out["log_scale"], out["quat"],
                         out["sh"], out["pose"])
    return out


def project_bwd_abs(scene, cam, cfg: Config, b2d, g2d=None) -> dict:
    """Per-item bounds b2d [n, 9] (>= 0) on the 2D adjoint carried through the
    projection adjoint with absolute Jacobians: the most each parameter
    gradient (mean, logit, log_scale, quat, sh) and the view's pose gradient
    can move. With g2d, pose_absum = sum over items of |pose contribution|."""
    n = scene.n
    out = dict(mean=np.zeros((n, 3)), logit=np.zeros(n), log_scale=np.zeros((n, 3)), quat=np.zeros((n, 4)),
               sh=np.zeros((n, 48)), pose=np.zeros(6), pose_absum=np.zeros(6))
    g = None if g2d is None else _c(g2d, np.float64)
    lib().or_project_bwd_abs(n, _c(scene.mean_opa, np.float64), _c(scene.scale, np.float64),
                             _c(scene.quat, np.float64), _c(scene.sh, np.float64), cam_array(cam), cfg.array(),
                             _c(b2d, np.float64), None if g is None else g.ctypes.data, out["mean"], out["logit"],
                             out["log_scale"], out["quat"], out["sh"], out["pose"], out["pose_absum"])
    return out


def pose_jacobian(scene, cam, cfg: Config) -> np.ndarray:
    """[n, 6, 9]: d(pose gradient of the view) / d(2D adjoint of item i)."""
    n = scene.n
    jac = np.zeros((n, 6, 9))
    lib().or_pose_jacobian(n, _c(scene.mean_opa, np.float64), _c(scene.scale, np.float64),
                           _c(scene.quat, np.float64), _c(scene.sh, np.float64), cam_array(cam), cfg.array(), jac)
    return jac


# ---------------------------------------------------------------------------
# 3-D smoothing filter (Mip-Splatting's 3-D filter; the "proper filtering" of
# Sec. 4.3). The filter adds v I to the 3-D covariance and scales the opacity by
# sqrt(det Sigma / det(Sigma + v I)). With Sigma = R diag(s^2) R^T this is the
# covariance of scales sqrt(s^2 + v) and the factor prod s / sqrt(s^2 + v), so
# the filtered Gaussian is a Gaussian of the unfiltered model with new scales
# and opacity: the oracle renders that one and carries its gradients back.
# ---------------------------------------------------------------------------

def filter3d_variance(scene, cams, near_z=0.2, s2=0.2, margin=1e-6):
    """Per Gaussian v = s2 / nu^2, nu = max over the cameras in which the mean
    is in front of near_z and projects inside the image enlarged by 15% on
    each side of fx / z; Gaussians no camera samples take the largest v of the
    sampled ones (0 if none). Returns (v, ambiguous: a visibility test or the
    maximum within `margin` relative of its threshold)."""
    mu = np.asarray(scene.mean_opa, np.float64)[:, :3]
    n = mu.shape[0]
    nu = np.zeros(n)
    amb = np.zeros(n, bool)
    rates = []
    for c in cams:
        R = np.asarray(c["R"], np.float64).reshape(3, 3)
        t = np.asarray(c["t"], np.float64)
        p = mu @ R.T + t
        z = p[:, 2]
        with np.errstate(divide="ignore", invalid="ignore"):
            u = c["fx"] * p[:, 0] / z + c["cx"]
            w = c["fy"] * p[:, 1] / z + c["cy"]
            W, H = c["width"], c["height"]
            inside = (z > near_z) & (u >= -0.15 * W) & (u <= 1.15 * W) & (w >= -0.15 * H) & (w <= 1.15 * H)
            edge = (np.abs(z - near_z) < margin * near_z) | (np.abs(u + 0.15 * W) < margin * W) | \
                   (np.abs(u - 1.15 * W) < margin * W) | (np.abs(w + 0.15 * H) < margin * H) | \
                   (np.abs(w - 1.15 * H) < margin * H)
            rate = np.where(inside, c["fx"] / z, 0.0)
        amb |= edge & (z > 0)
        rates.append(rate)
    rates = np.array(rates)
    nu = rates.max(axis=0)
    seen = nu > 0
    v = np.zeros(n)
    v[seen] = s2 / nu[seen] ** 2
    if seen.any():
        v[~seen] = v[seen].max()
    # two views with nearly equal rates: FP32 may pick either (values agree to the margin)
    return v, amb


def filtered_scene(scene, v):
    """The scene whose unfiltered Gaussians equal the 3-D-filtered ones: log-scales
    0.5 log(s^2 + v), opacity logit of sigmoid(logit) prod s / sqrt(s^2 + v); FP64."""
    mo = np.array(scene.mean_opa, np.float64)
    ls = np.array(scene.scale, np.float64)
    v = np.asarray(v, np.float64)
    s2 = np.exp(2 * ls[:, :3])
    p2 = s2 + v[:, None]
    f3 = np.prod(np.sqrt(s2 / p2), axis=1)
    o = 1.0 / (1.0 + np.exp(-mo[:, 3]))
    of = o * f3
    mo[:, 3] = np.log(of) - np.log1p(-of)
    ls[:, :3] = 0.5 * np.log(p2)
    return type(scene)(mo, ls, np.asarray(scene.quat, np.float64), np.asarray(scene.sh, np.float64),
                       scene.sh_degree)


def filter3d_chain(scene, v, g, absolute=False):
    """Gradients with respect to the filtered scene's log-scales and logits
    (g["log_scale"] [n, 3], g["logit"] [n]) carried back to the original
    parameters: d log s'_i / d log s_i = s_i^2 / (s_i^2 + v); the filtered logit
    l' = logit(o f3) has dl'/dl = (1 - o) / (1 - o f3) and
    dl'/d log s_i = (v / (s_i^2 + v)) / (1 - o f3). Other keys pass through.
    absolute: the same with |g| (every Jacobian entry is >= 0, so this carries
    bounds)."""
    ls = np.asarray(scene.scale, np.float64)[:, :3]
    lo = np.asarray(scene.mean_opa, np.float64)[:, 3]
    v = np.asarray(v, np.float64)
    s2 = np.exp(2 * ls)
    p2 = s2 + v[:, None]
    f3 = np.prod(np.sqrt(s2 / p2), axis=1)
    o = 1.0 / (1.0 + np.exp(-lo))
    one_m = 1.0 - o * f3
    gs_ = np.abs(g["log_scale"]) if absolute else g["log_scale"]
    gl = np.abs(g["logit"]) if absolute else g["logit"]
    out = dict(g)
    out["log_scale"] = gs_ * (s2 / p2) + (gl / one_m)[:, None] * (v[:, None] / p2)
    out["logit"] = gl * (1.0 - o) / one_m
    return out


def _subset(scene, idx):
    return type(scene)(scene.mean_opa[idx], scene.scale[idx], scene.quat[idx], scene.sh[idx], scene.sh_degree)


def ambiguous_memberships(view: dict, cam, cfg: Config, scene=None):
    """(tile, item, group) triples whose tile-list membership an FP32
    projection may decide the other way. A rect edge within the margin of a
    tile boundary (bits 4/8/16/32 of the projection's flags) may round to the
    other side: the column (row) just outside joins, or the one just inside
    leaves, whichever the oracle's side of the boundary (edge_side) makes the
    other rounding; a radius near an integer allows both. Items that may
    vanish or appear altogether (bit 1): visible ones may leave all their
    tiles; ones the near plane culled (given the scene) are projected with the
    plane moved just past them and may join every tile of that rect (their
    projections are returned in `extra`, item -> (projection, config)); any
    other such item's neighbourhood is returned as a mask [H, W] of pixels
    whose every contribution counts as uncertain. An item with an empty rect
    (culled, but projected) may join the column or row next to a flagged edge.
    The memberships of one edge (or one vanishing or appearing item) share a
    group: they change together. Returns (memb int64 [m, 3] sorted by tile,
    mask uint8 [H, W], extra)."""
    tx, ty = tiles_xy(cam, cfg)
    T = cfg.tile
    W, H = cam["width"], cam["height"]
    proj = view["proj"]
    amb = proj["amb"]
    side = proj.get("edge_side")
    out = []
    bad = np.zeros((ty, tx), bool)
    vis = proj["n_tiles"] > 0
    extra = {}
    group = 0

    def add(tiles, i):
        nonlocal group
        tiles = sorted(set(tiles))
        if tiles:
            out.extend((t, int(i), group) for t in tiles)
            group += 1

    for i in np.nonzero(amb & (1 | 4 | 8 | 16 | 32 | 64))[0]:
        x0, y0, x1, y1 = (int(c) for c in proj["rect"][i])
        a = int(amb[i])
        if a & (1 | 64):
            if vis[i]:
                # may vanish: it may leave all of its tiles
                add([ry * tx + cx for ry in range(y0, y1) for cx in range(x0, x1)], i)
            elif proj["opacity"][i] == 0 and np.all(proj["conic"][i] == 0):
                z = proj["depth"][i]
                if scene is not None and np.isfinite(z) and z <= cfg.near_z:
                    # culled by the near plane within its margin: project it with the plane moved
                    # just past it; it may join every tile of that rect
                    cfg2 = dataclasses.replace(cfg, near_z=float(z) - cfg.margin_geo * max(1.0, abs(float(z))))
                    one = project(_subset(scene, [i]), cam, cfg2)
                    if one["n_tiles"][0] > 0:
                        extra[int(i)] = (one, cfg2)
                        r0, s0, r1, s1 = (int(c) for c in one["rect"][0])
                        add([ry * tx + cx for ry in range(s0, s1) for cx in range(r0, r1)], i)
                    continue
                # culled before its projection otherwise (non-finite): not modelled
                u, v = proj["mean2d"][i]
                if np.isfinite(u) and np.isfinite(v):
                    cx, cy = int(np.clip(u // T, 0, tx - 1)), int(np.clip(v // T, 0, ty - 1))
                    bad[max(cy - 2, 0):cy + 3, max(cx - 2, 0):cx + 3] = True
            continue
        if proj["opacity"][i] == 0 and np.all(proj["conic"][i] == 0):
            continue
        sd = 0x0F | 0xF0 if side is None else int(side[i])
        # edge c: 0 = x0, 1 = y0, 2 = x1, 3 = y1; "down" = the other rounding is one less
        for c, (lo, hi, n_) in enumerate(((x0, x1, tx), (y0, y1, ty), (x0, x1, tx), (y0, y1, ty))):
            if not a & (4 << c):
                continue
            down = bool(sd & (1 << c))
            both = bool(sd & (16 << c))
            lines = []
            if c < 2:  # a lower edge at e: one less -> line e - 1 joins; one more -> line e leaves
                if down or both:
                    lines.append(lo - 1)
                if not down or both:
                    lines.append(lo)
            else:      # an upper edge at e (exclusive): one less -> line e - 1 leaves; one more -> line e joins
                if down or both:
                    lines.append(hi - 1)
                if not down or both:
                    lines.append(hi)
            for ln in lines:
                if not 0 <= ln < n_:
                    continue
                if c in (0, 2):
                    add([ry * tx + ln for ry in range(y0, y1)], i)
                else:
                    add([ln * tx + cx for cx in range(x0, x1)], i)
    memb = np.array(sorted(out), np.int64).reshape(-1, 3)
    mask = np.repeat(np.repeat(bad, T, 0), T, 1)[:H, :W].astype(np.uint8)
    return memb, mask, extra


def adjoint_bounds(scene, view: dict, cam, cfg: Config, dL_dcolor) -> dict:
    """render_bwd_bounds for a whole view with every uncertain membership
    modelled (ambiguous_memberships), the pose Jacobian of the projection
    adjoint, and the near-plane items that may appear projected as they would
    be. Adds the count of such items (near_plane) and of masked pixels."""
    memb, mask, extra = ambiguous_memberships(view, cam, cfg, scene)
    proj = view["proj"]
    jac = pose_jacobian(scene, cam, cfg)
    if extra:
        proj = {k: (np.array(v, copy=True) if isinstance(v, np.ndarray) else v) for k, v in proj.items()}
        for i, (one, cfg2) in extra.items():
            for k in ("mean2d", "conic", "opacity", "rgb", "depth", "depth_key"):
                proj[k][i] = one[k][0]
            jac[i] = pose_jacobian(_subset(scene, [i]), cam, cfg2)[0]
    out = render_bwd_bounds(proj, view["start"], view["ids"], cam, cfg, dL_dcolor, memb, mask, jac)
    out["near_plane"] = len(extra)
    out["masked_pixels"] = int(mask.sum())
    out["memberships"] = int(memb.shape[0])
    return out


def render_bwd_bounds(proj, start, ids, cam, cfg: Config, dL_dcolor, memb=None, amb_pixels=None, jac=None) -> dict:
    """How far an FP32 compositing adjoint may legitimately be from render_bwd
    (gs_oracle.c, or_render_bwd_bounds): flip [n, 9] from decisions within
    their margin and uncertain list memberships, fp32 [n, 9] from the rounding
    of a back-to-front adjoint; with the pose Jacobian, pose_flip [6] and
    pose_fp32 [6] for the view's pose gradient."""
    n = proj["mean2d"].shape[0]
    out = dict(flip=np.zeros((n, 9)), fp32=np.zeros((n, 9)), pose_flip=np.zeros(6), pose_fp32=np.zeros(6))
    z, zp = _depth_arg(proj)
    memb = np.zeros((0, 3), np.int64) if memb is None else _c(memb, np.int64)
    mask = None if amb_pixels is None else _c(amb_pixels, np.uint8)
    j = None if jac is None else _c(jac, np.float64)
    lib().or_render_bwd_bounds(cam_array(cam), cfg.array(), _c(start, np.int64), _c(ids, np.int32),
                               _c(proj["mean2d"], np.float64), _c(proj["conic"], np.float64),
                               _c(proj["opacity"], np.float64), _c(proj["rgb"], np.float64), zp,
                               _c(proj["depth_key"], np.float32), _c(dL_dcolor, np.float64), n,
                               memb if memb.size else np.zeros((1, 3), np.int64), int(memb.shape[0]),
                               None if mask is None else mask.ctypes.data, None if j is None else j.ctypes.data,
                               out["flip"], out["fp32"], out["pose_flip"], out["pose_fp32"])
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


def _alpha_on(proj, i, xs, ys):
    """alpha of item i on the pixel grid xs x ys (pixel centres at +0.5)."""
    u, v = proj["mean2d"][i]
    a, b, c = proj["conic"][i]
    dx = (xs[None, :] + 0.5) - u
    dy = (ys[:, None] + 0.5) - v
    power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
    return np.where(power > 0, 0.0, proj["opacity"][i] * np.exp(np.minimum(power, 0.0)))


def ambiguous_tiles(view: dict, cam, cfg: Config, any_alpha: bool = False) -> np.ndarray:
    """Tiles whose list the FP32 path may legitimately build differently.
    Ambiguity bits of or_project: 1 = near plane / determinant (the Gaussian
    may vanish: its whole rect plus one tile), 64 = opacity within the margin
    of alpha_min (listed or not: only where it reaches alpha_min, i.e. about its
    centre, can that change the image), 4/8/16/32 = rect edge x0/y0/x1/y1
    near a tile boundary: the one tile column (row) that edge adds or drops when
    it rounds the other way (from the side its FP64 value lies on; both columns
    when the radius itself may round either way) may or may not list the
    Gaussian; a tile of it is flagged only if the
    Gaussian reaches alpha_min there (a Gaussian below alpha_min everywhere in
    the tile composites to nothing either way), or, with any_alpha, always (its
    presence still shifts the list positions, e.g. n_contrib)."""
    tx, ty = tiles_xy(cam, cfg)
    T = cfg.tile
    W, H = cam["width"], cam["height"]
    bad = np.zeros((ty, tx), bool)
    proj = view["proj"]
    amb = proj["amb"]
    thr = cfg.alpha_min * (1 - 10 * cfg.margin_alpha)
    for i in np.nonzero(amb & (1 | 4 | 8 | 16 | 32 | 64))[0]:
        x0, y0, x1, y1 = (int(c) for c in proj["rect"][i])
        a = int(amb[i])
        if x1 <= x0 or y1 <= y0 or (a & (1 | 64)):
            # may vanish or appear: its (possible) rect plus a margin
            u, v = proj["mean2d"][i]
            blk = np.zeros_like(bad)
            if x1 > x0 and y1 > y0:
                blk[max(y0 - 1, 0):y1 + 1, max(x0 - 1, 0):x1 + 1] = True
            elif np.isfinite(u) and np.isfinite(v):
                cx, cy = int(np.clip(u // T, 0, tx - 1)), int(np.clip(v // T, 0, ty - 1))
                blk[max(cy - 2, 0):cy + 3, max(cx - 2, 0):cx + 3] = True
            if any_alpha or (a & 1) or not proj["opacity"][i] > 0:
                bad |= blk
            else:
                # a projected item that only an uncertain edge keeps out of every tile changes the
                # image only where it reaches alpha_min (the opacity-aware bounds make such items
                # common: a splat whose alpha_min region is off screen)
                for ry, cx in zip(*np.nonzero(blk)):
                    xs = np.arange(cx * T, min(cx * T + T, W), dtype=np.float64)
                    ys = np.arange(ry * T, min(ry * T + T, H), dtype=np.float64)
                    if xs.size and ys.size and _alpha_on(proj, i, xs, ys).max() >= thr:
                        bad[ry, cx] = True
            continue
        u, v = proj["mean2d"][i]
        r_lo, r_hi = max(y0 - 1, 0), min(y1 + 1, ty)
        c_lo, c_hi = max(x0 - 1, 0), min(x1 + 1, tx)
        # the column (row) an edge toggles follows from the side of the boundary its FP64 value lies
        # on (edge_side bit c): a lower edge at or above it may round down and add the column before
        # x0, else round up and drop column x0; an upper edge at or above it may drop column x1 - 1,
        # else add column x1. A radius near an integer (bit 16 << c) may move the edge either way.
        sd = int(proj["edge_side"][i])

        def toggled(c, lo, hi):
            if sd & (16 << c):
                return [lo - 1, lo] if c < 2 else [hi - 1, hi]
            if c < 2:
                return [lo - 1] if sd & (1 << c) else [lo]
            return [hi - 1] if sd & (1 << c) else [hi]

        cols, rows = [], []
        if a & 4:
            cols += toggled(0, x0, x1)
        if a & 16:
            cols += toggled(2, x0, x1)
        if a & 8:
            rows += toggled(1, y0, y1)
        if a & 32:
            rows += toggled(3, y0, y1)
        cand = set()
        for cx in cols:
            if 0 <= cx < tx:
                cand |= {(ry, cx) for ry in range(r_lo, r_hi)}
        for ry in rows:
            if 0 <= ry < ty:
                cand |= {(ry, cx) for cx in range(c_lo, c_hi)}
        for ry, cx in cand:
            xs = np.arange(cx * T, min(cx * T + T, W), dtype=np.float64)
            ys = np.arange(ry * T, min(ry * T + T, H), dtype=np.float64)
            if xs.size and ys.size and (any_alpha or _alpha_on(proj, i, xs, ys).max() >= thr):
                bad[ry, cx] = True
    return bad


# ---------------------------------------------------------------------------
# Direct spawn sampling (Sec. 4.2, Eq. 1-3 and the expected-NN scale)
# ---------------------------------------------------------------------------

def philox4x32_10(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def philox_uniforms(n, c1, c2, seed):
    u = np.zeros(n)
    lib().or_philox_uniforms(n, c1, c2, int(seed), u)
    return u


def log_kernel(sigma):
    k = np.zeros(25 * 25)
    R = lib().or_log_kernel(sigma, k)
    n = 2 * R + 1
    return k[:n * n].reshape(n, n)


def spawn_maps(image, render, sigma, seed, frame, margin=1e-5):
    """P_L (Eq. 1), P~ (Eq. 2), P_s (Eq. 3), the uniform draws and the mask."""
    image = _c(image, np.float64)
    _, H, W = image.shape
    out = {k: np.zeros((H, W)) for k in ("p_l", "p_pen", "p_s", "u")}
    out["mask"] = np.zeros((H, W), np.uint8)
    out["amb"] = np.zeros((H, W), np.uint8)
    r = None if render is None else _c(render, np.float64)
    lib().or_spawn_maps(image, None if r is None else r.ctypes.data, W, H, sigma, int(seed), int(frame), margin,
                        out["p_l"], out["p_pen"], out["p_s"], out["u"], out["mask"], out["amb"])
    return out


def spawn(image, render, depth, cam, sigma, seed, frame, margin=1e-5):
    """Spawned Gaussians, in pixel order: a pixel spawns iff its draw u < P_s
    and its depth z is positive and finite. Each gets the mean back-projected
    from the pixel centre at depth z, isotropic scale s = z s' / f with
    s' = 1 / (2 sqrt(P_L)) (expected nearest-neighbour distance of a 2-D
    Poisson process of intensity P_L), identity rotation, opacity 0.5 and the
    pixel's colour as its SH DC term (higher bands 0)."""
    m = spawn_maps(image, render, sigma, seed, frame, margin)
    depth = np.asarray(depth, np.float64)
    ok = (m["mask"] > 0) & np.isfinite(depth) & (depth > 0)
    ys, xs = np.nonzero(ok)  # row-major = pixel order
    z = depth[ys, xs]
    pl = m["p_l"][ys, xs]
    s_px = 1.0 / (2.0 * np.sqrt(pl))
    s = z * s_px / cam["fx"]
    pc = np.stack([(xs + 0.5 - cam["cx"]) * z / cam["fx"], (ys + 0.5 - cam["cy"]) * z / cam["fy"], z], 1)
    R = np.asarray(cam["R"], np.float64)
    t = np.asarray(cam["t"], np.float64)
    mu = (pc - t) @ R  # R^T (p - t), row vectors
    c0 = 0.5 / math.sqrt(math.pi)
    rgb = np.asarray(image, np.float64)[:, ys, xs].T
    n = len(xs)
    out = dict(pixel=ys * image.shape[2] + xs, mean=mu, log_scale=np.repeat(np.log(s)[:, None], 3, 1),
               quat=np.tile([1.0, 0, 0, 0], (n, 1)), opacity_logit=np.zeros(n), sh_dc=(rgb - 0.5) / c0,
               scale_px=s_px, maps=m)
    return out


# ---------------------------------------------------------------------------
# Anchor trigger (Sec. 4.4)
# ---------------------------------------------------------------------------

def anchor_sizes(scene, cam):
    """On-screen size in pixels of each Gaussian from a camera: fx S / D with S
    the largest scale and D the distance of the mean to the camera centre."""
    R = np.asarray(cam["R"], np.float64)
    t = np.asarray(cam["t"], np.float64)
    centre = -R.T @ t
    mu = np.asarray(scene.mean_opa, np.float64)[:, :3]
    D = np.linalg.norm(mu - centre, axis=1)
    S = np.exp(np.asarray(scene.scale, np.float64)[:, :3].max(axis=1))
    return cam["fx"] * S / D


def anchor_check(scene, cam, tau_px=1.0, share=0.4, margin=1e-5):
    """Too-fine flags (size < tau), their count, whether an anchor is due (more
    than `share` of the active set too fine) and the items within margin."""
    size = anchor_sizes(scene, cam)
    fine = size < tau_px
    amb = np.abs(size - tau_px) < margin * tau_px
    return dict(size=size, too_fine=fine, count=int(fine.sum()), due=bool(fine.sum() > share * len(size)), amb=amb)


def quat_to_rot(q):
    """Rotation matrix of a (not necessarily unit) quaternion (w, x, y, z)."""
    w, x, y, z = np.asarray(q, np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def covariance(log_scale, quat):
    """Sigma = R diag(exp(2 s)) R^T."""
    R = quat_to_rot(quat)
    return R @ np.diag(np.exp(2.0 * np.asarray(log_scale, np.float64)[:3])) @ R.T


def merge_group(mean_opa, scale, quat, sh):
    """Moment-matching merge of a group of Gaussians (rows of the inputs) into
    one (Sec. 4.4, following the hierarchical merge): weights w_i = o_i a_i with
    a_i the product of the two largest scales (the area of the Gaussian's
    largest cross-section up to pi); mean and covariance are the w-weighted mean
    and second moment about it, SH the w-weighted mean, and the opacity keeps
    the total o a: o = min(0.99, sum_i w_i / a) with a the product of the merged
    Gaussian's two largest scales. Returns (mean, covariance, opacity, sh)."""
    mo = np.asarray(mean_opa, np.float64)
    o = 1.0 / (1.0 + np.exp(-mo[:, 3]))
    s = np.exp(np.asarray(scale, np.float64)[:, :3])
    ss = np.sort(s, axis=1)
    w = o * ss[:, 1] * ss[:, 2]
    W = w.sum()
    mu = (w[:, None] * mo[:, :3]).sum(0) / W
    cov = np.zeros((3, 3))
    for i in range(len(w)):
        d = mo[i, :3] - mu
        cov += w[i] * (covariance(scale[i], quat[i]) + np.outer(d, d))
    cov /= W
    lam = np.sort(np.linalg.eigvalsh(cov))
    a = math.sqrt(lam[1] * lam[2])
    return mu, cov, min(0.99, W / a), (w[:, None] * np.asarray(sh, np.float64)).sum(0) / W


def anchor_merge(scene, too_fine, seed, radius, k=3, margin=1e-5):
    """Merging at an anchor (Sec. 4.4). Gaussian i is selected iff it is too
    fine and u_i < 1/(k+1), u_i the Philox draw of counter (i, 0, 2, 0). Every
    selected Gaussian proposes the k nearest (Euclidean distance of the means,
    ties by index, at most `radius` away) too-fine Gaussians that are not
    selected; a Gaussian proposed by several goes to the lowest selected index.
    Each selected Gaussian and the candidates it claimed merge (merge_group);
    claimed Gaussians leave the set; all others are kept unchanged. The output
    keeps index order (a merged Gaussian takes its selected Gaussian's place).
    Returns dict(kind = per output row 0 kept / 1 merged, src = input index,
    mean, cov, opacity, sh for merged rows, selected, claim, amb = selected
    Gaussians whose neighbour decision lies within margin (relative) of the
    radius or of the k-th/(k+1)-th distance tie)."""
    mo = np.asarray(scene.mean_opa, np.float64)
    n = mo.shape[0]
    fine = np.asarray(too_fine, bool)
    u = philox_uniforms(n, 0, 2, seed)
    sel = fine & (u < 1.0 / (k + 1))
    cand = np.nonzero(fine & ~sel)[0]
    claim = np.full(n, -1, np.int64)
    props = {}
    amb = np.zeros(n, bool)
    P = mo[cand, :3]
    for s_ in np.nonzero(sel)[0]:
        d = np.sqrt(((P - mo[s_, :3]) ** 2).sum(1)) if cand.size else np.zeros(0)
        inside = d <= radius
        order = np.lexsort((cand[inside], d[inside]))
        chosen = cand[inside][order][:k]
        props[s_] = chosen
        near = np.abs(d - radius) < margin * radius
        ds = np.sort(d[inside])
        if near.any() or (ds.size > k and ds[k] - ds[k - 1] < margin * max(ds[k], 1e-30)):
            amb[s_] = True
        for c in chosen:
            if claim[c] < 0 or s_ < claim[c]:
                claim[c] = s_
    kind, src, means, covs, opas, shs = [], [], [], [], [], []
    for i in range(n):
        if claim[i] >= 0:
            continue
        src.append(i)
        if sel[i]:
            grp = [i] + [c for c in props[i] if claim[c] == i]
            mu, cov, op, sh = merge_group(mo[grp], np.asarray(scene.scale)[grp], np.asarray(scene.quat)[grp],
                                          np.asarray(scene.sh)[grp])
            kind.append(1)
            means.append(mu); covs.append(cov); opas.append(op); shs.append(sh)
        else:
            kind.append(0)
            means.append(mo[i, :3]); covs.append(covariance(scene.scale[i], scene.quat[i]))
            opas.append(1.0 / (1.0 + math.exp(-mo[i, 3]))); shs.append(np.asarray(scene.sh[i], np.float64))
    return dict(kind=np.array(kind), src=np.array(src), mean=np.array(means).reshape(-1, 3),
                cov=np.array(covs).reshape(-1, 3, 3), opacity=np.array(opas), sh=np.array(shs).reshape(-1, 48),
                selected=sel, claim=claim, amb=amb)


def cull_opacity(mean_opa, min_opacity, margin=1e-6):
    """Opacity culling (Sec. 4.3, as in 3DGS): the Gaussians whose opacity
    sigmoid(logit) is at least min_opacity are kept, in index order. Returns
    (kept indices, ambiguous: opacity within margin (relative) of the bound)."""
    o = 1.0 / (1.0 + np.exp(-np.asarray(mean_opa, np.float64)[:, 3]))
    return np.nonzero(o >= min_opacity)[0], np.abs(o - min_opacity) < margin * min_opacity


def anchor_blend_weight(d1, d2, overlap=0.1):
    """Blending weight of the closest anchor (Sec. 4.4): r = d1 / d2 (d1 <= d2);
    1 for r < 1 - o, else 1 - (r - (1 - o)) * 0.5 / o (0.5 at r = 1)."""
    r = d1 / d2
    return 1.0 if r < 1.0 - overlap else 1.0 - (r - (1.0 - overlap)) * 0.5 / overlap


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


def downsample(image, factor):
    """Coarse-to-fine training image (Sec. 4.3, 2^l downsampling): output pixel
    (I, J) of [3][ceil(H/f)][ceil(W/f)] is the mean of the input pixels of the
    f x f block it covers (a partial block at a ragged edge averages the pixels
    it has)."""
    image = np.asarray(image, np.float64)
    _, H, W = image.shape
    h, w = -(-H // factor), -(-W // factor)
    out = np.zeros((3, h, w))
    for I in range(h):
        for J in range(w):
            out[:, I, J] = image[:, I * factor:(I + 1) * factor, J * factor:(J + 1) * factor].mean(axis=(1, 2))
    return out


def downsample_camera(cam, factor):
    """The camera of a 2^l-downsampled image: intrinsics divided by the factor,
    size rounded up (pixel centres stay at I + 0.5)."""
    c = dict(cam)
    for k in ("fx", "fy", "cx", "cy"):
        c[k] = cam[k] / factor
    c["width"], c["height"] = -(-cam["width"] // factor), -(-cam["height"] // factor)
    return c


def lr_decay(lr_scale, mask, decay):
    """Per-Gaussian learning-rate multipliers (App. A.3: learning rates are set
    when a Gaussian is introduced and multiplied by the decay ratio every time
    the sparse Adam step processes it): the rows in mask are multiplied by decay.
    adam_step takes lr as the per-row product of the group rate and this
    multiplier."""
    s = np.array(lr_scale, np.float64)
    s[np.asarray(mask, bool)] *= decay
    return s


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


def se3_ad(xi):
    """ad(xi) of xi = (rho, phi) in se(3), acting on (rho, phi): [[phi^, rho^], [0, phi^]]."""
    rho, phi = np.asarray(xi[:3], np.float64), np.asarray(xi[3:], np.float64)
    A = np.zeros((6, 6))
    A[:3, :3] = hat(phi)
    A[:3, 3:] = hat(rho)
    A[3:, 3:] = hat(phi)
    return A


def se3_left_jacobian(xi, terms=40):
    """Left Jacobian of SE(3) by its series, J_l = sum_n ad(xi)^n / (n+1)!:
    exp((xi + d)^) = exp((J_l d)^) exp(xi^) to first order in d."""
    A = se3_ad(xi)
    J = np.zeros((6, 6))
    P = np.eye(6)
    fact = 1.0
    for n in range(terms):
        fact *= n + 1
        J += P / fact
        P = P @ A
    return J


def pose_tangent_grad(xi, g_delta):
    """Gradient with respect to xi of a loss of the pose exp(xi^) T_ref, given
    g_delta = dL/d delta of the same loss under T <- exp(delta^) T at
    T = exp(xi^) T_ref (the gradient the rasteriser's backward returns):
    J_l(xi)^T g_delta (Sec. 4.3 pose update written on the SE(3) tangent)."""
    return se3_left_jacobian(xi).T @ np.asarray(g_delta, np.float64)
