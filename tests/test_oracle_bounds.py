"""Pins of the oracle's tolerance machinery: the bounds that say how far an
FP32 evaluation of the compositing adjoint may legitimately sit from the FP64
adjoint (decisions within their margin taking the other branch, uncertain
tile-list memberships, rounding), and their propagation through the
projection adjoint to the parameter and pose gradients.

Each bound is pinned to something computed another way: the flip bound to the
adjoint recomputed with the threshold (or the tile list) moved across the
decision, the propagation to brute force over every sign pattern of the 2D
adjoint, the pose Jacobian to the pose gradient of the projection adjoint
(itself pinned by finite differences in test_oracle_pins.py).

CPU only. Each test names the mistake it would catch.
"""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_2506_05558_gb300 import synth

TIGHT = dict(margin_geo=1e-12, margin_alpha=1e-12, margin_T=1e-12, margin_rect_px=1e-12, margin_depth=1e-15)


def _scene(sh_degree=3, seed=21, n=40, size=48):
    sc, cam, rng = synth.tiny_scene(seed=seed, n=n, width=size, height=size, f=60.0, sh_degree=sh_degree)
    sc = synth.Scene(sc.mean_opa.astype(np.float64), sc.scale.astype(np.float64), sc.quat.astype(np.float64),
                     sc.sh.astype(np.float64), sh_degree)
    sc.scale[:, :3] += 0.5
    if sh_degree > 0:
        sc.sh[:, 3:3 * (sh_degree + 1) ** 2] = rng.normal(0, 0.2, (n, 3 * (sh_degree + 1) ** 2 - 3))
    R, t = O.retract_pose(np.eye(3), np.zeros(3), [0.05, -0.03, 0.02, 0.02, -0.03, 0.01])
    return sc, dict(cam, R=R, t=t), rng


PARAMS = ("mean", "logit", "log_scale", "quat", "sh")


@pytest.mark.parametrize("through_sh,mip", [(0, 0), (1, 0), (0, 1)])
def test_bound_propagation_is_the_exact_worst_case(through_sh, mip):
    """project_bwd_abs(b) per item equals the largest |gradient| over all 2^9
    sign patterns of a 2D adjoint with entries +-b (the adjoint is linear), and
    no perturbation inside the box exceeds it: catches a signed (cancelling)
    propagation, a dropped Jacobian column or a missing pose term."""
    cfg = O.Config(sh_degree=3, pose_grad_through_sh=through_sh, mip_filter=mip, dilation=0.1 if mip else 0.3)
    sc, cam, rng = _scene()
    vis = np.nonzero(O.project(sc, cam, cfg)["n_tiles"] > 0)[0]
    assert vis.size > 10
    b2d = rng.uniform(0.1, 1.0, (sc.n, 9))
    for i in vis[:4]:
        bi = np.zeros_like(b2d)
        bi[i] = b2d[i]
        bound = O.project_bwd_abs(sc, cam, cfg, bi)
        worst = {k: 0.0 for k in PARAMS + ("pose",)}
        for signs in itertools.product((-1.0, 1.0), repeat=9):
            g = np.zeros_like(b2d)
            g[i] = np.array(signs) * b2d[i]
            out = O.project_bwd(sc, cam, cfg, g)
            for k in PARAMS:
                worst[k] = np.maximum(worst[k], np.abs(out[k][i]))
            worst["pose"] = np.maximum(worst["pose"], np.abs(out["pose"]))
        for k in PARAMS:
            np.testing.assert_allclose(bound[k][i], worst[k], rtol=1e-12, atol=1e-300, err_msg=k)
        np.testing.assert_allclose(bound["pose"], worst["pose"], rtol=1e-12, atol=1e-300)
    # random perturbations of every item inside the box stay inside the bound
    full = O.project_bwd_abs(sc, cam, cfg, b2d)
    g0 = rng.standard_normal((sc.n, 9))
    base = O.project_bwd(sc, cam, cfg, g0)
    for _ in range(5):
        d = O.project_bwd(sc, cam, cfg, g0 + rng.uniform(-1, 1, b2d.shape) * b2d)
        for k in PARAMS + ("pose",):
            assert np.all(np.abs(d[k] - base[k]) <= full[k] * (1 + 1e-12) + 1e-300), k


def test_pose_jacobian_reproduces_the_pose_gradient():
    """sum_i J_i g2d_i equals project_bwd's pose gradient for any 2D adjoint:
    catches a transposed (6 x 9) layout or a missing item."""
    for through_sh in (0, 1):
        cfg = O.Config(sh_degree=3, pose_grad_through_sh=through_sh)
        sc, cam, rng = _scene(seed=22)
        jac = O.pose_jacobian(sc, cam, cfg)
        g = rng.standard_normal((sc.n, 9))
        pose = np.einsum("icq,iq->c", jac, g)
        np.testing.assert_allclose(pose, O.project_bwd(sc, cam, cfg, g)["pose"], rtol=1e-11, atol=1e-12)


def _view(sc, cam, cfg):
    view = O.render_view(sc, cam, cfg)
    return view, view["proj"]


def test_flip_bound_equals_the_adjoint_across_the_threshold():
    """alpha_min placed a hair above one Gaussian's alpha at one pixel: the
    oracle skips it there and flags the decision. The flip bound must equal
    |adjoint with alpha_min a hair below - adjoint with it above| for every
    item (the Gaussian itself and those behind it), and the pose bound the
    change of the pose gradient: catches a flip applied to the wrong entry,
    a lost transmittance effect on later Gaussians, or a wrong sign of the
    forced branch."""
    sc, cam, rng = _scene(sh_degree=0, seed=23, n=30, size=32)
    base = O.Config(sh_degree=0, **TIGHT)
    view, proj = _view(sc, cam, base)
    H, W = cam["height"], cam["width"]
    # a Gaussian whose alpha at a pixel is a few times alpha_min (composited there by default)
    pick = None
    for i in np.nonzero(proj["n_tiles"] > 0)[0]:
        al = O._alpha_on(proj, i, np.arange(W, dtype=float), np.arange(H, dtype=float))
        ys, xs = np.nonzero((al > 0.02) & (al < 0.2))
        if ys.size:
            pick = (i, ys[0], xs[0], al[ys[0], xs[0]])
            break
    assert pick is not None
    i, y, x, a = pick
    dL = rng.standard_normal((3, H, W))
    cfg_hi = O.Config(sh_degree=0, alpha_min=a * (1 + 1e-9), **TIGHT)
    cfg_lo = O.Config(sh_degree=0, alpha_min=a * (1 - 1e-9), **TIGHT)
    v_hi, _ = _view(sc, cam, cfg_hi)
    v_lo, _ = _view(sc, cam, cfg_lo)
    assert v_hi["n_contrib"][y, x] != v_lo["n_contrib"][y, x] or not np.array_equal(v_hi["color"], v_lo["color"])
    g_hi = O.render_bwd(proj, v_hi["start"], v_hi["ids"], cam, cfg_hi, dL)
    g_lo = O.render_bwd(proj, v_lo["start"], v_lo["ids"], cam, cfg_lo, dL)
    jac = O.pose_jacobian(sc, cam, cfg_hi)
    bb = O.render_bwd_bounds(proj, v_hi["start"], v_hi["ids"], cam, cfg_hi, dL, jac=jac)
    diff = np.abs(g_lo - g_hi)
    assert diff[i].max() > 0
    scale = np.abs(g_hi).max()
    np.testing.assert_allclose(bb["flip"], diff, rtol=1e-9, atol=1e-12 * scale)
    dpose = np.abs(np.einsum("icq,iq->c", jac, g_lo - g_hi))
    np.testing.assert_allclose(bb["pose_flip"], dpose, rtol=1e-9, atol=1e-12 * np.abs(dpose).max())
    # the same flip from above: alpha_min a hair below (composited, flagged, forced out)
    bb_lo = O.render_bwd_bounds(proj, v_lo["start"], v_lo["ids"], cam, cfg_lo, dL)
    np.testing.assert_allclose(bb_lo["flip"], diff, rtol=1e-9, atol=1e-12 * scale)


@pytest.mark.parametrize("direction", ["join", "leave"])
def test_membership_bound_equals_the_adjoint_with_the_tile_toggled(direction):
    """A Gaussian whose rect is one tile high gains (or loses) the tile just
    right of (at) its right edge: the membership bound for that (tile, item)
    must equal |adjoint with the modified lists - adjoint with the oracle's|
    for every item, the joining Gaussian being inserted at its (depth key, id)
    place: catches an insertion at the wrong depth, a change not summed over
    the tile, or a missing pose term."""
    cfg = O.Config(sh_degree=0, **TIGHT)
    T = cfg.tile

    def reach(proj, rect, i, W, H):  # largest alpha of item i in the tile that changes
        x1, y0 = int(rect[i, 2]), int(rect[i, 1])
        c = x1 if direction == "join" else x1 - 1
        xs = np.arange(c * T, min(c * T + T, W), dtype=float)
        ys = np.arange(y0 * T, min(y0 * T + T, H), dtype=float)
        return O._alpha_on(proj, i, xs, ys).max() if xs.size else 0.0

    # first seeded scene with a one-tile-high Gaussian that reaches alpha_min in the tile that changes
    for seed in range(24, 60):
        sc, cam, rng = _scene(sh_degree=0, seed=seed, n=120, size=64)
        view, proj = _view(sc, cam, cfg)
        tx, ty = O.tiles_xy(cam, cfg)
        H, W = cam["height"], cam["width"]
        rect = proj["rect"].copy()
        cand = [i for i in np.nonzero(proj["n_tiles"] > 0)[0]
                if rect[i, 3] - rect[i, 1] == 1
                and (rect[i, 2] < tx if direction == "join" else rect[i, 2] - rect[i, 0] >= 2)
                and reach(proj, rect, i, W, H) > 1.5 * cfg.alpha_min]
        if cand:
            break
    assert cand
    i = cand[0]
    x0, y0, x1, y1 = rect[i]
    if direction == "join":
        rect[i, 2] = x1 + 1
        tile = y0 * tx + x1
    else:
        rect[i, 2] = x1 - 1
        tile = y0 * tx + x1 - 1
    start2, ids2 = O.tile_lists(rect, proj["depth_key"], tx, ty)
    dL = rng.standard_normal((3, H, W))
    g0 = O.render_bwd(proj, view["start"], view["ids"], cam, cfg, dL)
    g1 = O.render_bwd(proj, start2, ids2, cam, cfg, dL)
    jac = O.pose_jacobian(sc, cam, cfg)
    memb = np.array([[tile, i, 0]], np.int64)
    bb = O.render_bwd_bounds(proj, view["start"], view["ids"], cam, cfg, dL, memb=memb, jac=jac)
    # per-pixel decisions within the FP32 exponent uncertainty are flagged either way: the membership's own
    # share is what it adds to the bound without it
    bb0 = O.render_bwd_bounds(proj, view["start"], view["ids"], cam, cfg, dL, jac=jac)
    diff = np.abs(g1 - g0)
    assert diff[i].max() > 0
    scale = np.abs(g0).max()
    np.testing.assert_allclose(bb["flip"] - bb0["flip"], diff, rtol=1e-9, atol=1e-12 * scale)
    dpose = np.abs(np.einsum("icq,iq->c", jac, g1 - g0))
    np.testing.assert_allclose(bb["pose_flip"] - bb0["pose_flip"], dpose, rtol=1e-9, atol=1e-12 * np.abs(dpose).max())


def test_rounding_bound_properties():
    """The rounding bound is non-negative, zero for a zero adjoint input and of
    degree one in it (the error of a linear map): catches a bound that does
    not scale with the gradient it bounds."""
    sc, cam, rng = _scene(seed=25)
    cfg = O.Config(sh_degree=3)
    view, proj = _view(sc, cam, cfg)
    H, W = cam["height"], cam["width"]
    dL = rng.standard_normal((3, H, W))
    jac = O.pose_jacobian(sc, cam, cfg)
    b1 = O.render_bwd_bounds(proj, view["start"], view["ids"], cam, cfg, dL, jac=jac)
    b2 = O.render_bwd_bounds(proj, view["start"], view["ids"], cam, cfg, 2.0 * dL, jac=jac)
    b0 = O.render_bwd_bounds(proj, view["start"], view["ids"], cam, cfg, 0.0 * dL, jac=jac)
    assert (b1["fp32"] >= 0).all() and b1["fp32"].max() > 0
    assert not b0["fp32"].any() and not b0["flip"].any() and not b0["pose_fp32"].any()
    np.testing.assert_allclose(b2["fp32"], 2.0 * b1["fp32"], rtol=1e-12)
    np.testing.assert_allclose(b2["pose_fp32"], 2.0 * b1["pose_fp32"], rtol=1e-12)
    # every composited (item, pixel) contributes: items with a nonzero adjoint have a nonzero bound
    g = O.render_bwd(proj, view["start"], view["ids"], cam, cfg, dL)
    nz = np.abs(g).max(1) > 0
    assert (b1["fp32"].max(1)[nz] > 0).all()


def _pixel_sequence(proj, view, cam, cfg, x, y):
    """(id, alpha, T before it) of the Gaussians composited at pixel (x, y),
    recomputed in Python from the projected splats and the tile list."""
    tx, _ = O.tiles_xy(cam, cfg)
    t = (y // cfg.tile) * tx + x // cfg.tile
    seq, T = [], 1.0
    for i in view["ids"][view["start"][t]:view["start"][t + 1]]:
        og = O._alpha_on(proj, i, np.array([float(x)]), np.array([float(y)]))[0, 0]
        a = min(og, cfg.alpha_max)
        if a < cfg.alpha_min:
            continue
        if T * (1 - a) < cfg.t_min:
            break
        seq.append((int(i), a, T, og))
        T *= 1 - a
    return seq


@pytest.mark.parametrize("kind", ["clamp", "termination"])
def test_flip_bound_of_the_clamp_and_termination_decisions(kind):
    """The 0.99 clamp (alpha_max placed a hair either side of one Gaussian's
    o*g at one pixel: the clamped branch has no gradient through the exponent
    and opacity) and the termination test (t_min placed a hair either side of
    the transmittance after one Gaussian): the flip bound equals the change of
    the adjoint across the threshold: catches a forced branch that does not
    match the real one."""
    sc, cam, rng = _scene(sh_degree=0, seed=26, n=30, size=32)
    base = O.Config(sh_degree=0, **TIGHT)
    view, proj = _view(sc, cam, base)
    H, W = cam["height"], cam["width"]
    pick = None
    for y in range(H):
        for x in range(W):
            seq = _pixel_sequence(proj, view, cam, base, x, y)
            if len(seq) >= 3:
                pick = (x, y, seq)
                break
        if pick:
            break
    assert pick is not None
    x, y, seq = pick
    i, a, T, og = seq[1]
    if kind == "clamp":
        lo, hi = dict(alpha_max=og * (1 - 1e-9)), dict(alpha_max=og * (1 + 1e-9))
    else:
        lo, hi = dict(t_min=T * (1 - a) * (1 - 1e-9)), dict(t_min=T * (1 - a) * (1 + 1e-9))
    dL = np.zeros((3, H, W))
    dL[:, y, x] = rng.standard_normal(3)  # one pixel: its decision is the only one the bound flips
    out = []
    for c in (lo, hi):
        cfg = O.Config(sh_degree=0, **{**TIGHT, **c})
        v, _ = _view(sc, cam, cfg)
        g = O.render_bwd(proj, v["start"], v["ids"], cam, cfg, dL)
        out.append((cfg, v, g))
    diff = np.abs(out[0][2] - out[1][2])
    assert diff.max() > 0
    jac = O.pose_jacobian(sc, cam, base)
    # moving the threshold by 1e-9 also moves every other clamped alpha (or nothing else, for t_min) by that
    # much; the flip itself is of the order of a whole contribution
    for cfg, v, g in out:
        bb = O.render_bwd_bounds(proj, v["start"], v["ids"], cam, cfg, dL, jac=jac)
        np.testing.assert_allclose(bb["flip"], diff, rtol=1e-6, atol=1e-7 * np.abs(g).max())
        dpose = np.abs(np.einsum("icq,iq->c", jac, out[0][2] - out[1][2]))
        np.testing.assert_allclose(bb["pose_flip"], dpose, rtol=1e-6, atol=1e-7 * dpose.max())


def test_flip_bound_of_a_depth_tie_is_the_swap():
    """Two Gaussians at exactly the same depth are ordered by id; the other
    order (the larger id's fp32 key one ulp nearer) changes the adjoint at a
    pixel where both composite by exactly the depth-tie flip bound (dL/dC
    nonzero at that pixel only): catches a swap of the wrong entries or a
    missing transmittance effect."""
    sc, cam, rng = _scene(sh_degree=0, seed=27, n=30, size=32)
    cam = dict(cam, R=np.eye(3), t=np.zeros(3))
    cfg = O.Config(sh_degree=0, **TIGHT)
    H, W = cam["height"], cam["width"]
    view, proj = _view(sc, cam, cfg)
    # a pixel with at least two composited Gaussians; give the second the first's depth
    pick = None
    for y in range(H):
        for x in range(W):
            seq = _pixel_sequence(proj, view, cam, cfg, x, y)
            if len(seq) >= 2:
                pick = (x, y, seq[0][0], seq[1][0])
                break
        if pick:
            break
    assert pick is not None
    x, y, a, b = pick
    sc.mean_opa[b, 2] = sc.mean_opa[a, 2]
    view, proj = _view(sc, cam, cfg)
    lo, hi = min(a, b), max(a, b)
    key2 = proj["depth_key"].copy()
    key2[hi] = np.nextafter(key2[hi], np.float32(0))
    tx, ty = O.tiles_xy(cam, cfg)
    start2, ids2 = O.tile_lists(proj["rect"], key2, tx, ty)
    dL = np.zeros((3, H, W))
    dL[:, y, x] = rng.standard_normal(3)
    g0 = O.render_bwd(proj, view["start"], view["ids"], cam, cfg, dL)
    g1 = O.render_bwd(proj, start2, ids2, cam, cfg, dL)
    diff = np.abs(g1 - g0)
    assert diff[a].max() > 0 and diff[b].max() > 0
    jac = O.pose_jacobian(sc, cam, cfg)
    bb = O.render_bwd_bounds(proj, view["start"], view["ids"], cam, cfg, dL, jac=jac)
    np.testing.assert_allclose(bb["flip"], diff, rtol=1e-9, atol=1e-12 * np.abs(g0).max())
    dpose = np.abs(np.einsum("icq,iq->c", jac, g1 - g0))
    np.testing.assert_allclose(bb["pose_flip"], dpose, rtol=1e-9, atol=1e-12 * dpose.max())


def test_near_plane_item_may_appear_by_its_whole_splat():
    """A Gaussian a hair in front of the near plane is culled but flagged; the
    bound must cover the view with the plane moved past it, where it is a
    splat in front of everything: with dL/dC nonzero in one of its tiles only,
    the bound equals |adjoint with the item - adjoint without| (and the pose
    bound the pose change): catches a near-plane item left out of the bound or
    projected differently from the oracle's own projection."""
    sc, cam, rng = _scene(sh_degree=0, seed=28, n=30, size=48)
    cam = dict(cam, R=np.eye(3), t=np.zeros(3))
    cfg = O.Config(sh_degree=0, **dict(TIGHT, margin_geo=1e-5))
    i = 0
    sc.mean_opa[i, :3] = [0.002, -0.001, cfg.near_z * (1 - 2e-6)]
    sc.scale[i, :3] = np.log(0.02)
    sc.mean_opa[i, 3] = 1.0
    view, proj = _view(sc, cam, cfg)
    assert proj["n_tiles"][i] == 0 and proj["amb"][i] & 1
    cfg2 = O.Config(sh_degree=0, **dict(TIGHT, margin_geo=1e-5, near_z=cfg.near_z * (1 - 4e-6)))
    view2, proj2 = _view(sc, cam, cfg2)
    assert proj2["n_tiles"][i] > 1
    H, W = cam["height"], cam["width"]
    tx, _ = O.tiles_xy(cam, cfg)
    x0, y0, x1, y1 = proj2["rect"][i]
    T = cfg.tile
    dL = np.zeros((3, H, W))
    dL[:, y0 * T:(y0 + 1) * T, x0 * T:(x0 + 1) * T] = rng.standard_normal((3, T, T))
    g0 = O.render_bwd(proj, view["start"], view["ids"], cam, cfg, dL)
    # the adjoint with the item listed, from the same (unshifted) projection of the others
    start2, ids2 = O.tile_lists(proj2["rect"], proj2["depth_key"], tx, O.tiles_xy(cam, cfg)[1])
    g1 = O.render_bwd(proj2, start2, ids2, cam, cfg, dL)
    bb = O.adjoint_bounds(sc, view, cam, cfg, dL)
    assert bb["near_plane"] == 1 and bb["masked_pixels"] == 0
    diff = np.abs(g1 - g0)
    assert diff[i].max() > 0
    np.testing.assert_allclose(bb["flip"], diff, rtol=1e-9, atol=1e-12 * np.abs(g1).max())
    jac = O.pose_jacobian(sc, cam, cfg2)
    dpose = np.abs(np.einsum("icq,iq->c", jac, g1 - g0))
    np.testing.assert_allclose(bb["pose_flip"], dpose, rtol=1e-9, atol=1e-12 * dpose.max())


@pytest.mark.parametrize("alpha_rect", [0, 1])
def test_edge_sides_and_membership_groups(alpha_rect):
    """With a wide rect margin many edges are flagged. The side bit of each
    flagged edge must say on which side of the tile boundary the FP64 edge
    lies (edges recomputed here from the projected conic with numpy's
    eigvalsh, and with the opacity-aware bounds on, from the box where alpha
    reaches alpha_min; the flagged edge is the binding one of the two, the
    3-sigma edge when both bind), and the tiles of each membership group must
    be exactly the tiles whose membership changes when that one edge rounds
    the other way: catches a side inverted, or a join and a leave swapped."""
    sc, cam, rng = _scene(sh_degree=0, seed=29, n=300, size=96)
    cfg = O.Config(sh_degree=0, alpha_rect=alpha_rect, **dict(TIGHT, margin_rect_px=3.0))
    view, proj = _view(sc, cam, cfg)
    T = cfg.tile
    tx, ty = O.tiles_xy(cam, cfg)
    memb, mask, _ = O.ambiguous_memberships(view, cam, cfg)
    groups = {}
    for t, i, g in memb:
        groups.setdefault(int(g), (int(i), set()))[1].add(int(t))
    checked = 0
    seen = set()
    for i in np.nonzero(((proj["amb"] & (4 | 8 | 16 | 32)) > 0) & (proj["n_tiles"] > 0))[0]:
        S = np.linalg.inv(np.array([[proj["conic"][i, 0], proj["conic"][i, 1]], [proj["conic"][i, 1], proj["conic"][i, 2]]]))
        m = 0.5 * (S[0, 0] + S[1, 1])
        lam = m + np.sqrt(max(0.1, m * m - np.linalg.det(S)))
        assert lam >= np.linalg.eigvalsh(S).max() - 1e-9
        r = np.ceil(3 * np.sqrt(lam))
        u, v = proj["mean2d"][i]
        e3 = [(u - r) / T, (v - r) / T, (u + r + T - 1) / T, (v + r + T - 1) / T]
        ta = 2 * np.log(proj["opacity"][i] / cfg.alpha_min)
        hx, hy = np.sqrt(ta * S[0, 0]), np.sqrt(ta * S[1, 1])
        ea = [(u - hx) / T, (v - hy) / T, (u + hx) / T + 1, (v + hy) / T + 1]
        lim = [tx, ty, tx, ty]
        x0, y0, x1, y1 = (int(c) for c in proj["rect"][i])
        for c in range(4):
            if not proj["amb"][i] & (4 << c) or proj["edge_side"][i] & (16 << c):
                continue
            f3 = min(max(np.floor(e3[c]), 0), lim[c])
            fa = min(max(np.floor(ea[c]), 0), lim[c])
            near = lambda x: 1 <= np.rint(x) <= lim[c] and abs(x - np.rint(x)) * T < cfg.margin_rect_px
            bind3 = not alpha_rect or (f3 >= fa if c < 2 else f3 <= fa)
            binda = alpha_rect and (fa >= f3 if c < 2 else fa <= f3)
            e = e3 if bind3 and near(e3[c]) else ea
            assert (bind3 and near(e3[c])) or (binda and near(ea[c])), (i, c)
            k = np.rint(e[c])
            assert bool(proj["edge_side"][i] & (1 << c)) == (e[c] >= k), (i, c)
            # the edge rounded the other way
            alt = [x0, y0, x1, y1]
            alt[c] += -1 if e[c] >= k else 1
            old_t = {ry * tx + cx for ry in range(y0, y1) for cx in range(x0, x1)}
            new_t = {ry * tx + cx for ry in range(max(alt[1], 0), min(alt[3], ty))
                     for cx in range(max(alt[0], 0), min(alt[2], tx))}
            changed = old_t ^ new_t
            if not changed:
                continue
            match = [g for g, (it, ts) in groups.items() if it == i and ts == changed and g not in seen]
            assert match, (i, c, changed)
            seen.add(match[0])
            checked += 1
    assert checked > 20
