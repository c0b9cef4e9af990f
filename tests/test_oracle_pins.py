"""Pins of the FP64 oracle against facts fixed outside it: closed forms,
library routines, brute force, invariants and finite differences.

CPU only (no GPU marker). Each test names the mistake it would catch.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as O
from oracle import brute
from paper_2506_05558_gb300 import synth


def one_gaussian(mean, log_scale, quat_wxyz, opa_logit=0.0, dc=(0.0, 0.0, 0.0)):
    mo = np.array([[*mean, opa_logit]], np.float64)
    sc = np.array([[*log_scale, 0.0]], np.float64)
    q = np.array([quat_wxyz], np.float64)
    sh = np.zeros((1, 48))
    sh[0, :3] = dc
    return synth.Scene(mo, sc, q, sh, 0)


def sigma2d_from_conic(c):
    a, b, cc = c
    return np.linalg.inv(np.array([[a, b], [b, cc]]))


# ---------------------------------------------------------------------------
# Projection (EWA): closed forms
# ---------------------------------------------------------------------------

def test_projection_axis_aligned_closed_form():
    """Sigma2D = J W Sigma W^T J^T + 0.3 I for an axis-aligned Gaussian with W = I,
    written out by hand: catches a transposed J, a dropped third column of J or
    a missing dilation."""
    fx, fy, W, H = 300.0, 250.0, 640, 480
    cam = synth.camera(np.eye(3), np.zeros(3), fx, W, H, fy=fy)
    x, y, z = 0.7, -0.4, 3.0
    s = np.array([0.05, 0.08, 0.12])
    sc = one_gaussian([x, y, z], np.log(s), [1, 0, 0, 0])
    cfg = O.Config(sh_degree=0)
    p = O.project(sc, cam, cfg)
    sx2, sy2, sz2 = s ** 2
    a = fx * fx * (sx2 / z ** 2 + x * x * sz2 / z ** 4) + 0.3
    b = fx * fy * x * y * sz2 / z ** 4
    c = fy * fy * (sy2 / z ** 2 + y * y * sz2 / z ** 4) + 0.3
    S = sigma2d_from_conic(p["conic"][0])
    np.testing.assert_allclose(S, [[a, b], [b, c]], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(p["mean2d"][0], [fx * x / z + W / 2, fy * y / z + H / 2], rtol=1e-14)
    assert p["depth"][0] == z
    assert p["opacity"][0] == 0.5


def test_projection_rotation_cancels():
    """A Gaussian rotated by q seen by a camera whose rotation is R(q)^T at the
    origin sees the axis-aligned covariance diag(s^2) in camera space. The
    rotation comes from scipy, so a wrong quaternion convention (order, sign,
    transpose) or a wrong W placement fails."""
    rot = Rotation.from_rotvec([0.3, -0.5, 0.9])
    qx, qy, qz, qw = rot.as_quat()
    Rq = rot.as_matrix()
    s = np.array([0.03, 0.06, 0.1])
    # mean on the optical axis at depth 4 in camera coordinates
    mean_world = Rq @ np.array([0.0, 0.0, 4.0])
    cam = synth.camera(Rq.T, np.zeros(3), 200.0, 320, 240, dtype=np.float64)
    sc = one_gaussian(mean_world, np.log(s), [qw, qx, qy, qz])
    p = O.project(sc, cam, O.Config(sh_degree=0))
    z = 4.0
    S = sigma2d_from_conic(p["conic"][0])
    f = 200.0
    np.testing.assert_allclose(S, [[f * f * s[0] ** 2 / z ** 2 + 0.3, 0], [0, f * f * s[1] ** 2 / z ** 2 + 0.3]],
                               rtol=1e-10, atol=1e-10)
    # an unnormalised quaternion gives the same result
    sc2 = one_gaussian(mean_world, np.log(s), [3 * qw, 3 * qx, 3 * qy, 3 * qz])
    p2 = O.project(sc2, cam, O.Config(sh_degree=0))
    np.testing.assert_allclose(p2["conic"], p["conic"], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("alpha_rect", [0, 1])
def test_projection_radius_and_rect(alpha_rect):
    """3-sigma radius from the largest eigenvalue (numpy eigvalsh) and the tile
    rect; with the opacity-aware bounds, intersected with the tiles of the box
    where o exp(-q/2) reaches alpha_min (its half-widths sqrt(2 ln(o / alpha_min)
    Sigma2D_xx) and likewise in y: the extent of that ellipse)."""
    sc, cam, _ = synth.tiny_scene(n=200)
    cfg = O.Config(sh_degree=0, alpha_rect=alpha_rect)
    p = O.project(sc, cam, cfg)
    T = cfg.tile
    checked = 0
    for i in np.nonzero(p["n_tiles"])[0][:50]:
        S = sigma2d_from_conic(p["conic"][i])
        lam = np.linalg.eigvalsh(S).max()
        r = math.ceil(3 * math.sqrt(max(lam, 0.5 * np.trace(S) + math.sqrt(0.1))))
        u, v = p["mean2d"][i]
        cl = lambda f: min(max(f, 0), 4)
        rect = [cl(math.floor((u - r) / T)), cl(math.floor((v - r) / T)), cl(math.floor((u + r + T - 1) / T)),
                cl(math.floor((v + r + T - 1) / T))]
        if alpha_rect:
            t = 2 * math.log(p["opacity"][i] / cfg.alpha_min)
            # the ellipse's extent along x: max x of {d : d^T S^-1 d <= t} is sqrt(t S_xx) (Cauchy-Schwarz)
            hx, hy = math.sqrt(t * S[0, 0]), math.sqrt(t * S[1, 1])
            box = [cl(math.floor((u - hx) / T)), cl(math.floor((v - hy) / T)), cl(math.floor((u + hx) / T) + 1),
                   cl(math.floor((v + hy) / T) + 1)]
            rect = [max(rect[0], box[0]), max(rect[1], box[1]), min(rect[2], box[2]), min(rect[3], box[3])]
            checked += rect != [cl(math.floor((u - r) / T)), cl(math.floor((v - r) / T)),
                                cl(math.floor((u + r + T - 1) / T)), cl(math.floor((v + r + T - 1) / T))]
        assert list(p["rect"][i]) == rect, (i, list(p["rect"][i]), rect)
    assert not alpha_rect or checked > 0


def test_opacity_aware_rect_drops_no_composited_pair():
    """The opacity-aware tile bounds only drop list entries no pixel composites:
    the image, the final transmittance and the adjoint equal those of the
    3-sigma rects (to rounding: the same composited pairs in the same order),
    with fewer pairs."""
    sc, cam, rng = synth.tiny_scene(n=1000)
    w = rng.standard_normal((3, cam["height"], cam["width"]))
    res = {}
    for ar in (0, 1):
        cfg = O.Config(sh_degree=0, alpha_rect=ar)
        v = O.render_view(sc, cam, cfg)
        b = O.backward_view(sc, cam, cfg, v, w)
        res[ar] = (v, b, int(v["proj"]["n_tiles"].sum()))
    (v0, b0, p0), (v1, b1, p1) = res[0], res[1]
    assert p1 < 0.95 * p0, (p1, p0)
    np.testing.assert_allclose(v1["color"], v0["color"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(v1["t_final"], v0["t_final"], rtol=0, atol=1e-13)
    for k in ("mean", "logit", "log_scale", "quat", "sh", "pose"):
        np.testing.assert_allclose(b1[k], b0[k], rtol=1e-12, atol=1e-12 * np.abs(b0[k]).max())


def test_near_plane_and_nonfinite_cull():
    sc = one_gaussian([0, 0, 0.1], np.log([0.1] * 3), [1, 0, 0, 0])
    cam = synth.camera(np.eye(3), np.zeros(3), 80.0, 64, 64)
    assert O.project(sc, cam, O.Config(sh_degree=0))["n_tiles"][0] == 0
    for field, idx in (("mean_opa", 0), ("scale", 1), ("quat", 2), ("sh", 0), ("mean_opa", 3)):
        s2 = one_gaussian([0, 0, 3], np.log([0.1] * 3), [1, 0, 0, 0])
        getattr(s2, field)[0, idx] = np.nan
        assert O.project(s2, cam, O.Config(sh_degree=0))["n_tiles"][0] == 0, field


# ---------------------------------------------------------------------------
# Spherical harmonics
# ---------------------------------------------------------------------------

def _dirs(n=50, seed=0):
    d = np.random.default_rng(seed).standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_sh_matches_scipy():
    """Real SH (Condon-Shortley phase) against scipy's complex SH:
    Y_l^m = sqrt2 Re(Y_lm), Y_l^-m = sqrt2 Im(Y_lm), Y_l^0 = Y_l0."""
    from scipy.special import sph_harm_y
    for d in _dirs():
        Y, _ = O.sh_basis(3, d)
        theta = math.acos(d[2])
        phi = math.atan2(d[1], d[0])
        for l in range(4):
            for m in range(-l, l + 1):
                ref = complex(sph_harm_y(l, abs(m), theta, phi))
                want = ref.real if m == 0 else (math.sqrt(2) * (ref.real if m > 0 else ref.imag))
                assert abs(Y[l * l + l + m] - want) < 1e-12, (l, m)


def test_sh_low_order_closed_forms():
    """Textbook l <= 1: Y00 = 1/(2 sqrt(pi)), Y1(-1,0,1) = sqrt(3/(4pi)) (-y, z, -x)."""
    c0 = 1 / (2 * math.sqrt(math.pi))
    c1 = math.sqrt(3 / (4 * math.pi))
    for d in _dirs(10):
        Y, _ = O.sh_basis(1, d)
        np.testing.assert_allclose(Y[:4], [c0, -c1 * d[1], c1 * d[2], -c1 * d[0]], rtol=0, atol=1e-14)


def test_sh_orthonormal_by_quadrature():
    """Gauss-Legendre in cos(theta) x uniform phi integrates degree <= 6 products exactly."""
    xs, ws = np.polynomial.legendre.leggauss(12)
    nphi = 16
    G = np.zeros((16, 16))
    for z, w in zip(xs, ws):
        for k in range(nphi):
            phi = 2 * math.pi * k / nphi
            r = math.sqrt(1 - z * z)
            Y, _ = O.sh_basis(3, np.array([r * math.cos(phi), r * math.sin(phi), z]))
            G += w * (2 * math.pi / nphi) * np.outer(Y, Y)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_gradient_by_finite_differences():
    for d in _dirs(10, 3):
        _, dY = O.sh_basis(3, d)
        h = 1e-6
        for c in range(3):
            e = np.zeros(3)
            e[c] = h
            fd = (O.sh_basis(3, d + e)[0] - O.sh_basis(3, d - e)[0]) / (2 * h)
            np.testing.assert_allclose(dY[:, c], fd, atol=1e-8)


# ---------------------------------------------------------------------------
# Compositing
# ---------------------------------------------------------------------------

def _cam_px(W=32, H=32, f=40.0):
    return synth.camera(np.eye(3), np.zeros(3), f, W, H)


def _at_pixel(cam, px, py, z):
    """World point that projects exactly onto the centre of pixel (px, py)."""
    u, v = px + 0.5, py + 0.5
    return [(u - cam["cx"]) * z / cam["fx"], (v - cam["cy"]) * z / cam["fy"], z]


def test_single_gaussian_at_its_centre():
    """A single Gaussian at a pixel centre composites to o*rgb + (1-o) bg."""
    cam = _cam_px()
    o = 0.7
    logit = math.log(o / (1 - o))
    sc = one_gaussian(_at_pixel(cam, 10, 12, 3.0), np.log([0.05] * 3), [1, 0, 0, 0], logit, (0.5, -0.3, 1.0))
    bg = (0.2, 0.1, 0.05)
    cfg = O.Config(sh_degree=0, bg=bg)
    v = O.render_view(sc, cam, cfg)
    rgb = v["proj"]["rgb"][0]
    got = v["color"][:, 12, 10]
    np.testing.assert_allclose(got, o * rgb + (1 - o) * np.array(bg), rtol=1e-12)
    assert abs(v["t_final"][12, 10] - (1 - o)) < 1e-12
    assert v["n_contrib"][12, 10] == 1
    np.testing.assert_allclose(rgb, 0.5 + np.array([0.5, -0.3, 1.0]) / (2 * math.sqrt(math.pi)), rtol=1e-12)


def test_opacity_clamp():
    """o > 0.99 at the centre composites with alpha = 0.99."""
    cam = _cam_px()
    sc = one_gaussian(_at_pixel(cam, 5, 5, 3.0), np.log([0.05] * 3), [1, 0, 0, 0], 8.0, (1.0, 1.0, 1.0))
    v = O.render_view(sc, cam, O.Config(sh_degree=0))
    assert abs(v["t_final"][5, 5] - 0.01) < 1e-12


def test_two_gaussians_front_to_back():
    """Two Gaussians centred on the same pixel: a1 c1 + (1 - a1) a2 c2, nearer first
    whatever the input order."""
    cam = _cam_px()
    g_near = (_at_pixel(cam, 7, 9, 2.0), 0.4, (0.9, -1.0, 0.1))
    g_far = (_at_pixel(cam, 7, 9, 5.0), -0.2, (-1.2, 0.8, 0.6))
    o1, o2 = 1 / (1 + math.exp(-0.4)), 1 / (1 + math.exp(0.2))
    for order in ((g_near, g_far), (g_far, g_near)):
        mo = np.array([[*g[0], g[1]] for g in order])
        sc = synth.Scene(mo, np.tile(np.log([0.05, 0.05, 0.05, 1.0]), (2, 1)), np.tile([1.0, 0, 0, 0], (2, 1)),
                         np.zeros((2, 48)), 0)
        sc.sh[0, :3] = order[0][2]
        sc.sh[1, :3] = order[1][2]
        v = O.render_view(sc, cam, O.Config(sh_degree=0))
        c1 = 0.5 + np.array(g_near[2]) / (2 * math.sqrt(math.pi))
        c2 = 0.5 + np.array(g_far[2]) / (2 * math.sqrt(math.pi))
        c1, c2 = np.maximum(c1, 0), np.maximum(c2, 0)
        np.testing.assert_allclose(v["color"][:, 9, 7], o1 * c1 + (1 - o1) * o2 * c2, rtol=1e-12)


def test_transmittance_bounds_and_colour_bound():
    sc, cam, _ = synth.tiny_scene()
    v = O.render_view(sc, cam, O.Config(sh_degree=0))
    assert np.all(v["t_final"] >= O.Config().t_min) and np.all(v["t_final"] <= 1)
    rgb_max = v["proj"]["rgb"].max()
    assert np.all(v["color"] <= rgb_max + 1e-12) and np.all(v["color"] >= 0)
    # transmittance is non-increasing along a pixel's list: check via prefixes
    tx, ty = O.tiles_xy(cam, O.Config())
    start, ids = v["start"], v["ids"]
    prev = None
    for cut in (1, 3, 10, 1000):
        st = start.copy()
        for t in range(tx * ty):
            st[t + 1] = st[t] + min(cut, start[t + 1] - start[t])
        ids_cut = np.concatenate([ids[start[t]:start[t] + min(cut, start[t + 1] - start[t])]
                                  for t in range(tx * ty)])
        T = O.render_fwd(v["proj"], st, ids_cut, cam, O.Config(sh_degree=0))["t_final"]
        if prev is not None:
            assert np.all(T <= prev + 1e-15)
        prev = T


def test_brute_force_twin():
    """Tiled oracle == per-pixel global-order brute force to 1e-12 on tiny scenes,
    and the same number of composited Gaussians per pixel (the count the
    benchmark's roofline uses)."""
    for seed in (1, 2, 3):
        sc, cam, _ = synth.tiny_scene(seed=seed, n=50, width=48, height=40, f=60.0)
        # larger Gaussians so that lists overlap across tiles
        sc.scale[:, :3] += 1.0
        cfg = O.Config(sh_degree=0)
        v = O.render_view(sc, cam, cfg)
        assert len(v["ids"]) > 60
        col, T, nc = brute.render(v["proj"], cam["width"], cam["height"], cfg.tile)
        np.testing.assert_allclose(v["color"], col, atol=1e-12)
        np.testing.assert_allclose(v["t_final"], T, atol=1e-12)
        assert np.array_equal(v["n_composited"], nc)


def test_permutation_invariance():
    """Permuting Gaussians with distinct depths leaves the image bit-identical."""
    sc, cam, rng = synth.tiny_scene(n=300)
    cfg = O.Config(sh_degree=0)
    v = O.render_view(sc, cam, cfg)
    perm = rng.permutation(sc.n)
    v2 = O.render_view(synth.scene_subset(sc, perm), cam, cfg)
    assert np.array_equal(v["color"], v2["color"])


def test_equal_depth_tie_break_by_id():
    """Equal fp32 depths are ordered by Gaussian id inside a tile."""
    cam = _cam_px()
    mo = np.array([[*_at_pixel(cam, 4, 4, 3.0), 0.0], [*_at_pixel(cam, 5, 4, 3.0), 0.0]])
    mo[1, 0] = mo[0, 0] + 0.01
    sc = synth.Scene(mo, np.tile(np.log([0.05, 0.05, 0.05, 1.0]), (2, 1)), np.tile([1.0, 0, 0, 0], (2, 1)),
                     np.zeros((2, 48)), 0)
    p = O.project(sc, cam, O.Config(sh_degree=0))
    assert p["depth_key"][0] == p["depth_key"][1]
    start, ids = O.tile_lists(p["rect"], p["depth_key"], 2, 2)
    assert list(ids[start[0]:start[1]]) == [0, 1]


# ---------------------------------------------------------------------------
# Gradients: FP64 central finite differences of the oracle forward
# ---------------------------------------------------------------------------

def _loss(sc, cam, cfg, w, lists=None):
    proj = O.project(sc, cam, cfg)
    if lists is None:
        tx, ty = O.tiles_xy(cam, cfg)
        lists = O.tile_lists(proj["rect"], proj["depth_key"], tx, ty)
    img = O.render_fwd(proj, lists[0], lists[1], cam, cfg)
    return float((w * img["color"]).sum()), lists


def _fd_scene(sh_degree, seed):
    sc, cam, rng = synth.tiny_scene(seed=seed, n=25, width=32, height=32, f=40.0, sh_degree=sh_degree)
    # FP64 copies so that finite-difference steps are not rounded to fp32
    sc = synth.Scene(sc.mean_opa.astype(np.float64), sc.scale.astype(np.float64), sc.quat.astype(np.float64),
                     sc.sh.astype(np.float64), sh_degree)
    sc.scale[:, :3] += 0.5
    sc.mean_opa[:, 3] = rng.normal(-0.5, 0.5, sc.n)
    if sh_degree > 0:
        sc.sh[:, 3:48] = rng.normal(0, 0.2, (sc.n, 45)) * (np.arange(45) < 3 * (sh_degree + 1) ** 2 - 3)
    # tilt the camera so that the pose has all six components active
    R, t = O.retract_pose(np.eye(3), np.zeros(3), [0.05, -0.03, 0.02, 0.02, -0.03, 0.01])
    cam = dict(cam, R=R, t=t)
    return sc, cam, rng


@pytest.mark.parametrize("sh_degree,through_sh,mip", [(0, 0, 0), (3, 1, 0), (3, 0, 0), (0, 0, 1), (3, 0, 1)])
def test_gradients_match_central_differences(sh_degree, through_sh, mip):
    cfg = O.Config(sh_degree=sh_degree, pose_grad_through_sh=through_sh, bg=(0.1, 0.2, 0.3), mip_filter=mip,
                   dilation=0.1 if mip else 0.3)
    # first seed whose scene has no decision within the ambiguity margins
    for seed in range(11, 40):
        sc, cam, rng = _fd_scene(sh_degree, seed)
        v = O.render_view(sc, cam, cfg)
        if v["amb"].sum() == 0 and v["proj"]["amb"].sum() == 0:
            break
    assert v["amb"].sum() == 0 and v["proj"]["amb"].sum() == 0
    w = rng.standard_normal((3, cam["height"], cam["width"]))
    g = O.backward_view(sc, cam, cfg, v, w)
    lists = (v["start"], v["ids"])
    h = 1e-6

    def fd_param(field, i, c):
        arr = getattr(sc, field)
        old = arr[i, c]
        step = h * max(1.0, abs(old))
        arr[i, c] = old + step
        lp, _ = _loss(sc, cam, cfg, w, lists)
        arr[i, c] = old - step
        lm, _ = _loss(sc, cam, cfg, w, lists)
        arr[i, c] = old
        return (lp - lm) / (2 * step)

    vis = np.nonzero(v["proj"]["n_tiles"])[0]
    checks = []
    for i in vis[:8]:
        for c in range(3):
            checks.append((fd_param("mean_opa", i, c), g["mean"][i, c]))
            checks.append((fd_param("scale", i, c), g["log_scale"][i, c]))
        checks.append((fd_param("mean_opa", i, 3), g["logit"][i]))
        for c in range(4):
            checks.append((fd_param("quat", i, c), g["quat"][i, c]))
        for c in range(3 * (sh_degree + 1) ** 2):
            checks.append((fd_param("sh", i, c), g["sh"][i, c]))
    fd = np.array([a for a, _ in checks])
    an = np.array([b for _, b in checks])
    scale = np.abs(fd).max()
    np.testing.assert_allclose(an, fd, rtol=1e-5, atol=1e-6 * scale)

    # pose: left perturbation exp(xi^) T_cw. With SH > 0 and the SH path
    # excluded, finite differences are taken with the view direction frozen,
    # i.e. the SH colours held at their unperturbed values.
    for k in range(6):
        xi = np.zeros(6)
        xi[k] = h
        vals = []
        for s in (1, -1):
            c2 = O.perturbed_cam(cam, s * xi)
            if sh_degree > 0 and not through_sh:
                proj = O.project(sc, c2, cfg)
                proj["rgb"] = v["proj"]["rgb"]
                img = O.render_fwd(proj, lists[0], lists[1], c2, cfg)
                vals.append(float((w * img["color"]).sum()))
            else:
                vals.append(_loss(sc, c2, cfg, w, lists)[0])
        fdk = (vals[0] - vals[1]) / (2 * h)
        assert abs(fdk - g["pose"][k]) <= 1e-5 * abs(fdk) + 1e-6 * np.abs(g["pose"]).max(), (k, fdk, g["pose"][k])


def test_gradient_of_clamped_alpha_is_zero_in_opacity():
    cam = _cam_px()
    sc = one_gaussian(_at_pixel(cam, 5, 5, 3.0), np.log([0.02] * 3), [1, 0, 0, 0], 8.0, (1.0, 1.0, 1.0))
    cfg = O.Config(sh_degree=0)
    v = O.render_view(sc, cam, cfg)
    w = np.zeros((3, 32, 32))
    w[:, 5, 5] = 1.0
    g = O.backward_view(sc, cam, cfg, v, w)
    assert g["g2d"][0, 5] == 0.0


# ---------------------------------------------------------------------------
# Optimiser, loss, pose retraction
# ---------------------------------------------------------------------------

def test_adam_closed_forms():
    """First step moves each entry by -lr sign(g) (|g| >> eps); a constant
    gradient keeps that step size; masked rows are untouched."""
    rng = np.random.default_rng(0)
    p = rng.standard_normal((5, 7))
    g = rng.standard_normal((5, 7))
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    mask = np.array([1, 1, 0, 1, 0], bool)
    p1, m1, v1 = O.adam_step(p, g, m, v, 1, 0.01, mask=mask)
    np.testing.assert_allclose(p1[mask], p[mask] - 0.01 * np.sign(g[mask]), rtol=1e-12)
    assert np.array_equal(p1[~mask], p[~mask]) and np.all(m1[~mask] == 0)
    p2, m2, v2 = p1, m1, v1
    for step in range(2, 6):
        p2, m2, v2 = O.adam_step(p2, g, m2, v2, step, 0.01, mask=mask)
    np.testing.assert_allclose(p2[mask], p[mask] - 0.05 * np.sign(g[mask]), rtol=1e-10)


def test_l1_loss_gradient():
    c = np.array([0.2, 0.5, 0.9, 0.4])
    t = np.array([0.1, 0.5, 1.0, 0.0])
    loss, grad = O.l1_loss_grad(c, t)
    assert abs(loss - (0.1 + 0 + 0.1 + 0.4) / 4) < 1e-15
    np.testing.assert_array_equal(grad, [0.25, 0.0, -0.25, 0.25])


def test_se3_exp_matches_matrix_exponential():
    from scipy.linalg import expm
    for xi in ([0.1, -0.2, 0.3, 0.4, -0.1, 0.25], [1.0, 0.0, 0.0, 0.0, 0.0, 0.0], [0, 0, 0, 1e-14, 0, 0]):
        xi = np.array(xi)
        X = np.zeros((4, 4))
        X[:3, :3] = O.hat(xi[3:])
        X[:3, 3] = xi[:3]
        E = expm(X)
        R, t = O.se3_exp(xi)
        np.testing.assert_allclose(R, E[:3, :3], atol=1e-12)
        np.testing.assert_allclose(t, E[:3, 3], atol=1e-12)


def _se3_mat(xi):
    R, t = O.se3_exp(xi)
    M = np.eye(4)
    M[:3, :3], M[:3, 3] = R, t
    return M


def _twist_mat(d):
    M = np.zeros((4, 4))
    M[:3, :3] = O.hat(d[3:])
    M[:3, 3] = d[:3]
    return M


def test_se3_left_jacobian_first_order_composition():
    """exp((xi + e v)^) exp(xi^)^-1 = I + e (J_l v)^ + O(e^2), checked by a
    central difference of the group elements (no rendering involved): a
    transposed block or a wrong sign in J_l fails."""
    rng = np.random.default_rng(3)
    for _ in range(5):
        xi = np.concatenate([rng.normal(0, 1.0, 3), rng.normal(0, 0.6, 3)])
        J = O.se3_left_jacobian(xi)
        inv = np.linalg.inv(_se3_mat(xi))
        for k in range(6):
            v = np.zeros(6)
            v[k] = 1.0
            e = 1e-6
            D = (_se3_mat(xi + e * v) @ inv - _se3_mat(xi - e * v) @ inv) / (2 * e)
            np.testing.assert_allclose(D, _twist_mat(J[:, k]), atol=2e-9)


def test_se3_left_jacobian_special_cases():
    """xi = 0 gives I; pure translation gives [[I, rho^ / 2], [0, I]] (ad^2 = 0)."""
    np.testing.assert_allclose(O.se3_left_jacobian(np.zeros(6)), np.eye(6), atol=0)
    rho = np.array([0.3, -1.2, 2.0])
    J = O.se3_left_jacobian(np.concatenate([rho, np.zeros(3)]))
    want = np.eye(6)
    want[:3, 3:] = 0.5 * O.hat(rho)
    np.testing.assert_allclose(J, want, atol=1e-15)


def test_pose_tangent_gradient_matches_central_differences():
    """dL/dxi of L(exp(xi^) T_ref) at a nonzero xi: J_l(xi)^T applied to the
    backward pass's gradient at the composed pose equals FP64 central
    differences of the rendered loss."""
    cfg = O.Config(sh_degree=0, bg=(0.1, 0.2, 0.3))
    xi0 = np.array([0.04, -0.02, 0.03, 0.05, -0.04, 0.03])
    for seed in range(11, 40):
        sc, cam, rng = _fd_scene(0, seed)
        cam1 = O.perturbed_cam(cam, xi0)
        v = O.render_view(sc, cam1, cfg)
        if v["amb"].sum() == 0 and v["proj"]["amb"].sum() == 0:
            break
    assert v["amb"].sum() == 0 and v["proj"]["amb"].sum() == 0
    w = rng.standard_normal((3, cam["height"], cam["width"]))
    g = O.backward_view(sc, cam1, cfg, v, w)
    an = O.pose_tangent_grad(xi0, g["pose"])
    lists = (v["start"], v["ids"])
    h = 1e-6
    fd = np.zeros(6)
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        lp, _ = _loss(sc, O.perturbed_cam(cam, xi0 + e), cfg, w, lists)
        lm, _ = _loss(sc, O.perturbed_cam(cam, xi0 - e), cfg, w, lists)
        fd[k] = (lp - lm) / (2 * h)
    np.testing.assert_allclose(an, fd, rtol=1e-5, atol=1e-6 * np.abs(fd).max())
    # the plain gradient (J_l dropped) is measurably different at this xi
    assert np.abs(g["pose"] - fd).max() > 1e-3 * np.abs(fd).max()


def test_depth_integral_closed_forms():
    """Depth integral sum_i alpha_i T_i z_i: one Gaussian at a pixel centre
    gives o z; two on the same pixel give o1 z1 + (1 - o1) o2 z2 in either
    input order; a background colour does not enter it; away from all splats 0."""
    cam = _cam_px()
    o = 0.7
    sc = one_gaussian(_at_pixel(cam, 10, 12, 3.0), np.log([0.05] * 3), [1, 0, 0, 0], math.log(o / (1 - o)))
    cfg = O.Config(sh_degree=0, bg=(0.3, 0.3, 0.3))
    v = O.render_view(sc, cam, cfg)
    d = O.render_depth(v["proj"], v["start"], v["ids"], cam, cfg)
    assert abs(d[12, 10] - o * 3.0) < 1e-12
    assert d[0, 0] == 0.0
    o1, o2 = 1 / (1 + math.exp(-0.4)), 1 / (1 + math.exp(0.2))
    near, far = (_at_pixel(cam, 7, 9, 2.0), 0.4), (_at_pixel(cam, 7, 9, 5.0), -0.2)
    for order in ((near, far), (far, near)):
        mo = np.array([[*g[0], g[1]] for g in order])
        sc2 = synth.Scene(mo, np.tile(np.log([0.05, 0.05, 0.05, 1.0]), (2, 1)), np.tile([1.0, 0, 0, 0], (2, 1)),
                          np.zeros((2, 48)), 0)
        v2 = O.render_view(sc2, cam, cfg)
        d2 = O.render_depth(v2["proj"], v2["start"], v2["ids"], cam, cfg)
        assert abs(d2[9, 7] - (o1 * 2.0 + (1 - o1) * o2 * 5.0)) < 1e-12


def test_mip_filter_single_gaussian_closed_form():
    """With the filter, an axis-aligned Gaussian on the optical axis (Sigma2D =
    diag(sx^2, sy^2), sx = fx Sx / z) composites at its centre to
    o sqrt(sx^2 sy^2 / ((sx^2 + s)(sy^2 + s))) rgb, s the filter variance; the
    conic is that of Sigma2D + s I."""
    cam = synth.camera(np.eye(3), np.zeros(3), 40.0, 33, 33, dtype=np.float64)
    cam = dict(cam, cx=16.5, cy=16.5)  # the optical axis through the centre of pixel (16, 16)
    o, z, S = 0.6, 4.0, (0.07, 0.03, 0.05)
    sc = one_gaussian([0.0, 0.0, z], np.log(S), [1, 0, 0, 0], math.log(o / (1 - o)), (0.4, 0.2, -0.1))
    s = 0.1
    cfg = O.Config(sh_degree=0, mip_filter=1, dilation=s)
    v = O.render_view(sc, cam, cfg)
    sx2, sy2 = (40.0 * S[0] / z) ** 2, (40.0 * S[1] / z) ** 2
    f = math.sqrt(sx2 * sy2 / ((sx2 + s) * (sy2 + s)))
    rgb = v["proj"]["rgb"][0]
    np.testing.assert_allclose(v["color"][:, 16, 16], o * f * rgb, rtol=1e-12)
    np.testing.assert_allclose(v["proj"]["opacity"][0], o * f, rtol=1e-12)
    np.testing.assert_allclose(v["proj"]["conic"][0], [1 / (sx2 + s), 0.0, 1 / (sy2 + s)], rtol=1e-12, atol=1e-15)
    # without the filter the same dilation leaves the opacity unchanged
    v0 = O.render_view(sc, cam, O.Config(sh_degree=0, mip_filter=0, dilation=s))
    np.testing.assert_allclose(v0["proj"]["opacity"][0], o, rtol=1e-12)


def test_per_gaussian_learning_rate_decay():
    """A Gaussian processed k times since its introduction has multiplier
    decay^k; the first Adam step it takes moves it by lr * multiplier * sign(g)."""
    rng = np.random.default_rng(0)
    n, decay = 50, 0.99
    s = np.ones(n)
    seen = np.zeros(n, int)
    for _ in range(7):
        mask = rng.random(n) < 0.6
        s = O.lr_decay(s, mask, decay)
        seen += mask
    np.testing.assert_allclose(s, decay ** seen, rtol=1e-14)
    p, g = rng.standard_normal(n), rng.standard_normal(n)
    p1, _, _ = O.adam_step(p, g, np.zeros(n), np.zeros(n), 1, 0.01 * s)
    np.testing.assert_allclose(p1, p - 0.01 * s * np.sign(g), rtol=0, atol=1e-12)


def test_downsample_hand_cases():
    """Factor 1 is the identity; a constant stays constant; a 4x4 ramp gives the
    block means; a 5x3 frame at factor 2 averages its partial edge blocks."""
    rng = np.random.default_rng(1)
    im = rng.random((3, 6, 7))
    np.testing.assert_array_equal(O.downsample(im, 1), im)
    np.testing.assert_allclose(O.downsample(np.full((3, 9, 5), 0.25), 4), np.full((3, 3, 2), 0.25))
    ramp = np.tile(np.arange(16.0).reshape(4, 4), (3, 1, 1))
    np.testing.assert_allclose(O.downsample(ramp, 2)[0], [[2.5, 4.5], [10.5, 12.5]])
    r = np.tile(np.arange(15.0).reshape(3, 5), (3, 1, 1))
    np.testing.assert_allclose(O.downsample(r, 2)[0], [[3.0, 5.0, 6.5], [10.5, 12.5, 14.0]])


def test_downsampled_camera_keeps_pixel_centres():
    """A world point at the centre of full-resolution pixel block (2I.., 2J..)
    projects to the centre of downsampled pixel (I, J)."""
    cam = synth.camera(np.eye(3), np.zeros(3), 40.0, 32, 24, dtype=np.float64)
    c2 = O.downsample_camera(cam, 4)
    for I, J in ((0, 0), (3, 5), (5, 7)):
        u, v = 4 * J + 2.0, 4 * I + 2.0  # centre of the block in full-resolution pixel coordinates
        z = 3.0
        p = [(u - cam["cx"]) * z / cam["fx"], (v - cam["cy"]) * z / cam["fy"], z]
        assert abs(c2["fx"] * p[0] / z + c2["cx"] - (J + 0.5)) < 1e-12
        assert abs(c2["fy"] * p[1] / z + c2["cy"] - (I + 0.5)) < 1e-12
