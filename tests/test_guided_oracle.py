"""Pins of the guided-matching oracle (App. A.2) against closed forms and an
independently built stereo scene: the candidate window, rectified-stereo
disparity, bilinear sampling of affine fields, the parabola vertex, the
adaptive neighbour choice, depth recovery on a textured plane, and the
degenerate pixels (no usable neighbour, invalid monocular depth, maximum at
the window's end)."""
import math

import numpy as np

from oracle import guided as G


def cam(R, t, f, W, H):
    return dict(R=np.asarray(R, np.float64), t=np.asarray(t, np.float64), fx=f, fy=f, cx=W / 2, cy=H / 2,
                width=W, height=H)


def to_bf16(x):
    u = np.ascontiguousarray(np.asarray(x, np.float32)).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)


def test_candidate_window():
    d = G.candidates(np.array([2.0, 20.0]), 5)
    assert np.allclose(d[0], [0.4, 0.45, 0.5, 0.55, 0.6], atol=1e-15)
    assert np.allclose(d[1], [0.0, 0.0375, 0.075, 0.1125, 0.15], atol=1e-15)  # 1/20 - 0.1 < 0: clamped at 0


def test_rectified_disparity_and_identity():
    f, W, H, B = 200.0, 64, 48, 0.25
    ci = cam(np.eye(3), [0, 0, 0], f, W, H)
    cj = cam(np.eye(3), [-B, 0, 0], f, W, H)  # centre at +B on x
    r = G.pixel_rays(ci)
    Rji, b = G.relative(ci, cj)
    d = np.full(len(r), 0.3)
    x, y, z = G.reproject(r @ Rji.T, b, d, cj)
    u = np.tile(np.arange(W) + 0.5, H)
    v = np.repeat(np.arange(H) + 0.5, W)
    assert np.allclose(x, u - f * B * 0.3, atol=1e-12) and np.allclose(y, v, atol=1e-12) and np.all(z == 1)
    x, y, _ = G.reproject(r, np.zeros(3), d * 7, ci)  # the same camera: every depth maps to the pixel itself
    assert np.allclose(x, u, atol=1e-12) and np.allclose(y, v, atol=1e-12)


def test_reprojection_round_trip_general_pose():
    rng = np.random.default_rng(3)
    from scipy.spatial.transform import Rotation
    Ri, Rj = Rotation.random(2, random_state=5).as_matrix()
    ti, tj = rng.normal(size=3), rng.normal(size=3)
    ci, cj = cam(Ri, ti, 300.0, 80, 60), cam(Rj, tj, 250.0, 80, 60)
    r = G.pixel_rays(ci)[::37]
    d = rng.uniform(0.1, 1.0, len(r))
    Rji, b = G.relative(ci, cj)
    x, y, zq = G.reproject(r @ Rji.T, b, d, cj)
    Xw = (r / d[:, None] - ti) @ Ri  # world point R_i^T (r / d - t_i)
    Xc = Xw @ Rj.T + tj
    assert np.allclose(x, 250 * Xc[:, 0] / Xc[:, 2] + 40, atol=1e-9)
    assert np.allclose(y, 250 * Xc[:, 1] / Xc[:, 2] + 30, atol=1e-9)
    assert np.allclose(zq / d, Xc[:, 2], rtol=1e-12) if np.all(d > 0) else True


def test_bilinear_exact_on_affine_fields_and_centres():
    rng = np.random.default_rng(4)
    H, W, C = 7, 9, 3
    a, bx, by = rng.normal(size=C), rng.normal(size=C), rng.normal(size=C)
    v, u = np.mgrid[0:H, 0:W]
    F = a + bx * (u[..., None] + 0.5) + by * (v[..., None] + 0.5)  # affine in the pixel-centre coordinates
    x = rng.uniform(0.5, W - 0.5, 200)
    y = rng.uniform(0.5, H - 0.5, 200)
    x[:3] = [W - 0.5, 0.5, W - 0.5]
    y[:3] = [H - 0.5, 0.5, 0.5]
    s = G.bilinear(F, x, y)
    assert np.allclose(s, a + bx * x[:, None] + by * y[:, None], atol=1e-12)
    R = rng.normal(size=(H, W, C))
    assert np.array_equal(G.bilinear(R, u.ravel() + 0.5, v.ravel() + 0.5), R.reshape(-1, C))
    assert G.in_domain(np.array([0.5, W - 0.5, 0.4999]), np.array([0.5, H - 0.5, 1.0]), W, H).tolist() == \
        [True, True, False]


def test_parabola_vertex():
    for k0 in (-0.4, 0.0, 0.27):
        c = [-(k - k0) ** 2 * 3.0 + 5.0 for k in (-1, 0, 1)]
        assert abs(G.fit_peak(*c) - k0) < 1e-14
    assert G.fit_peak(1.0, 1.0, 1.0) == 0.0


def plane_features(ci, cams, Z, channels=16, period=(0.2, 0.6), seed=1):
    """Features of a fronto-parallel plane z = Z (world = reference camera):
    each pixel of each camera sees the plane point along its ray; the feature
    is a smooth random field of that point, unit length, bf16."""
    rng = np.random.default_rng(seed)
    w = rng.normal(size=(6, 2))
    w *= (2 * np.pi / rng.uniform(*period, 6) / np.linalg.norm(w, axis=1))[:, None]
    ph = rng.uniform(0, 2 * np.pi, 6)
    mix = rng.normal(size=(6, channels))
    out = []
    for c in cams:
        W, H = c["width"], c["height"]
        v, u = np.mgrid[0:H, 0:W]
        ray_c = np.stack([(u + 0.5 - c["cx"]) / c["fx"], (v + 0.5 - c["cy"]) / c["fy"], np.ones((H, W))], -1)
        dw = ray_c @ c["R"]  # R^T ray
        centre = -c["R"].T @ c["t"]
        s = (Z - centre[2]) / dw[..., 2]
        P = centre + s[..., None] * dw
        fv = np.sin(P[..., :2] @ w.T + ph) @ mix
        out.append(to_bf16(fv / np.linalg.norm(fv, axis=-1, keepdims=True)))
    return out


def test_depth_recovered_on_textured_plane():
    f, W, H, Z = 400.0, 96, 64, 4.0
    ci = cam(np.eye(3), [0, 0, 0], f, W, H)
    cj = cam(np.eye(3), [-0.3, 0, 0], f, W, H)
    Fi, Fj = plane_features(ci, [ci, cj], Z)
    z_mono = np.full((H, W), Z * 1.15)
    o = G.guided_depth(Fi, [Fj], ci, [cj], z_mono, n_cand=32, margins=True)
    ok = o["nb"] == 0
    # usable iff the segment stays in the map: x - f B d_hi >= 0.5 (disparity moves left)
    d_hi = 1 / (Z * 1.15) + 0.1
    u = np.arange(W) + 0.5
    expect = np.broadcast_to(u - f * 0.3 * d_hi >= 0.5, (H, W))
    assert np.array_equal(ok, expect)
    # error in candidate steps: the nearest candidate alone is 0.45 off for every pixel, a sign-flipped
    # parabola offset 0.85; bilinear interpolation locks some pixels toward whole-pixel disparities
    err = np.abs(1 / o["depth"][ok] - 1 / Z) / o["inv_step"][ok]
    assert np.median(err) < 0.2 and np.quantile(err, 0.95) < 0.5
    assert np.all(o["depth"][~ok] == z_mono[~ok]) and np.all(o["corr"][~ok] == 0)
    assert np.all(o["corr"][ok] > 0.9)  # unit features: the matched ones correlate near 1


def test_adaptive_choice_prefers_longer_segment():
    f, W, H = 200.0, 64, 32
    ci = cam(np.eye(3), [0, 0, 0], f, W, H)
    near = cam(np.eye(3), [-0.05, 0, 0], f, W, H)
    far = cam(np.eye(3), [-0.2, 0, 0], f, W, H)
    Fi = to_bf16(np.ones((H, W, 8)) / math.sqrt(8))
    z = np.full((H, W), 2.0)
    o = G.guided_depth(Fi, [Fi, Fi], ci, [near, far], z, n_cand=8)
    d_hi = 0.6
    u = np.arange(W) + 0.5
    exp = np.where(u - f * 0.2 * d_hi >= 0.5, 1, np.where(u - f * 0.05 * d_hi >= 0.5, 0, -1))
    assert np.array_equal(o["nb"], np.broadcast_to(exp, (H, W)))
    o2 = G.guided_depth(Fi, [Fi, Fi], ci, [far, far], z, n_cand=8)  # equal segments: the lower index
    assert set(np.unique(o2["nb"])) <= {-1, 0}


def test_degenerate_pixels():
    f, W, H = 200.0, 32, 16
    ci = cam(np.eye(3), [0, 0, 0], f, W, H)
    cj = cam(np.eye(3), [-0.1, 0, 0], f, W, H)
    rng = np.random.default_rng(9)
    Fi = to_bf16(rng.normal(size=(H, W, 8)))
    z = np.full((H, W), 3.0)
    z[0, 20], z[1, 20], z[2, 20] = 0.0, np.nan, -1.0
    o = G.guided_depth(Fi, [Fi], ci, [cj], z, n_cand=8)
    assert o["nb"][0, 20] == -1 and o["depth"][0, 20] == 0.0 and o["corr"][0, 20] == 0
    assert o["nb"][1, 20] == -1 and np.isnan(o["depth"][1, 20])
    assert o["nb"][2, 20] == -1 and o["depth"][2, 20] == -1.0
    # behind the neighbour: a camera turned around sees nothing of the segment
    back = cam(np.diag([-1.0, 1.0, -1.0]), [0, 0, 0], f, W, H)
    o = G.guided_depth(Fi, [Fi], ci, [back], np.full((H, W), 3.0), n_cand=8)
    assert np.all(o["nb"] == -1)


def test_maximum_at_window_end_keeps_candidate():
    f, W, H, Z = 400.0, 96, 32, 4.0
    ci = cam(np.eye(3), [0, 0, 0], f, W, H)
    cj = cam(np.eye(3), [-0.3, 0, 0], f, W, H)
    # periods of 1-2 m (100-200 px): the correlation falls monotonically over the 18-42 px shifts of the
    # window [0.4, 0.6], which misses the true 0.25, so the best candidate is d_lo itself
    Fi, Fj = plane_features(ci, [ci, cj], Z, period=(1.0, 2.0))
    z_mono = np.full((H, W), 2.0)
    o = G.guided_depth(Fi, [Fj], ci, [cj], z_mono, n_cand=16)
    ok = o["nb"] == 0
    assert ok.sum() == 24 * H  # columns with u + 0.5 - f B d_hi >= 0.5, d_hi = 0.6
    assert np.all(np.abs(o["depth"][ok] - 1 / 0.4) < 1e-12)
