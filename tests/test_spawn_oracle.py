"""Pins of the direct-spawn-sampling oracle (Sec. 4.2, Eq. 1-3) against facts
fixed outside it: published RNG vectors, exact invariants of Eq. 1-3, the
two-peak response of the LoG norm to a step (Fig. 3), the Laplacian of a
quadratic, the Clark-Evans nearest-neighbour distance behind the scale
formula, and the camera geometry of the back-projected means. CPU only."""
import math
import os

import numpy as np
from scipy.spatial import cKDTree

from oracle import oracle as O
from paper_2506_05558_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answer_vectors():
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        assert list(O.philox4x32_10(w[0:4], w[4:6])) == w[6:10]


def _img(rng, W=64, H=48):
    return rng.random((3, H, W))


def test_penalty_equals_probability_when_render_matches():
    """Eq. 2 on I~ = I gives P~ = P_L, so P_s = 0 and nothing spawns."""
    rng = np.random.default_rng(0)
    im = _img(rng)
    m = O.spawn_maps(im, im, 1.0, 7, 3)
    assert np.array_equal(m["p_pen"], m["p_l"])
    assert np.all(m["p_s"] == 0) and m["mask"].sum() == 0


def test_probability_bounds_and_first_frame():
    rng = np.random.default_rng(1)
    im, rd = _img(rng), _img(rng)
    m = O.spawn_maps(im, rd, 1.0, 7, 3)
    assert np.all(m["p_s"] >= 0) and np.all(m["p_s"] <= m["p_l"]) and np.all(m["p_l"] <= 1)
    first = O.spawn_maps(im, None, 1.0, 7, 3)
    assert np.array_equal(first["p_s"], first["p_l"]) and np.all(first["p_pen"] == 0)
    # the mask is u < P_s with u uniform in [0, 1)
    assert np.all((first["mask"] > 0) == (first["u"] < first["p_s"]))


def test_step_edge_gives_two_peaks():
    """The LoG norm of a step has one peak on each side of the discontinuity,
    a zero on it and nothing away from it (Fig. 3). The step is centred on
    pixel 20 (value halfway there), so the response is odd about it."""
    W, H = 40, 9
    for sigma, want in ((1.0, [19, 21]), (2.0, [18, 22])):
        im = np.zeros((3, H, W))
        im[:, :, 21:] = 0.6
        im[:, :, 20] = 0.3
        m = O.spawn_maps(im, None, sigma, 0, 0)
        row = m["p_l"][4]
        peaks = [x for x in range(1, W - 1) if row[x] > row[x - 1] and row[x] > row[x + 1] and row[x] > 1e-3]
        assert peaks == want, (sigma, peaks)
        assert row[20] < 1e-12
        r = int(np.ceil(3 * sigma))
        assert np.all(row[:20 - r] < 1e-12) and np.all(row[21 + r:] < 1e-12)
        assert np.allclose(row[20 - r:20], row[21:21 + r][::-1], atol=1e-12)  # symmetric about the edge


def test_log_of_quadratic_is_its_laplacian():
    """Away from the border, LoG * (a x^2 + b y^2) = 2a + 2b up to the kernel's
    sampling/truncation error (< 2% at sigma = 1): pins sign and scale."""
    W, H = 41, 41
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    a, b = 1e-4, 3e-4
    im = np.stack([a * (x - 20) ** 2 + b * (y - 20) ** 2] * 3)
    m = O.spawn_maps(im, None, 1.0, 0, 0)
    want = math.sqrt(3) * (2 * a + 2 * b)
    assert abs(m["p_l"][20, 20] - want) < 0.02 * want
    k = O.log_kernel(1.0)
    assert k.shape == (7, 7) and abs(k.sum()) < 1e-15 and k[3, 3] < 0


def test_scale_is_expected_nearest_neighbour_distance():
    """A Bernoulli(p) mask with small p is close to a Poisson process of
    intensity p per px^2, whose mean nearest-neighbour distance is 1/(2 sqrt(p))
    (Clark & Evans 1954): the s' the oracle assigns at P_L = p."""
    W = H = 600
    im = np.zeros((3, H, W))
    m = O.spawn_maps(im, None, 1.0, 12345, 1)
    for p in (0.005, 0.02):
        ys, xs = np.nonzero(m["u"] < p)
        pts = np.stack([xs, ys], 1).astype(np.float64)
        d, _ = cKDTree(pts).query(pts, k=2)
        inner = (xs > 40) & (xs < W - 40) & (ys > 40) & (ys < H - 40)
        mean_nn = d[inner, 1].mean()
        s_px = 1 / (2 * math.sqrt(p))
        assert abs(mean_nn - s_px) < 0.04 * s_px, (p, mean_nn, s_px)


def test_spawned_means_reproject_to_their_pixels():
    rng = np.random.default_rng(2)
    W, H = 48, 40
    im = _img(rng, W, H)
    depth = rng.uniform(2, 8, (H, W))
    depth[5, 5] = -1.0
    R, t = O.retract_pose(np.eye(3), np.zeros(3), [0.3, -0.2, 0.1, 0.2, 0.1, -0.3])
    cam = synth.camera(R, t, 60.0, W, H, dtype=np.float64)
    sp = O.spawn(im, None, depth, cam, 1.0, 99, 4)
    assert len(sp["pixel"]) > 50 and 5 * W + 5 not in set(sp["pixel"].tolist())
    pc = sp["mean"] @ R.T + t
    px = sp["pixel"] % W + 0.5
    py = sp["pixel"] // W + 0.5
    np.testing.assert_allclose(cam["fx"] * pc[:, 0] / pc[:, 2] + cam["cx"], px, atol=1e-9)
    np.testing.assert_allclose(cam["fy"] * pc[:, 1] / pc[:, 2] + cam["cy"], py, atol=1e-9)
    np.testing.assert_allclose(pc[:, 2], depth.reshape(-1)[sp["pixel"]], rtol=1e-12)
    # s = z s' / f, s' = 1 / (2 sqrt(P_L)); colour survives as the SH DC term
    pl = sp["maps"]["p_l"].reshape(-1)[sp["pixel"]]
    np.testing.assert_allclose(np.exp(sp["log_scale"][:, 0]), pc[:, 2] / (2 * np.sqrt(pl) * cam["fx"]), rtol=1e-12)
    rgb = im.reshape(3, -1)[:, sp["pixel"]].T
    np.testing.assert_allclose(0.5 + sp["sh_dc"] / (2 * math.sqrt(math.pi)), rgb, rtol=1e-12)
