"""Pins of the learned-proposal MLP oracle (CPU): bfloat16 rounding against
torch's bfloat16 conversion, GELU against torch, the whole-network gradient
against central finite differences of the loss (with the rounding turned off),
the patch layout against a direct loop, and Adam's first step."""
import math

import numpy as np
import pytest
import torch

from oracle import mlp as M


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(10000) * 10 ** rng.uniform(-8, 8, 10000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.0039063, 3.0e38]])
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16(x), want)


def test_gelu_matches_torch():
    z = np.linspace(-8, 8, 2001)
    t = torch.tensor(z, dtype=torch.float64, requires_grad=True)
    y = torch.nn.functional.gelu(t)
    y.sum().backward()
    np.testing.assert_allclose(M.gelu(z), y.detach().numpy(), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(M.gelu_grad(z), t.grad.numpy(), rtol=1e-12, atol=1e-14)


def test_patch_features_layout():
    rng = np.random.default_rng(1)
    im = rng.random((3, 16, 24))
    X = M.patch_features(im)
    assert X.shape == (6, 194)
    for py in range(2):
        for px in range(3):
            row = X[py * 3 + px]
            for c in range(3):
                for dy in range(8):
                    for dx in range(8):
                        assert row[c * 64 + dy * 8 + dx] == im[c, 8 * py + dy, 8 * px + dx]
            assert row[192] == (px + 0.5) / 3 * 2 - 1 and row[193] == (py + 0.5) / 2 * 2 - 1


def test_gradients_match_central_differences(monkeypatch):
    """With the bfloat16 rounding disabled the network is smooth: every
    parameter's gradient equals the central difference of the loss."""
    monkeypatch.setattr(M, "bf16", lambda x: np.asarray(x, np.float64))
    rng = np.random.default_rng(2)
    params = M.init_params(rng)
    X = rng.standard_normal((20, M.IN))
    t = rng.random(20)
    zt, st = rng.normal(5, 1, 20), rng.normal(-3, 0.5, 20)
    mask = (rng.random(20) < 0.7).astype(float)
    Y, cache = M.forward(params, X)
    # keep L1 terms away from their kinks
    zt += np.sign(Y[:, 1] - zt) * 0.1
    st += np.sign(Y[:, 2] - st) * 0.1
    L, dY = M.loss(Y, t, zt, st, mask)
    grads = M.backward(params, cache, dY)
    h = 1e-6
    for l in range(4):
        for which in (0, 1):
            arr = params[l][which]
            flat = arr.reshape(-1)
            for idx in rng.choice(flat.size, min(6, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + h
                lp = M.loss(M.forward(params, X)[0], t, zt, st, mask)[0]
                flat[idx] = old - h
                lm = M.loss(M.forward(params, X)[0], t, zt, st, mask)[0]
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                an = grads[l][which].reshape(-1)[idx]
                assert abs(fd - an) <= 1e-5 * max(1e-3, abs(fd)), (l, which, idx, fd, an)


def test_loss_closed_form():
    Y = np.array([[0.0, 2.0, -1.0], [2.0, 1.0, 0.5]])
    L, dY = M.loss(Y, np.array([0.5, 1.0]), np.array([1.0, 1.0]), np.array([0.0, 0.0]), np.array([1.0, 0.0]))
    want = (math.log(2) - 0 + math.log(1 + math.e ** 2) - 2) / 2 + (1.0 + 1.0) / 2
    assert abs(L - want) < 1e-14
    assert abs(dY[0, 0] - 0.0) < 1e-15 and abs(dY[1, 0] - (1 / (1 + math.e ** -2) - 1) / 2) < 1e-15


def test_adam_first_step_is_sign():
    rng = np.random.default_rng(3)
    params = M.init_params(rng)
    grads = [(rng.standard_normal(W.shape), rng.standard_normal(b.shape)) for W, b in params]
    z = M.zeros_like_params(params)
    p2, _, _ = M.adam(params, grads, z, z, 1, 1e-3, eps=1e-12)
    for (W, b), (W2, b2), (dW, db) in zip(params, p2, grads):
        np.testing.assert_allclose(W2, W - 1e-3 * np.sign(dW), rtol=0, atol=1e-9)


def test_targets_from_spawns_hand_case():
    """Two 8x8 patches of a 16x8 frame; values written out by hand."""
    W, H = 16, 8
    # pixels: (x, y) -> p = y W + x; patch 0 = x < 8, patch 1 = x >= 8
    pixel = np.array([0 * W + 1, 3 * W + 7, 5 * W + 2, 2 * W + 9, 7 * W + 15])
    depth = np.array([2.0, 4.0, 100.0, 6.0, 8.0])
    ls = np.array([-3.0, -5.0, 7.0, -2.0, -4.0])
    kept = np.array([1, 1, 0, 0, 1])
    t = M.targets_from_spawns(pixel, depth, ls, kept, W, H)
    np.testing.assert_array_equal(t, [[2 / 64, 3.0, -4.0, 1.0], [1 / 64, 8.0, -4.0, 1.0]])
    t0 = M.targets_from_spawns(pixel, depth, ls, np.zeros(5), W, H)
    np.testing.assert_array_equal(t0, np.zeros((2, 4)))


def test_targets_from_rows_hand_case():
    """Kept by opacity, camera depth and log-scale change of optimised rows,
    by hand: camera R = rotation about y by 90 degrees (row 2 of R = (-1, 0, 0)),
    t = (0, 0, 5): z = 5 - mu_x; opacity logits 0 (0.5), -4 (0.018) and 2 (0.88)
    against the threshold 0.05."""
    W, H = 16, 8
    c, s_ = 0.0, 1.0
    cam = dict(R=np.array([[c, 0, s_], [0, 1, 0], [-s_, 0, c]]), t=np.array([0.0, 0.0, 5.0]))
    pixel = np.array([0 * W + 1, 3 * W + 7, 2 * W + 9])
    mean_opa = np.array([[1.0, 9.0, 9.0, 0.0], [2.0, 0.0, 0.0, -4.0], [-3.0, 1.0, 1.0, 2.0]])
    scale = np.array([[-3.0, -4.0, -5.0, 0.0], [0.0, 0.0, 0.0, 0.0], [-1.0, -1.0, -4.0, 0.0]])
    scale0 = np.array([[-3.5, -3.5, -3.5, 0.0], [-1.0, -1.0, -1.0, 0.0], [-2.5, -2.5, -2.5, 0.0]])
    t, opa = M.targets_from_rows(pixel, mean_opa, scale, scale0, cam, 0.05, W, H)
    np.testing.assert_allclose(opa, [0.5, 1 / (1 + np.exp(4.0)), 1 / (1 + np.exp(-2.0))], rtol=1e-15)
    # spawn 0 kept in patch 0: z = 5 - 1 = 4, ls = -4 + 3.5 = -0.5; spawn 1 dropped (0.018);
    # spawn 2 kept in patch 1: z = 5 + 3 = 8, ls = -2 + 2.5 = 0.5
    np.testing.assert_allclose(t, [[1 / 64, 4.0, -0.5, 1.0], [1 / 64, 8.0, 0.5, 1.0]], rtol=1e-14, atol=1e-14)


def _pin_cam(W, H):
    from oracle import oracle as O
    from paper_2506_05558_gb300 import synth
    R, t = O.retract_pose(np.eye(3), np.zeros(3), [0.3, -0.2, 0.1, 0.05, -0.1, 0.2])
    return synth.camera(R, t, 50.0, W, H, dtype=np.float64)


def _textured(rng, W, H):
    """An image with detail everywhere (sum of random sinusoids + noise), so
    every 8x8 patch has a positive LoG response."""
    yy, xx = np.mgrid[0:H, 0:W]
    img = np.zeros((3, H, W))
    for c in range(3):
        for _ in range(4):
            f = rng.uniform(0.2, 1.2, 2)
            img[c] += 0.1 * np.sin(f[0] * xx + f[1] * yy + rng.uniform(0, 6))
    return np.clip(0.5 + img + rng.normal(0, 0.02, img.shape), 0, 1)


def test_spawn_learned_expected_count_and_placement():
    """Without saturation the probabilities of a patch sum to 64 sigmoid(logit)
    (the predicted count) and are proportional to P_s (Eq. 3) inside the patch;
    a render equal to the image (P_s = 0) spawns nothing; logit -40 spawns
    nothing. Spawned means reproject to their pixel centres at the chosen depth
    (projection written here independently), the depth map wins where valid,
    and SH DC gives back the pixel colour."""
    from oracle import oracle as O
    rng = np.random.default_rng(0)
    W, H = 32, 24
    n_p = (W // 8) * (H // 8)
    cam = _pin_cam(W, H)
    image = _textured(rng, W, H)
    out = np.stack([rng.uniform(-4, -2, n_p), rng.uniform(1, 9, n_p), np.full(n_p, -4.0)], 1)
    out[1, 1] = -2.0  # a patch with a negative predicted depth (log-scale offset -4 everywhere)
    depth = rng.uniform(2, 12, (H, W))
    depth[rng.random((H, W)) < 0.3] = 0.0  # holes fall back to the prediction
    ps = O.spawn_maps(image, None, 1.0, 5, 3)["p_s"]
    for dmap in (None, depth):
        r = M.spawn_learned(image, out, cam, 5, 3, depth=dmap)
        prob = r["prob"].reshape(H // 8, 8, W // 8, 8).transpose(0, 2, 1, 3).reshape(n_p, 64)
        psp = ps.reshape(H // 8, 8, W // 8, 8).transpose(0, 2, 1, 3).reshape(n_p, 64)
        sig = 1 / (1 + np.exp(-out[:, 0]))
        assert (psp.sum(1) > M.PATCH_FLOOR).all() and (prob < 1).all()
        np.testing.assert_allclose(prob.sum(1), 64 * sig, rtol=1e-12)
        np.testing.assert_allclose(prob / psp, np.repeat((prob.sum(1) / psp.sum(1))[:, None], 64, 1), rtol=1e-12)
        p = np.arange(W * H)
        x, y = p % W, p // W
        m = (y // 8) * (W // 8) + x // 8
        z = out[m, 1] if dmap is None else np.where(depth.reshape(-1) > 0, depth.reshape(-1), out[m, 1])
        u = O.philox_uniforms(W * H, 3, 1, 5)
        want = p[(u < r["prob"]) & (z > 0)]
        np.testing.assert_array_equal(r["pixel"], want)
        zi = z[want]
        q = r["mean"] @ np.asarray(cam["R"]).T + np.asarray(cam["t"])
        np.testing.assert_allclose(q[:, 2], zi, rtol=1e-12)
        np.testing.assert_allclose(cam["fx"] * q[:, 0] / q[:, 2] + cam["cx"], x[want] + 0.5, atol=1e-9)
        np.testing.assert_allclose(cam["fy"] * q[:, 1] / q[:, 2] + cam["cy"], y[want] + 0.5, atol=1e-9)
        np.testing.assert_allclose(r["sh_dc"] * (0.5 / math.sqrt(math.pi)) + 0.5, image.reshape(3, -1)[:, want].T,
                                   atol=1e-12)
        # direct sampling's scale at the same pixel and depth (the plain oracle, whose draws
        # differ: pool its spawns over several frames), times exp(offset)
        plain_ls = {}
        for fr in range(12):
            pl = O.spawn(image, None, z.reshape(H, W), cam, 1.0, 5, fr)
            plain_ls.update(zip(pl["pixel"].tolist(), pl["log_scale"][:, 0].tolist()))
        both = [i for i, px in enumerate(want.tolist()) if px in plain_ls]
        assert len(both) > 0.5 * want.size
        np.testing.assert_allclose(r["log_scale"][both, 0], np.array([plain_ls[want[i]] for i in both]) - 4.0,
                                   rtol=1e-12)
    assert M.spawn_learned(image, out, cam, 5, 3, render=image)["pixel"].size == 0
    out[:, 0] = -40.0
    assert M.spawn_learned(image, out, cam, 5, 3)["pixel"].size == 0


def test_spawn_learned_count_follows_the_logit():
    """Over a 256x256 textured frame the number of spawns matches the sum of
    the probabilities (= 64 sigmoid(logit) per unsaturated patch) within 4
    standard deviations of the Poisson-binomial count."""
    rng = np.random.default_rng(1)
    W, H = 256, 256
    cam = _pin_cam(W, H)
    n_p = (W // 8) * (H // 8)
    image = _textured(rng, W, H)
    for logit in (-3.0, -2.0):
        out = np.stack([np.full(n_p, logit), np.full(n_p, 5.0), np.zeros(n_p)], 1)
        r = M.spawn_learned(image, out, cam, 11, 2)
        mean, var = r["prob"].sum(), (r["prob"] * (1 - r["prob"])).sum()
        assert abs(r["pixel"].size - mean) < 4 * math.sqrt(var), (logit, r["pixel"].size, mean)
        assert abs(mean - 64 * n_p / (1 + math.exp(-logit))) < 0.02 * mean
