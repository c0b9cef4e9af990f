"""FP64 oracle of the learned spawn proposal: a per-patch MLP over 8x8 image
patches (192 pixel values + 2 patch coordinates -> 3 x (Linear 128 + GELU) ->
Linear 3: spawn logit, depth, log-scale offset), its loss against the spawns
that plain direct sampling (Sec. 4.2) produced and kept, the backward pass and
Adam.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).

The paper has no learned proposal; the network is the one the workload
specifies. Arithmetic is FP64; the points where the tensor-core path stores
values in bfloat16 are emulated by rounding there (round to nearest even):
the patch features, the weights, the hidden activations H and the
pre-activation gradients dZ that feed the matrix products. Everything else
(biases, accumulation, GELU and its derivative, the loss) is exact FP64.
"""
from __future__ import annotations

import math

import numpy as np

IN = 194       # 8 x 8 x 3 pixel values + 2 patch coordinates
IN_PAD = 208   # padded to a multiple of 16
HID = 128
OUT = 3        # spawn logit, depth, log-scale
PATCH = 8


def bf16(x):
    """Round to bfloat16 (nearest even) and return as float64. Values are
    first rounded to float32, as the GPU stores float32 before converting."""
    f = np.asarray(x, np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    from scipy.special import erf
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def patch_features(image):
    """image [3][H][W] -> X [n_patches][IN]: row (py, px) in row-major patch
    order holds image[c][8py+dy][8px+dx] at c*64 + dy*8 + dx, then the patch
    centre in [-1, 1]^2 (x first). H and W must be multiples of 8."""
    image = np.asarray(image, np.float64)
    _, H, W = image.shape
    ny, nx = H // PATCH, W // PATCH
    t = image.reshape(3, ny, PATCH, nx, PATCH).transpose(1, 3, 0, 2, 4).reshape(ny * nx, 192)
    py, px = np.divmod(np.arange(ny * nx), nx)
    cx = (px + 0.5) / nx * 2.0 - 1.0
    cy = (py + 0.5) / ny * 2.0 - 1.0
    return np.concatenate([t, cx[:, None], cy[:, None]], 1)


def init_params(rng, scale=1.0):
    """W_l [out][in] (nn.Linear layout), b_l [out]; uniform(-1/sqrt(in), 1/sqrt(in))."""
    dims = [(HID, IN), (HID, HID), (HID, HID), (OUT, HID)]
    ps = []
    for o, i in dims:
        a = scale / math.sqrt(i)
        ps.append((rng.uniform(-a, a, (o, i)), rng.uniform(-a, a, o)))
    return ps


def forward(params, X):
    """Returns (Y [M][3], cache). Matrix inputs are bfloat16-rounded."""
    H = bf16(X)
    cache = {"H0": H, "Z": []}
    for l, (W, b) in enumerate(params):
        Z = H @ bf16(W).T + b
        cache["Z"].append(Z)
        if l < 3:
            H = bf16(gelu(Z))
            cache[f"H{l + 1}"] = H
    return Z, cache


def loss(Y, t_spawn, z_target, s_target, mask, w_depth=1.0, w_scale=1.0):
    """Mean over patches of BCE(sigmoid(logit), t_spawn) plus weighted L1 on
    depth and log-scale where mask (the patch kept at least one spawn).
    Returns (loss, dL/dY)."""
    M = Y.shape[0]
    logit, depth, ls = Y[:, 0], Y[:, 1], Y[:, 2]
    sp = np.logaddexp(0.0, logit)
    L = (sp - t_spawn * logit).sum() / M
    L += w_depth * (mask * np.abs(depth - z_target)).sum() / M
    L += w_scale * (mask * np.abs(ls - s_target)).sum() / M
    dY = np.zeros_like(Y)
    dY[:, 0] = (1.0 / (1.0 + np.exp(-logit)) - t_spawn) / M
    dY[:, 1] = w_depth * mask * np.sign(depth - z_target) / M
    dY[:, 2] = w_scale * mask * np.sign(ls - s_target) / M
    return float(L), dY


def backward(params, cache, dY):
    """Gradients [(dW_l, db_l)] for dL/dY. The matrix-product inputs dZ are
    bfloat16-rounded (as the tensor-core path stores them); db is the FP64 sum
    of the unrounded dZ."""
    grads = [None] * 4
    G = dY
    for l in range(3, -1, -1):
        W, _ = params[l]
        Hin = cache[f"H{l}"]
        Gb = bf16(G)
        grads[l] = (Gb.T @ Hin, G.sum(0))
        if l > 0:
            dH = Gb @ bf16(W)
            G = dH * gelu_grad(cache["Z"][l - 1])
    return grads


def adam(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam with bias correction on the FP64 master weights."""
    out_p, out_m, out_v = [], [], []
    for (W, b), (dW, db), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        res = []
        for p, g, mm, vv in ((W, dW, mW, vW), (b, db, mb, vb)):
            mm = beta1 * mm + (1 - beta1) * g
            vv = beta2 * vv + (1 - beta2) * g * g
            p = p - lr * (mm / (1 - beta1 ** step)) / (np.sqrt(vv / (1 - beta2 ** step)) + eps)
            res.append((p, mm, vv))
        out_p.append((res[0][0], res[1][0]))
        out_m.append((res[0][1], res[1][1]))
        out_v.append((res[0][2], res[1][2]))
    return out_p, out_m, out_v


def zeros_like_params(params):
    return [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]


# ---------------------------------------------------------------------------
# Targets from direct sampling and spawning from the network's predictions
# ---------------------------------------------------------------------------

def targets_from_spawns(pixel, depth, log_scale, kept, W, H):
    """Per 8x8 patch: (kept count / 64, mean depth, mean log_scale value, any
    kept) over the spawned Gaussians that were kept after the frame's
    optimisation (log_scale: whatever per-spawn scale quantity the network is
    to predict, e.g. the change the optimisation made to the log-scale)."""
    nx, ny = W // PATCH, H // PATCH
    out = np.zeros((nx * ny, 4))
    pixel = np.asarray(pixel)
    keep = np.asarray(kept, bool)
    for p, z, s in zip(pixel[keep], np.asarray(depth)[keep], np.asarray(log_scale)[keep]):
        m = (p // W // PATCH) * nx + (p % W) // PATCH
        out[m, 0] += 1
        out[m, 1] += z
        out[m, 2] += s
    has = out[:, 0] > 0
    out[has, 1] /= out[has, 0]
    out[has, 2] /= out[has, 0]
    out[:, 3] = has
    out[:, 0] /= PATCH * PATCH
    return out


def targets_from_rows(pixel, mean_opa, scale, scale0, cam, keep_threshold, W, H):
    """Targets from one frame's spawns after its optimisation (Sec. 4.2: the
    primitives direct sampling produces and keeps): spawn i is kept when
    sigmoid(opacity logit) > keep_threshold; its depth is the camera depth
    R_2 . mu + t_2 of its optimised mean; its log-scale value is the mean of
    its three optimised log-scales minus its log-scale when spawned. Returns
    (targets as targets_from_spawns, the spawns' opacities) in FP64."""
    mo = np.asarray(mean_opa, np.float64)
    sc = np.asarray(scale, np.float64)
    R = np.asarray(cam["R"], np.float64).reshape(3, 3)
    t = np.asarray(cam["t"], np.float64)
    opa = 1.0 / (1.0 + np.exp(-mo[:, 3]))
    kept = opa > keep_threshold
    z = mo[:, :3] @ R[2] + t[2]
    ls = sc[:, :3].mean(1) - np.asarray(scale0, np.float64)[:, 0]
    return targets_from_spawns(pixel, z, ls, kept, W, H), opa


PATCH_FLOOR = 64 * 1e-3  # lower bound of a patch's P_s sum in the placement ratio


def spawn_learned(image, mlp_out, cam, seed, frame, depth=None, render=None, sigma=1.0):
    """Spawning from the network's per-patch outputs with direct sampling's
    placement: pixel p of patch m spawns with probability
    min(1, sigmoid(logit_m) * 64 * P_s(p) / max(sum_{q in m} P_s(q), 0.064)),
    P_s the spawn probability of Eq. 3 (render penalty included), so the patch
    receives on average the network's predicted number of kept spawns where
    direct sampling would have placed them. The draw u is the Philox output of
    counter (p, frame, 1, 0); the pixel spawns iff u < probability and its depth
    is positive. The depth is the map's value where a map is given and that
    value is positive and finite, else the patch's predicted depth. The
    Gaussian sits at the pixel centre at that depth z with, on all axes, direct
    sampling's log-scale log(z / (2 fx sqrt(P_L(p)))) plus the patch's predicted
    log-scale offset, identity rotation, opacity 0.5 and the pixel colour as SH
    DC. Returns the spawns in pixel order and, as `amb`, the pixels whose
    decision an FP32 evaluation may take the other way (|u - probability|
    within a bound of the FP32 errors of P_s and of the patch sum)."""
    from . import oracle as O
    image = np.asarray(image, np.float64)
    _, H, W = image.shape
    nx = W // PATCH
    maps = O.spawn_maps(image, render, sigma, seed, frame)
    ps = maps["p_s"].reshape(-1)
    u = O.philox_uniforms(W * H, frame, 1, seed)
    p = np.arange(W * H)
    x, y = p % W, p // W
    m = (y // PATCH) * nx + x // PATCH
    S = np.bincount(m, weights=ps, minlength=nx * (H // PATCH))
    Sf = np.maximum(S, PATCH_FLOOR)[m]
    out = np.asarray(mlp_out, np.float64)
    sig = 1.0 / (1.0 + np.exp(-out[m, 0]))
    prob = np.minimum(1.0, sig * 64.0 * ps / Sf)
    z = out[m, 1]
    if depth is not None:
        d = np.asarray(depth, np.float64).reshape(-1)
        use = np.isfinite(d) & (d > 0)
        z = np.where(use, d, z)
    spawn = (u < prob) & (z > 0)
    # FP32 P_s is within ~2e-6 of the FP64 value (P_L <= 1) and the patch sum
    # within 64 times that; propagate through the ratio
    err = sig * 64.0 / Sf * (2e-6 + 128e-6 * ps / Sf) + 2e-6
    amb = np.abs(u - prob) < err
    idx = np.nonzero(spawn)[0]
    zi = z[idx]
    pc = np.stack([(x[idx] + 0.5 - cam["cx"]) * zi / cam["fx"], (y[idx] + 0.5 - cam["cy"]) * zi / cam["fy"], zi], 1)
    R = np.asarray(cam["R"], np.float64)
    t = np.asarray(cam["t"], np.float64)
    mu = (pc - t) @ R
    c0 = 0.5 / math.sqrt(math.pi)
    rgb = image.reshape(3, -1)[:, idx].T
    pl = maps["p_l"].reshape(-1)[idx]
    ls = np.log(zi / (2.0 * np.sqrt(pl)) / cam["fx"]) + out[m[idx], 2]
    return dict(pixel=idx, mean=mu, log_scale=np.repeat(ls[:, None], 3, 1), sh_dc=(rgb - 0.5) / c0, amb=amb,
                prob=prob)
