"""FP64 oracle of the learned spawn proposal: a per-patch MLP over 8x8 image
patches (192 pixel values + 2 patch coordinates -> 3 x (Linear 128 + GELU) ->
Linear 3: spawn logit, depth, log-scale), its loss against the spawns that
plain direct sampling (Sec. 4.2) produced and kept, the backward pass and
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
