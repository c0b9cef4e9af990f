"""Brute-force NumPy twin of the tiled compositing, for tiny scenes (<= 64x64
pixels, <= 50 Gaussians).

Test infrastructure only. For every pixel it walks ALL Gaussians in global
(fp32 depth bits, id) order and keeps a Gaussian iff the pixel's tile lies in
the Gaussian's tile rect, then composites front to back exactly as the 3DGS
image-formation model does (alpha = min(alpha_max, o exp(power)), skip below
alpha_min, stop before T drops under t_min). It never builds per-tile lists,
so agreement with the tiled oracle checks the list building and ordering.
Returns colour, final transmittance and the number of composited Gaussians
per pixel.
"""
from __future__ import annotations

import math

import numpy as np


def render(proj: dict, width: int, height: int, tile: int, alpha_min=1 / 255, alpha_max=0.99,
           t_min=1e-4, bg=(0.0, 0.0, 0.0)):
    keys = proj["depth_key"].astype(np.float32).view(np.uint32)
    n = keys.shape[0]
    order = sorted(range(n), key=lambda i: (int(keys[i]), i))
    color = np.zeros((3, height, width))
    t_final = np.ones((height, width))
    n_comp = np.zeros((height, width), np.int32)
    for y in range(height):
        for x in range(width):
            tx, ty = x // tile, y // tile
            T = 1.0
            C = [0.0, 0.0, 0.0]
            for i in order:
                r = proj["rect"][i]
                if not (r[0] <= tx < r[2] and r[1] <= ty < r[3]):
                    continue
                u, v = proj["mean2d"][i]
                a, b, c = proj["conic"][i]
                dx, dy = x + 0.5 - u, y + 0.5 - v
                power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
                if power > 0:
                    continue
                alpha = min(alpha_max, proj["opacity"][i] * math.exp(power))
                if alpha < alpha_min:
                    continue
                nT = T * (1 - alpha)
                if nT < t_min:
                    break
                for ch in range(3):
                    C[ch] += alpha * T * proj["rgb"][i][ch]
                T = nT
                n_comp[y, x] += 1
            for ch in range(3):
                color[ch, y, x] = C[ch] + T * bg[ch]
            t_final[y, x] = T
    return color, t_final, n_comp
