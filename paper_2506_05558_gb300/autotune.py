"""Picks the tile size, the per-round batch depths of the compositing kernels
and the render schedule for one workload by timing the forward + adjoint on
the GPU (coordinate descent over the launch configurations libgs builds).

The knobs change only how the work is laid out: tile size changes the tile
lists (every candidate is a correct render, checked against the oracle at
tiles 8, 16 and 32 by the parity tests); batch depth and schedule change only
the kernels' staging and work order.
"""
from __future__ import annotations

import torch

from . import gs
from .raster import Rasterizer, copy_config

FWD_BATCHES = {8: (64, 128, 256), 16: (64, 128, 256), 32: (128, 256)}
BWD_BATCHES = {8: (64, 128, 256), 16: (32, 64, 128), 32: (32,)}
TILES = (8, 16, 32)


def time_config(g: gs.Gaussians, cams: torch.Tensor, sizes, targets: torch.Tensor, cfg: gs.gs_config,
                steps: int = 3, device="cuda") -> float:
    """Milliseconds per forward + loss + adjoint of all views under cfg."""
    r = Rasterizer(g.n, sizes, 1 << 20, cfg, device)
    r.fit_capacity(g, cams)
    dL = torch.empty_like(r.img.color)
    loss = torch.zeros((1,), device=device)
    ws = gs.workspace(4 * 4096, device)

    def once():
        r.forward(g, cams)
        gs.gs_l1_loss(r.img.color, targets, dL, loss, ws)
        r.backward(g, cams, dL)

    once()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        once()
    b.record()
    torch.cuda.synchronize()
    ok = r.status() == gs.GS_OK
    del r
    return a.elapsed_time(b) / steps if ok else float("inf")


def tune(g: gs.Gaussians, cams: torch.Tensor, sizes, targets: torch.Tensor, base: gs.gs_config, steps: int = 3,
         device="cuda", log=None):
    """Returns (best config, table of (tile, fwd_batch, bwd_batch, schedule, ms))."""
    table = []

    def run(tile, fb, bb, sched):
        cfg = copy_config(base, tile=tile, fwd_batch=fb, bwd_batch=bb, schedule=sched)
        ms = time_config(g, cams, sizes, targets, cfg, steps, device)
        table.append((tile, fb, bb, sched, ms))
        if log:
            log(f"autotune tile={tile} fwd_batch={fb} bwd_batch={bb} schedule={sched}: {ms:.3f} ms")
        return ms

    best = None
    for tile in TILES:
        ms = run(tile, 0, 0, 0)
        if best is None or ms < best[-1]:
            best = (tile, 0, 0, 0, ms)
    tile = best[0]
    for sched in (1, 2):
        ms = run(tile, 0, 0, sched)
        if ms < best[-1]:
            best = (tile, 0, 0, sched, ms)
    sched = best[3]
    for fb in FWD_BATCHES[tile]:
        ms = run(tile, fb, 0, sched)
        if ms < best[-1]:
            best = (tile, fb, 0, sched, ms)
    fb = best[1]
    for bb in BWD_BATCHES[tile]:
        ms = run(tile, fb, bb, sched)
        if ms < best[-1]:
            best = (tile, fb, bb, sched, ms)
    tile, fb, bb, sched, _ = best
    return copy_config(base, tile=tile, fwd_batch=fb, bwd_batch=bb, schedule=sched), table
