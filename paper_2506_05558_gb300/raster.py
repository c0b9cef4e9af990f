"""Buffer ownership and the training step around the C ABI.

`Rasterizer` holds every device buffer the hot path needs for a fixed Gaussian
count and a fixed list of view sizes, so a step allocates nothing and can be
captured into a CUDA graph. `JointOptimizer` is the paper's per-keyframe loop
body (Sec. 4.3): render every view, L1 loss, adjoint with pose gradients,
sparse Adam on the Gaussians and Adam + SE(3) retraction on the poses.
"""
from __future__ import annotations

import math

import torch

from . import gs


class Rasterizer:
    def __init__(self, n: int, sizes, capacity: int, cfg: gs.gs_config | None = None, device="cuda"):
        self.n = int(n)
        self.sizes = list(sizes)
        self.n_views = len(self.sizes)
        self.cfg = cfg if cfg is not None else gs.config()
        self.f = gs.frame(self.sizes, self.cfg.tile)
        self.items = self.n * self.n_views
        self.n_pix = int(self.f.pix_base[self.n_views])
        self.n_tiles = int(self.f.tile_base[self.n_views])
        self.device = device
        self.proj = gs.Projected.alloc(self.items, device)
        self.img = gs.Image.alloc(self.n_pix, device)
        self.ws_render = gs.workspace(gs.gs_render_workspace_size(self.f), device)
        self.grads = gs.Grads.alloc(self.n, device)
        self.dpose = torch.zeros((self.n_views, 6), dtype=torch.float32, device=device)
        self.set_capacity(capacity)

    def set_capacity(self, capacity: int):
        self.capacity = max(int(capacity), 1)
        # the tile work order is only read by schedules 1 and 2; without it gs_sort skips that sort
        self.pairs = gs.Pairs.alloc(self.items, self.n_tiles, self.capacity, self.device,
                                    with_order=self.cfg.schedule in (1, 2))
        self.ws_sort = gs.workspace(gs.gs_sort_workspace_size(self.n, self.f, self.capacity), self.device)
        self.ws_bwd = gs.workspace(gs.gs_backward_workspace_size(self.n, self.f, self.capacity), self.device)

    # -- stages ---------------------------------------------------------------
    def forward(self, g: gs.Gaussians, cams: torch.Tensor, stream=None):
        gs.gs_project(g, cams, self.f, self.cfg, self.proj, stream)
        gs.gs_sort(self.proj, self.n, self.f, self.pairs, self.ws_sort, stream)
        gs.gs_render_fwd(self.proj, self.pairs, self.f, self.cfg, self.img, self.ws_render, stream)
        return self.img

    def backward(self, g: gs.Gaussians, cams: torch.Tensor, dL_dcolor: torch.Tensor, d_proj=None, stream=None):
        gs.gs_render_bwd(g, cams, self.proj, self.pairs, self.f, self.cfg, self.img, dL_dcolor, self.grads,
                         self.dpose, self.ws_bwd, d_proj, stream)
        return self.grads, self.dpose

    # -- host-side helpers (synchronising; not for the timed loop) ---------------
    def pair_count(self) -> int:
        return int(self.pairs.count.item())

    def status(self) -> int:
        return int(self.pairs.status.item())

    def fit_capacity(self, g: gs.Gaussians, cams: torch.Tensor, slack: float = 1.25) -> int:
        """Runs project + sort once and grows the pair buffer to slack x the
        observed pair count when needed. Returns the pair count."""
        gs.gs_project(g, cams, self.f, self.cfg, self.proj)
        gs.gs_sort(self.proj, self.n, self.f, self.pairs, self.ws_sort)
        torch.cuda.synchronize()
        p = self.pair_count()
        if p > self.capacity:
            self.set_capacity(int(math.ceil(p * slack)) + 1024)
        return p

    def view_color(self, v: int) -> torch.Tensor:
        w, h = self.sizes[v]
        b = 3 * int(self.f.pix_base[v])
        return self.img.color[b:b + 3 * w * h].view(3, h, w)

    def view_pixels(self, t: torch.Tensor, v: int) -> torch.Tensor:
        w, h = self.sizes[v]
        b = int(self.f.pix_base[v])
        return t[b:b + w * h].view(h, w)


def copy_config(cfg: gs.gs_config, **kw) -> gs.gs_config:
    c = gs.gs_config()
    C_bytes = bytes(cfg)
    import ctypes
    ctypes.memmove(ctypes.addressof(c), C_bytes, ctypes.sizeof(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


class JointOptimizer:
    """One iteration = render all views, L1 loss against the targets, adjoint
    (Gaussian and pose gradients), sparse Adam on the visible Gaussians and Adam
    + retraction on the poses. Every stage is a libgs kernel. The step number
    lives on the device, so `capture()` can record one whole iteration into a
    CUDA graph that `replay()` re-launches with no per-kernel host work."""

    def __init__(self, g: gs.Gaussians, cams: torch.Tensor, sizes, targets: torch.Tensor, capacity: int,
                 cfg: gs.gs_config | None = None, adam: gs.gs_adam_config | None = None, lr_pose=(1e-3, 1e-3),
                 device="cuda"):
        self.g = g
        self.cams = cams
        self.r = Rasterizer(g.n, sizes, capacity, cfg, device)
        self.step_dev = torch.ones((1,), dtype=torch.int32, device=device)
        self.graph = None
        self.graphs = []
        self.targets = targets  # flat, same layout as Image.color
        self.m = gs.Gaussians.zeros(g.n, device)
        self.v = gs.Gaussians.zeros(g.n, device)
        self.pm = torch.zeros((self.r.n_views, 6), dtype=torch.float32, device=device)
        self.pv = torch.zeros((self.r.n_views, 6), dtype=torch.float32, device=device)
        self.adam = adam if adam is not None else gs.adam_config()
        self.lr_pose = lr_pose
        self.dL = torch.zeros_like(self.r.img.color)
        self.loss = torch.zeros((1,), dtype=torch.float32, device=device)
        self.ws_loss = gs.workspace(4 * 4096, device)
        self.t = 0

    STAGES = ("project", "sort", "render_fwd", "loss", "composite_bwd", "project_bwd", "adam", "pose")

    def stage_calls(self, stream=None):
        """The iteration as (stage name, call) pairs, in order."""
        r, sd = self.r, self.step_dev
        return [
            ("project", lambda: gs.gs_project(self.g, self.cams, r.f, r.cfg, r.proj, stream)),
            ("sort", lambda: gs.gs_sort(r.proj, r.n, r.f, r.pairs, r.ws_sort, stream)),
            ("render_fwd", lambda: gs.gs_render_fwd(r.proj, r.pairs, r.f, r.cfg, r.img, r.ws_render, stream)),
            ("loss", lambda: gs.gs_l1_loss(r.img.color, self.targets, self.dL, self.loss, self.ws_loss, stream)),
            ("composite_bwd", lambda: gs.gs_composite_bwd(r.proj, r.pairs, r.f, r.cfg, r.img, self.dL, r.n,
                                                          r.ws_bwd, stream)),
            ("project_bwd", lambda: gs.gs_project_bwd(self.g, self.cams, r.proj, r.pairs, r.f, r.cfg, r.grads,
                                                      r.dpose, r.ws_bwd, None, stream)),
            ("adam", lambda: gs.gs_adam_step(self.g, r.grads, self.m, self.v, self.adam, 0, stream, step_dev=sd)),
            ("pose", lambda: (gs.gs_pose_step(self.cams, r.n_views, r.dpose, self.pm, self.pv, self.lr_pose[0],
                                              self.lr_pose[1], 0, stream=stream, step_dev=sd),
                              gs.gs_counter_add(sd, 1, stream))),
        ]

    def set_targets(self, targets: torch.Tensor):
        """Points the loss stage at another target buffer (same shape, dtype and
        device). step() reads it at call time; graphs keep the buffer they were
        captured with."""
        if targets.shape != self.targets.shape or targets.dtype != self.targets.dtype or \
                targets.device != self.targets.device:
            raise ValueError("targets must match the optimiser's target buffer")
        self.targets = targets

    def step(self, stream=None):
        """Enqueues one iteration (the step number advances on the device)."""
        for _, call in self.stage_calls(stream):
            call()
        self.t += 1
        return self.loss

    def capture(self, per_stage: bool = False):
        """Records one iteration into CUDA graphs: one graph for the whole
        iteration, or one per stage (so events can time the stages between
        replays). Call step() once first so every one-time set-up has happened
        outside the capture."""
        self.graphs = []
        calls = self.stage_calls()
        groups = [[c] for c in calls] if per_stage else [calls]
        for grp in groups:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                for _, call in grp:
                    call()
            self.graphs.append((grp[0][0] if per_stage else "step", g))
        self.graph = self.graphs[0][1]

    def replay(self, events=None):
        """Replays the captured iteration; events (len(graphs) + 1 CUDA events)
        are recorded between the graphs when given."""
        for i, (_, g) in enumerate(self.graphs):
            if events is not None:
                events[i].record()
            g.replay()
        if events is not None:
            events[len(self.graphs)].record()
        self.t += 1
        return self.loss

