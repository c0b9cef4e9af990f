"""Frame-by-frame reconstruction loop (Sec. 4.2-4.4) with known poses, used to
compare plain direct spawn sampling with the learned spawn proposal, with
anchors (Sec. 4.4): when more than 40% of the active Gaussians are below one
pixel from the previous camera, the active set and its Adam state are copied
to pinned host memory as an anchor at that camera's centre and the set is
coarsened by merging; novel views render the closest anchor, blending the two
closest when their distances are similar.

Per new frame: render the active Gaussians from its pose (the penalty image
of Eq. 2), spawn new Gaussians (direct sampling with the frame's depth map, or
the learned per-patch proposal), append them, run the joint optimisation over
a sliding window of recent frames, mark which of the frame's spawns survived
(opacity above a threshold), turn those into per-patch training targets for
the learned proposal and train it on the frame, and test the anchor rule from
the previous camera. Every step is a libgs call; PyTorch only owns memory.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import gs
from .raster import Rasterizer


class Anchor:
    """An anchor: its location (camera centre) and the active set stored there
    (pinned host copies of the Gaussians and their Adam moments)."""

    def __init__(self, location, store: "GaussianStore"):
        n = store.n
        self.location = np.asarray(location, np.float64)
        self.n = n
        self.p, self.m, self.v = gs.pinned_gaussians(n), gs.pinned_gaussians(n), gs.pinned_gaussians(n)
        g, m, v = store.active()
        gs.gs_anchor_offload(g, m, v, self.p, self.m, self.v)

    def load(self, device="cuda") -> gs.Gaussians:
        g = gs.Gaussians.zeros(self.n, device)
        gs.gs_anchor_load(self.p, None, None, g, None, None)
        return g


def camera_centre(cam: torch.Tensor):
    c = gs.cameras_from_tensor(cam)[0]
    return -np.asarray(c["R"], np.float64).T @ np.asarray(c["t"], np.float64)


class GaussianStore:
    """Preallocated Gaussians, Adam moments and an active count."""

    def __init__(self, capacity: int, device="cuda"):
        self.cap = capacity
        self.p = gs.Gaussians.zeros(capacity, device)
        self.m = gs.Gaussians.zeros(capacity, device)
        self.v = gs.Gaussians.zeros(capacity, device)
        self.lr = torch.ones((capacity,), dtype=torch.float32, device=device)  # per-Gaussian rate multipliers
        self.n = 0

    @staticmethod
    def _view(g: gs.Gaussians, n: int) -> gs.Gaussians:
        return gs.Gaussians(g.mean_opa[:n], g.scale[:n], g.quat[:n], g.sh[:n])

    def active(self):
        return self._view(self.p, self.n), self._view(self.m, self.n), self._view(self.v, self.n)

    def append(self, sp: gs.Spawned, k: int) -> int:
        k = min(k, self.cap - self.n)
        if k <= 0:
            return 0
        for dst, src in ((self.p.mean_opa, sp.g.mean_opa), (self.p.scale, sp.g.scale), (self.p.quat, sp.g.quat),
                         (self.p.sh, sp.g.sh)):
            dst[self.n:self.n + k].copy_(src[:k])
        for st in (self.m, self.v):
            for t in (st.mean_opa, st.scale, st.quat, st.sh):
                t[self.n:self.n + k].zero_()
        self.lr[self.n:self.n + k] = 1.0  # rates start fresh when a Gaussian is introduced
        self.n += k
        return k


def psnr(a: torch.Tensor, b: torch.Tensor) -> float:
    mse = torch.mean((a.clamp(0, 1) - b) ** 2).item()
    return 10 * math.log10(1.0 / max(mse, 1e-12))


def render_depth(g: gs.Gaussians, cam: torch.Tensor, size, cfg, device="cuda"):
    """Colour image and expected depth per pixel (the depth integral of the
    forward pass normalised by 1 - T_final; 0 where less than half the pixel is
    covered)."""
    r = Rasterizer(g.n, [size], 1 << 20, cfg, device)
    r.img.depth = torch.zeros_like(r.img.t_final)
    r.fit_capacity(g, cam)
    r.forward(g, cam)
    acc = (1.0 - r.img.t_final).clamp_min(1e-6)
    depth = r.img.depth / acc
    depth[acc < 0.5] = 0.0  # no reliable depth where little was rendered
    return r.img.color.clone(), depth


class OnTheFly:
    def __init__(self, capacity: int, size, window: int = 4, iters: int = 30, mode: str = "plain",
                 mlp_warmup_frames: int = 3, mlp_steps: int = 40, keep_threshold: float = 0.05, seed: int = 7,
                 anchor_tau: float = 1.0, anchor_share: float = 0.4, merge_radius: float = 0.5,
                 coarse_to_fine: int = 0, mip_filter: bool = False, lr_decay: float = 1.0,
                 min_opacity: float = 0.0, guided_neighbours: int = 0, learned_depth: str = "map",
                 mlp_online: bool = False, device="cuda"):
        self.store = GaussianStore(capacity, device)
        self.W, self.H = size
        self.window = window
        self.iters = iters
        self.mode = mode
        # coarse_to_fine = l: a new frame is first trained at 2^l downsampling, l
        # decremented every five iterations (Sec. 4.3); mip_filter: the
        # integral-keeping 2-D filter that makes the multi-scale training consistent
        self.c2f = coarse_to_fine
        self.cfg = gs.config(sh_degree=0, mip_filter=1, dilation=0.1) if mip_filter else gs.config(sh_degree=0)
        self.min_opacity = min_opacity
        self.adam = gs.adam_config(decay=lr_decay, lr_mean=1e-3, lr_opacity=0.05, lr_scale=5e-3, lr_rot=1e-3, lr_sh_dc=5e-3,
                                   lr_sh_rest=0.0)
        self.frames = []  # [image [3HW], camera tensor, coarse-to-fine level]
        self.seed = seed
        self.device = device
        self.keep_threshold = keep_threshold
        # learned spawning takes its depth from the frame's map where valid ("map") or
        # from the network everywhere ("predicted"); with mlp_online the network keeps
        # training on each frame's kept spawns after the warm-up frames
        self.learned_depth = learned_depth
        self.mlp_online = mlp_online
        self.mlp_warmup_frames = mlp_warmup_frames
        self.mlp_steps = mlp_steps
        hw = self.W * self.H
        self.spawned = gs.Spawned.alloc(hw, hw, device)
        self.ws_spawn = gs.workspace(gs.gs_spawn_workspace_size(self.W, self.H), device)
        self.iter_count = 0
        self.step_dev = torch.ones((1,), dtype=torch.int32, device=device)
        if mode == "learned":
            rng = np.random.default_rng(seed)
            layers = [(rng.uniform(-1, 1, (o, i)) / math.sqrt(i), rng.uniform(-1, 1, o) / math.sqrt(i))
                      for o, i in ((128, 194), (128, 128), (128, 128), (3, 128))]
            self.mlp = gs.MlpParams.from_numpy(layers, device)
            self.mlp_m, self.mlp_v = gs.MlpParams.zeros(device), gs.MlpParams.zeros(device)
            self.n_patches = gs.gs_mlp_patches(self.W, self.H)
            self.ws_mlp = gs.workspace(gs.gs_mlp_workspace_size(self.n_patches), device)
            self.mlp_out = torch.zeros((self.n_patches, 3), device=device)
            self.mlp_targets = torch.zeros((self.n_patches, 4), device=device)
            self.ws_tg = gs.workspace(gs.gs_mlp_targets_workspace_size(self.W, self.H), device)
            self.mlp_loss = torch.zeros(1, device=device)
            self.mlp_cfg = gs.mlp_config(tensor_path=1, lr=1e-3)
            self.mlp_step = 0
        self.log = []
        self.anchors: list[Anchor] = []
        self.prev_cam = None
        self.anchor_tau = anchor_tau
        self.anchor_share = anchor_share
        self.merge_radius = merge_radius
        self.too_fine = torch.zeros((capacity,), dtype=torch.uint8, device=device)
        self.count = torch.zeros((1,), dtype=torch.int64, device=device)
        # guided matching (App. A.2): the given depth of a new frame is a monocular
        # estimate, refined against the feature maps of up to this many earlier frames
        self.guided_neighbours = guided_neighbours
        self.feat_frames = []  # (feature map [H][W][C] bf16 bits, camera)

    # -- anchors -------------------------------------------------------------------
    def _maybe_anchor(self, frame_idx):
        """Anchor rule from the previous camera; on trigger, store the active set
        at an anchor and merge the too-fine Gaussians. Returns the merge log."""
        if self.prev_cam is None or self.store.n == 0 or self.anchor_tau <= 0:
            return None
        g, m, v = self.store.active()
        fine = self.too_fine[:g.n]
        gs.gs_anchor_check(g, self.prev_cam, self.anchor_tau, fine, self.count)
        cnt = int(self.count.item())
        if cnt <= self.anchor_share * g.n:
            return None
        self.anchors.append(Anchor(camera_centre(self.prev_cam), self.store))
        out = GaussianStore(self.store.cap, self.device)
        n_out = torch.zeros((1,), dtype=torch.int64, device=self.device)
        ws = gs.workspace(gs.gs_anchor_merge_workspace_size(g.n, 3), self.device)
        go, mo, vo = out.p, out.m, out.v
        gs.gs_anchor_merge(g, fine, self.merge_radius, self.seed * 7919 + frame_idx, go, n_out, ws, m=m, v=v,
                           m_out=mo, v_out=vo, lr=self.store.lr[:g.n], lr_out=out.lr)
        out.n = int(n_out.item())
        before = g.n
        self.store = out
        return dict(frame=frame_idx, too_fine=cnt, before=before, after=out.n)

    def finish(self, cam):
        """The active set at the end of the path is stored in a last anchor."""
        self.anchors.append(Anchor(camera_centre(cam), self.store))

    def render_anchors(self, cam, overlap=0.1):
        """Novel view from the anchors (Sec. 4.4): the closest anchor's
        Gaussians, or the two closest blended by opacity weights w, 1 - w."""
        c = camera_centre(cam)
        d = sorted((float(np.linalg.norm(a.location - c)), i) for i, a in enumerate(self.anchors))
        if len(d) == 1 or d[1][0] <= 0.0:
            parts = [(self.anchors[d[0][1]], 1.0)]
        else:
            w = gs.gs_anchor_blend_weight(d[0][0], d[1][0], overlap)
            parts = [(self.anchors[d[0][1]], w)] + ([(self.anchors[d[1][1]], 1.0 - w)] if w < 1.0 else [])
        sets = []
        for a, w in parts:
            g = a.load(self.device)
            if w < 1.0:
                gs.gs_scale_opacity(g.mean_opa, w)
            sets.append(g)
        g = gs.Gaussians(*[torch.cat([getattr(x, f) for x in sets]) for f in ("mean_opa", "scale", "quat", "sh")])
        r = Rasterizer(g.n, [(self.W, self.H)], 1 << 18, self.cfg, self.device)
        r.fit_capacity(g, cam)
        r.forward(g, cam)
        return r.img.color.clone()

    # -- steps -------------------------------------------------------------------
    def _render_active(self, cam):
        g, _, _ = self.store.active()
        if g.n == 0:
            return None
        r = Rasterizer(g.n, [(self.W, self.H)], 1 << 18, self.cfg, self.device)
        r.fit_capacity(g, cam)
        r.forward(g, cam)
        return r.img.color.clone()

    def _spawn(self, image, render, depth, cam, frame_idx):
        hw = self.W * self.H
        use_learned = self.mode == "learned" and frame_idx >= self.mlp_warmup_frames
        if use_learned:
            gs.gs_mlp_forward(self.mlp, image, self.W, self.H, self.mlp_out, self.mlp_cfg, self.ws_mlp)
            gs.gs_spawn_learned(image, self.mlp_out, self.W, self.H, cam, self.seed, frame_idx, self.spawned,
                                self.ws_spawn, depth=depth if self.learned_depth == "map" else None,
                                render=render)
        else:
            gs.gs_spawn_propose(image, render, depth, self.W, self.H, cam, 1.0, self.seed, frame_idx, self.spawned,
                                self.ws_spawn)
        torch.cuda.synchronize()
        k = min(int(self.spawned.count.item()), hw)
        return k, use_learned

    def _optimise(self, iters):
        """iters iterations over the sliding window; each frame renders at its
        current coarse-to-fine level, lowered every five iterations."""
        g, m, v = self.store.active()
        frames = self.frames[-self.window:]
        loss = torch.zeros(1, device=self.device)
        ws = gs.workspace(4 * 4096, self.device)
        lr = self.store.lr[:g.n] if self.adam.decay != 1.0 else None
        done = 0
        while done < iters:
            run = min(5, iters - done) if self.c2f else iters
            sizes, cams, targets = [], [], []
            for fr in frames:
                f = 1 << fr[2]
                if f > 1:
                    cams.append(gs.downsample_cameras(fr[1], f))
                    targets.append(gs.gs_downsample(fr[0], self.W, self.H, f))
                    sizes.append((-(-self.W // f), -(-self.H // f)))
                else:
                    cams.append(fr[1])
                    targets.append(fr[0])
                    sizes.append((self.W, self.H))
            cams, targets = torch.cat(cams), torch.cat(targets)
            r = Rasterizer(g.n, sizes, 1 << 18, self.cfg, self.device)
            r.fit_capacity(g, cams)
            dL = torch.zeros_like(r.img.color)
            for _ in range(run):
                r.forward(g, cams)
                gs.gs_l1_loss(r.img.color, targets, dL, loss, ws)
                r.backward(g, cams, dL)
                gs.gs_adam_step(g, r.grads, m, v, self.adam, 0, step_dev=self.step_dev, lr_scale=lr)
                gs.gs_counter_add(self.step_dev, 1)
                self.iter_count += 1
            done += run
            for fr in frames:
                fr[2] = max(0, fr[2] - 1)
        return float(loss.item())

    def _cull(self):
        """Opacity culling (Sec. 4.3): Gaussians below min_opacity leave the set
        with their optimiser state."""
        if self.min_opacity <= 0 or self.store.n == 0:
            return 0
        g, m, v = self.store.active()
        out = GaussianStore(self.store.cap, self.device)
        n_out = torch.zeros((1,), dtype=torch.int64, device=self.device)
        ws = gs.workspace(gs.gs_cull_opacity_workspace_size(g.n), self.device)
        gs.gs_cull_opacity(g, self.min_opacity, out.p, n_out, ws, m=m, v=v, m_out=out.m, v_out=out.v,
                           lr=self.store.lr[:g.n], lr_out=out.lr)
        out.n = int(n_out.item())
        removed = g.n - out.n
        self.store = out
        return removed

    def _train_mlp(self, image, n0, k, cam):
        """Targets from this frame's spawns after the optimisation (kept when
        still opaque: their optimised camera depth and the change of their mean
        log-scale), so the network learns where spawns survive and how their
        scale converges; then a few training steps of the proposal network."""
        if k == 0:
            return None
        g, _, _ = self.store.active()
        gs.gs_mlp_targets(self.spawned.pixel[:k], g.mean_opa[n0:n0 + k], g.scale[n0:n0 + k],
                          self.spawned.g.scale[:k], cam, self.keep_threshold, k, self.W, self.H, self.mlp_targets,
                          self.ws_tg)
        for _ in range(self.mlp_steps):
            self.mlp_step += 1
            gs.gs_mlp_train_step(self.mlp, self.mlp_m, self.mlp_v, image, self.W, self.H, self.mlp_targets,
                                 self.mlp_cfg, self.mlp_step, self.mlp_loss, self.ws_mlp)
        return float(self.mlp_loss.item())

    def _guided_depth(self, depth: torch.Tensor, feats, cam: torch.Tensor):
        """The frame's monocular depth refined by guided matching against the
        stored earlier frames (unchanged for the first frame)."""
        if feats is None:
            return depth
        prev = self.feat_frames[-self.guided_neighbours:]
        self.feat_frames.append((feats, cam))
        if not prev:
            return depth
        stack = torch.stack([feats] + [f for f, _ in prev]).contiguous()
        cams = torch.cat([cam] + [c for _, c in prev])
        out = gs.gs_guided_depth(stack, cams, depth.reshape(self.H, self.W).contiguous())
        return out.reshape(depth.shape)

    def add_frame(self, image: torch.Tensor, depth: torch.Tensor, cam: torch.Tensor, frame_idx: int,
                  feats: torch.Tensor | None = None):
        """One new frame: image [3HW], depth [HW] (the spawn depth; with
        guided_neighbours > 0 and feats [H][W][C] given, a monocular estimate
        refined by guided matching first), camera tensor."""
        if self.guided_neighbours > 0:
            depth = self._guided_depth(depth, feats, cam)
        anchor = self._maybe_anchor(frame_idx)
        render = self._render_active(cam)
        k, learned = self._spawn(image, render, depth, cam, frame_idx)
        n0 = self.store.n
        k = self.store.append(self.spawned, k)
        self.frames.append([image, cam, self.c2f])
        loss = self._optimise(self.iters)
        mlp_loss = None
        if self.mode == "learned" and (not learned or self.mlp_online):
            # the direct-sampling spawns of the warm-up frames that survived
            # the optimisation teach the proposal (before culling moves rows)
            mlp_loss = self._train_mlp(image, n0, k, cam)
        culled = self._cull()
        self.log.append(dict(frame=frame_idx, spawned=k, n=self.store.n, loss=loss, learned=learned,
                             mlp_loss=mlp_loss, iters=self.iter_count, anchor=anchor, culled=culled))
        self.prev_cam = cam

    def evaluate(self, frames):
        """Mean PSNR of the active set rendered at the given (image, camera) frames."""
        vals = []
        for image, cam in frames:
            r = self._render_active(cam)
            vals.append(psnr(r, image))
        return float(np.mean(vals))
