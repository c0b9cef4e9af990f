#!/usr/bin/env python
"""Throughput of the joint pose + Gaussian optimisation step on one GB300.

Workload (the headline configuration): 1,000,000 Gaussians with degree-3 SH
(fp32), 8 views of 1920x1080 on a smooth camera path (0.3 m / 5 degrees between
frames), poses perturbed by N(0, 0.01) rad/m. One step renders every view,
takes the L1 loss against the targets, runs the adjoint (Gaussian and SE(3)
pose gradients), a sparse Adam step on the visible Gaussians and an Adam +
retraction step on the poses. The metric counts view iterations: one
iteration = project + sort + render forward + render backward (with pose) of
one 1080p view. Inputs are synthetic (seeded) and far larger than L2.

Arms: "batched" (all views in each launch, launch configuration picked by the
autotuner, the step replayed from CUDA graphs; the value reported) and
"plain" (one launch sequence per view, default configuration). A second
workload, 2M Gaussians over 16 views of uneven resolution, is reported under
"uneven" with the same two arms.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent replica (the path is replicated,
not sharded, on this machine); value = views processed by all ranks / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "fwd+bwd splat iters/s @1080p, 1M Gaussians; batched vs plain; % roofline"
UNIT = "iters/s"
N_GAUSS = 1_000_000
N_VIEWS = 8
WIDTH, HEIGHT = 1920, 1080
SEED = 1002

# Algorithmic work per compositing evaluation - one (pixel, Gaussian) pair
# where the Gaussian reaches alpha_min before the pixel terminates - counted
# operation by operation from the definitions (3DGS image formation, Sec. 4.3);
# add, sub, mul = 1 flop, FMA = 2, compares and min/max not counted, shared
# subexpressions once.
# Forward (front to back):
#   d = pixel - mean2d                                  2
#   exponent -(a dx^2 + c dy^2)/2 - b dx dy: dx^2, dy^2, dx dy (3 mul),
#     a' dx^2 (1), + c' dy^2 (FMA 2), + b' dx dy (FMA 2)   8
#   g = exp(exponent)                                   MUFU ex2
#   o g                                                 1
#   T (1 - alpha)                                       2
#   w = alpha T; C += w rgb (3 FMA)                     7
#   total                                              20 flops, 1 MUFU
FWD_FLOPS_PER_EVAL = 20
FWD_MUFU_PER_EVAL = 1
# Adjoint (back to front, per composited Gaussian):
#   d, exponent, g, o g as forward                      11, 1 MUFU ex2
#   r = 1 / (1 - alpha): sub + reciprocal               1, 1 MUFU rcp
#   T_i = T_{i+1} r; w = alpha T_i                      2
#   dL/drgb = w gC (3)                                  3
#   dL/dalpha = sum_ch gC (T c - (A + T_N bg) r): per channel add, mul, mul,
#     sub, FMA                                         18
#   A += w c (3 FMA)                                    6
#   dL/dexponent = dL/dalpha o g; dL/do = dL/dalpha g   2
#   dL/dmean2d: (a dx + b dy), (b dx + c dy) (mul + FMA each) x dL/dexp  8
#   dL/dconic: dx^2, dx dy, dy^2 (reused) x dL/dexp      3
#   sum of the 9 terms over the tile's pixels            9
#   total                                              63 flops, 2 MUFU
BWD_FLOPS_PER_EVAL = 63
BWD_MUFU_PER_EVAL = 2
# Projection: EWA (world->camera, covariance from scale and rotation, J W S
# W^T J^T, inverse, radius, rect) about 100 flops, SH degree 3 (16 basis
# terms x 3 channels FMA + basis) about 150: 250 per visible item; its
# adjoint about twice that.
PROJECT_FLOPS_PER_ITEM = 250
PROJECT_BWD_FLOPS_PER_ITEM = 500
SMS = 152
FP32_LANES = 128


# render schedules of gs_config.schedule
SCHEDULES = {0: "grid", 1: "persistent", 2: "ordered grid"}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


PROFILE_OF_STAGE = {"composite_bwd": "render_bwd_1M_2x1080p.md", "render_fwd": "render_fwd_1M_2x1080p.md"}


def profiled_traffic(stage, n_views, root=ROOT):
    """DRAM bytes per launch from the committed ncu summary of the stage's
    kernel (measured on 2 views, scaled by views: traffic grows with the views
    rendered), or None when no summary exists or the kernel source changed
    since the counters were taken."""
    import hashlib
    import re
    name = PROFILE_OF_STAGE.get(stage)
    if not name:
        return None
    try:
        text = open(os.path.join(root, "profiles", name)).read()
        src = open(os.path.join(root, "paper_2506_05558_gb300", "csrc", "render.cu"), "rb").read()
    except OSError:
        return None
    m_sha = re.search(r"source_sha256: ([0-9a-f]+)", text)
    m_tb = re.search(r"traffic_bytes_per_view \| ([0-9.e+]+)", text)
    if not m_sha or not m_tb or not hashlib.sha256(src).hexdigest().startswith(m_sha.group(1)):
        return None
    return float(m_tb.group(1)) * n_views


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        return self.summarise(self.lines)

    @staticmethod
    def summarise(lines):
        """Median SM clock, the maximum clock and the throttle reasons seen
        active, from CSV lines of the query in FIELDS (no header, no units)."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def make_workload(torch, gs, synth, device, n, n_views, sizes=None, seed=SEED):
    """Scene, per-view sizes, true-pose targets (rendered by the path itself,
    untimed), training Gaussians (means jittered by N(0, 0.01)) and perturbed
    training poses."""
    from paper_2506_05558_gb300.raster import Rasterizer
    sc, cams, rng = synth.multiview_scene(seed=seed, n=n, n_views=n_views, sizes=sizes)
    sizes = [(c["width"], c["height"]) for c in cams]
    cfg = gs.config(sh_degree=3)
    g_true = gs.Gaussians.from_scene(sc, device)
    cams_true = gs.cameras_tensor(cams, device)
    r = Rasterizer(n, sizes, capacity=1 << 20, cfg=cfg, device=device)
    p = r.fit_capacity(g_true, cams_true)
    r.forward(g_true, cams_true)
    targets = r.img.color.clone()
    del r, g_true
    sc.mean_opa[:, :3] += rng.normal(0, 0.01, (n, 3)).astype(np.float32)
    g = gs.Gaussians.from_scene(sc, device)
    pert = []
    for c in cams:
        R, t = synth.perturb_pose(rng, c["R"].astype(np.float64), c["t"].astype(np.float64))
        pert.append(dict(c, R=R.astype(np.float32), t=t.astype(np.float32)))
    cams_train = gs.cameras_tensor(pert, device)
    torch.cuda.synchronize()
    return dict(sizes=sizes, cfg=cfg, g=g, cams=cams_train, targets=targets, pairs=p,
                g0=[t.clone() for t in (g.mean_opa, g.scale, g.quat, g.sh)], cams0=cams_train.clone())


def reset(W):
    g = W["g"]
    for t, s in zip((g.mean_opa, g.scale, g.quat, g.sh), W["g0"]):
        t.copy_(s)
    W["cams"].copy_(W["cams0"])


class PlainStep:
    """One launch sequence per view (views rendered one after another); the
    gradients of all views are accumulated before the single optimiser step."""

    def __init__(self, torch, gs, W, device):
        from paper_2506_05558_gb300.raster import Rasterizer
        self.gs = gs
        self.g, self.cams, self.targets, self.sizes = W["g"], W["cams"], W["targets"], W["sizes"]
        nv = len(self.sizes)
        self.cam_views = [self.cams[v * 72:(v + 1) * 72] for v in range(nv)]
        self.rs = []
        for v in range(nv):
            cfg_v = gs.config(sh_degree=W["cfg"].sh_degree, accumulate=1 if v > 0 else 0)
            r = Rasterizer(self.g.n, [self.sizes[v]], 1 << 20, cfg_v, device)
            r.fit_capacity(self.g, self.cam_views[v])
            self.rs.append(r)
        self.grads = self.rs[0].grads
        for r in self.rs[1:]:
            r.grads = self.grads  # one accumulation buffer
        self.dpose = torch.zeros((nv, 6), device=device)
        self.m, self.v = gs.Gaussians.zeros(self.g.n, device), gs.Gaussians.zeros(self.g.n, device)
        self.pm = torch.zeros((nv, 6), device=device)
        self.pv = torch.zeros((nv, 6), device=device)
        self.dLs = [torch.zeros_like(r.img.color) for r in self.rs]
        self.loss = torch.zeros((nv,), device=device)
        self.ws_loss = gs.workspace(4 * 4096, device)
        offs = np.cumsum([0] + [3 * w * h for w, h in self.sizes])
        self.tgt = [self.targets[offs[v]:offs[v + 1]] for v in range(nv)]
        self.adam = gs.adam_config()
        self.t = 0

    def step(self):
        gs = self.gs
        self.t += 1
        for v, r in enumerate(self.rs):
            cam = self.cam_views[v]
            gs.gs_project(self.g, cam, r.f, r.cfg, r.proj)
            gs.gs_sort(r.proj, r.n, r.f, r.pairs, r.ws_sort)
            gs.gs_render_fwd(r.proj, r.pairs, r.f, r.cfg, r.img, r.ws_render)
            gs.gs_l1_loss(r.img.color, self.tgt[v], self.dLs[v], self.loss[v:v + 1], self.ws_loss)
            gs.gs_render_bwd(self.g, cam, r.proj, r.pairs, r.f, r.cfg, r.img, self.dLs[v], self.grads,
                             self.dpose[v:v + 1], r.ws_bwd)
        gs.gs_adam_step(self.g, self.grads, self.m, self.v, self.adam, self.t)
        gs.gs_pose_step(self.cams, len(self.rs), self.dpose, self.pm, self.pv, 1e-3, 1e-3, self.t)
        return self.loss

    def ok(self):
        return all(r.status() == self.gs.GS_OK for r in self.rs)


class HostTargets:
    """Per-step upload of the targets from pinned host memory, double-buffered:
    the copy for step i + 1 runs on a side stream while step i computes. Each
    copy is ordered after everything already enqueued on the compute stream (so
    it never overwrites a buffer a step is still reading); each step waits for
    its own copy. start(k) begins a run of k steps: its first step waits for its
    own copy and its last step prefetches nothing, so a timed run of k steps
    contains exactly k host-to-device copies."""

    def __init__(self, torch, host, like):
        self.torch = torch
        self.host = host
        self.bufs = [torch.empty_like(like), torch.empty_like(like)]
        self.cs = torch.cuda.Stream()
        self.copied = [torch.cuda.Event(), torch.cuda.Event()]
        self.i = 0
        self.n = 0

    def start(self, steps):
        self.i, self.n = 0, steps

    def _copy(self, k):
        ready = self.torch.cuda.Event()
        ready.record(self.torch.cuda.current_stream())
        with self.torch.cuda.stream(self.cs):
            self.cs.wait_event(ready)
            self.bufs[k % 2].copy_(self.host, non_blocking=True)
            self.copied[k % 2].record(self.cs)

    def next(self):
        if self.i == 0:
            self._copy(0)
        if self.i + 1 < self.n:
            self._copy(self.i + 1)
        self.torch.cuda.current_stream().wait_event(self.copied[self.i % 2])
        buf = self.bufs[self.i % 2]
        self.i += 1
        return buf


def timed(torch, fn, steps, barrier):
    barrier()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        fn()
    b.record()
    torch.cuda.synchronize()
    barrier()
    return a.elapsed_time(b)


# ---------------------------------------------------------------------------
# the other rows of the path, timed on their own (1080p frame, 1M set)
# ---------------------------------------------------------------------------
MLP_FLOPS_PER_PATCH_FWD = 2 * (194 * 128 + 128 * 128 * 2 + 128 * 3)
MLP_FLOPS_PER_PATCH_TRAIN = 2 * MLP_FLOPS_PER_PATCH_FWD + 2 * (128 * 128 * 2 + 128 * 3)


def event_ms(torch, fn, reps):
    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def measure_mlp(torch, gs, device, peaks, img, Wd, Hd, rng, reps=10):
    """The learned proposal on one frame: a training step (forward, loss,
    backward, Adam) and an inference, on each tensor-core path."""
    out = {}
    prng = np.random.default_rng(1)
    layers = [(prng.uniform(-1, 1, (o, i)) / np.sqrt(i), prng.uniform(-1, 1, o) / np.sqrt(i))
              for o, i in ((128, 194), (128, 128), (128, 128), (3, 128))]
    n_p = gs.gs_mlp_patches(Wd, Hd)
    tg = torch.tensor(np.stack([rng.random(n_p), rng.uniform(2, 20, n_p), rng.normal(-4, 0.5, n_p),
                                (rng.random(n_p) < 0.5)], 1).astype(np.float32), device=device)
    wsm = gs.workspace(gs.gs_mlp_workspace_size(n_p), device)
    loss = torch.zeros(1, device=device)
    mo = torch.zeros((n_p, 3), device=device)
    for path in (0, 1):
        p = gs.MlpParams.from_numpy(layers, device)
        m, v = gs.MlpParams.zeros(device), gs.MlpParams.zeros(device)
        cfg = gs.mlp_config(tensor_path=path)
        step_dev = torch.ones(1, dtype=torch.int32, device=device)
        t_ms = event_ms(torch, lambda: gs.gs_mlp_train_step(p, m, v, img, Wd, Hd, tg, cfg, 0, loss, wsm,
                                                            step_dev=step_dev), reps)
        f_ms = event_ms(torch, lambda: gs.gs_mlp_forward(p, img, Wd, Hd, mo, cfg, wsm), reps)
        tf = MLP_FLOPS_PER_PATCH_TRAIN * n_p / t_ms / 1e9
        itf = MLP_FLOPS_PER_PATCH_FWD * n_p / f_ms / 1e9
        out[f"mlp_path{path}"] = {"path": "tcgen05 + TMEM" if path else "mma.sync",
                                  "infer": "one fused persistent kernel" if path else "GEMMs + epilogue kernels",
                                  "train_ms": t_ms, "infer_ms": f_ms, "train_tflops": tf, "infer_tflops": itf,
                                  "bound": "tensor", "peak": peaks["bf16"], "frac": tf / peaks["bf16"],
                                  "infer_frac": itf / peaks["bf16"], "patches": n_p}
    return out


def measure_rows(torch, gs, W, device, peaks, reps=10):
    out = {}
    Wd, Hd = WIDTH, HEIGHT
    hw = Wd * Hd
    img = W["targets"][:3 * hw]
    rng = np.random.default_rng(5)
    depth = torch.tensor(rng.uniform(2, 40, hw).astype(np.float32), device=device)
    cam0 = W["cams"][:72]
    # a8: direct spawn sampling on a 1080p frame; the render reproduces the
    # right half of the frame and is empty on the left, so the left half spawns
    render = img.clone()
    render.view(3, Hd, Wd)[:, :, :Wd // 2] = 0.0
    sp = gs.Spawned.alloc(hw)
    ws = gs.workspace(gs.gs_spawn_workspace_size(Wd, Hd), device)
    ms = event_ms(torch, lambda: gs.gs_spawn_propose(img, render, depth, Wd, Hd, cam0, 1.0, 7, 0, sp, ws), reps)
    n_sp = int(sp.count.item())
    # image + render + depth read, flags/positions written and read, spawned rows written
    bytes_ = (3 + 3 + 1) * 4 * hw + 16 * hw + n_sp * 240
    out["spawn_propose"] = {"ms": ms, "bound": "hbm", "achieved": bytes_ / ms / 1e6, "unit": "GB/s",
                            "frac": bytes_ / ms / 1e6 / peaks["hbm"], "spawned": n_sp}
    # a10: learned proposal, one training step and one inference on a 1080p frame
    out.update(measure_mlp(torch, gs, device, peaks, img, Wd, Hd, rng, reps))
    # a9: anchor size test on the 1M set and host offload of the set + Adam moments
    g = W["g"]
    fine = torch.zeros(g.n, dtype=torch.uint8, device=device)
    cnt = torch.zeros(1, dtype=torch.int64, device=device)
    a_ms = event_ms(torch, lambda: gs.gs_anchor_check(g, cam0, 1.0, fine, cnt), reps)
    hosts = [gs.pinned_gaussians(g.n) for _ in range(3)]
    mm = gs.Gaussians.zeros(g.n, device)
    o_ms = event_ms(torch, lambda: gs.gs_anchor_offload(g, mm, mm, hosts[0], hosts[1], hosts[2]), 3)
    hosts_dev = [gs.Gaussians.zeros(g.n, device) for _ in range(2)]
    # f1: merge of the too-fine set (k = 3, 0.5 m search radius) with Adam state
    mout = gs.Gaussians.zeros(g.n, device)
    n_out = torch.zeros(1, dtype=torch.int64, device=device)
    wsa = gs.workspace(gs.gs_anchor_merge_workspace_size(g.n, 3), device)
    m_ms = event_ms(torch, lambda: gs.gs_anchor_merge(g, fine, 0.5, 7, mout, n_out, wsa, m=mm, v=mm,
                                                      m_out=hosts_dev[0], v_out=hosts_dev[1]), 3)
    out["anchor"] = {"check_ms": a_ms, "check_gbs": (33 * g.n) / a_ms / 1e6, "too_fine": int(cnt.item()),
                     "offload_ms": o_ms, "offload_gbs": 3 * 240 * g.n / o_ms / 1e6,
                     "offload_bytes": 3 * 240 * g.n, "merge_ms": m_ms, "merged_rows_out": int(n_out.item())}
    return out


def measure_ba_pose(torch, gs, device, iterations=20):
    """Pose refinement of a new frame shaped like the paper's (6144 keypoints
    against triangulated points, 20 Levenberg-Marquardt iterations): eager
    launches and one CUDA graph holding all iterations."""
    from paper_2506_05558_gb300 import synth
    pr = synth.ba_pose_problem()
    M = pr["X"].shape[0]
    W, H = pr["width"], pr["width"] * 9 // 16
    cx, cy = W / 2.0, H / 2.0
    f32 = lambda a: torch.tensor(np.asarray(a, np.float32), device=device).contiguous()
    ident = gs.cameras_tensor([synth.camera(np.eye(3), np.zeros(3), 1.0, 16, 16)], device)
    cam_gt = torch.empty_like(ident)
    gs.gs_pose_apply(ident, f32(pr["xi"][None]), 1, cam_gt)
    cam_0 = torch.empty_like(ident)
    gs.gs_pose_apply(cam_gt, f32(pr["start_xi"][None]), 1, cam_0)
    rt = lambda c: c.view(torch.float32)[:12].clone()
    pts = f32(np.concatenate([pr["X"], np.zeros((M, 1))], 1))
    fl = f32([pr["fl"]])
    obs = torch.empty((M, 1, 2), dtype=torch.float32, device=device)
    gs.gs_ba_project(fl, rt(cam_gt)[None], pts, cx, cy, obs)
    obs = (obs.view(M, 2) + f32(pr["noise"])).contiguous()
    ws = gs.workspace(gs.gs_ba_pose_workspace_size(M), device)
    failed = torch.zeros(1, dtype=torch.int32, device=device)
    hist = torch.zeros((iterations, 3), device=device)
    stream = torch.cuda.Stream()
    pose, lam = rt(cam_0), f32([1e-5])
    with torch.cuda.stream(stream):
        gs.gs_ba_pose_lm(pts, obs, fl, cx, cy, pose, lam, 2, ws, failed, stream=stream)  # warm-up
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pose, lam = rt(cam_0), f32([1e-5])
    with torch.cuda.stream(stream):
        a.record(stream)
        gs.gs_ba_pose_lm(pts, obs, fl, cx, cy, pose, lam, iterations, ws, failed, history=hist, stream=stream)
        b.record(stream)
    torch.cuda.synchronize()
    eager_ms = a.elapsed_time(b)
    pose, lam = rt(cam_0), f32([1e-5])
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        gs.gs_ba_pose_lm(pts, obs, fl, cx, cy, pose, lam, iterations, ws, failed, history=hist, stream=stream)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        a.record(stream)
        g.replay()
        b.record(stream)
    torch.cuda.synchronize()
    graph_ms = a.elapsed_time(b)
    Rg = rt(cam_gt).cpu().numpy().astype(np.float64)
    Rp = pose.cpu().numpy().astype(np.float64)
    ang = float(np.arccos(np.clip((np.trace(Rp[:9].reshape(3, 3) @ Rg[:9].reshape(3, 3).T) - 1) / 2, -1, 1)))
    h = hist.cpu().numpy()
    return {"observations": M, "iterations": iterations, "graph_ms": graph_ms, "eager_ms": eager_ms,
            "cost_start": float(h[0, 0]), "cost_end": float(h[-1, 0]), "failed": int(failed.item()),
            "rot_err_rad": ang, "trans_err_m": float(np.linalg.norm(Rp[9:] - Rg[9:])),
            "paper": "4 ms with CUDA graphs, 95 ms without (incremental mini bundle adjustment, RTX 4090; context)"}


# Guided matching: per candidate of a refined pixel, 4 corner dot products of C
# channels (4C FMA), the bilinear weighting (4 FMA) and the projection (about 10
# flops); the neighbour choice adds a few dozen flops per pixel, not counted.
def guided_flops_per_candidate(C):
    return 8 * C + 8 + 10


def measure_guided(torch, gs, device, fp32_peak_tflops, reps=20, n_cand=32):
    """Guided-matching depth refinement of one 1920x1080 frame: four neighbours,
    32 bf16 channels per pixel, 32 inverse-depth candidates (the synthetic room
    of the generator); feature maps (663 MB) exceed L2."""
    from paper_2506_05558_gb300 import synth
    sc = synth.guided_scene()
    feats = torch.from_numpy(sc["feats"].view(np.int16)).to(device)
    cams = gs.cameras_tensor(sc["cams"], device)
    z = torch.from_numpy(sc["z_mono"]).to(device)
    H, W = sc["z_mono"].shape
    C = feats.shape[-1]
    depth = torch.empty((H, W), device=device)
    nb = torch.empty((H, W), dtype=torch.int32, device=device)
    corr = torch.empty((H, W), device=device)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        gs.gs_guided_depth(feats, cams, z, n_cand=n_cand, depth=depth, nb=nb, corr=corr)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        gs.gs_guided_depth(feats, cams, z, n_cand=n_cand, depth=depth, nb=nb, corr=corr)
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ms = float(np.median(ts))
    refined = int((nb >= 0).sum().item())
    tflops = refined * n_cand * guided_flops_per_candidate(C) / (ms / 1000.0) / 1e12
    v = nb.cpu().numpy() >= 0
    zt = sc["z_true"]
    err_g = float(np.median(np.abs(1 / depth.cpu().numpy()[v] - 1 / zt[v])))
    err_m = float(np.median(np.abs(1 / sc["z_mono"][v] - 1 / zt[v])))
    return {"size": [W, H], "neighbours": feats.shape[0] - 1, "channels": C, "candidates": n_cand, "ms": ms,
            "mpix_per_s": W * H / ms / 1e3, "refined_frac": refined / (W * H), "achieved_tflops": tflops,
            "fp32_frac": tflops / fp32_peak_tflops, "median_inv_depth_err": err_g,
            "median_inv_depth_err_mono": err_m,
            "paper": "11.2 ms per keyframe for guided matching (RTX 4090; context)"}


def measure_ba(torch, gs, device, iterations=200):
    """Bootstrapping mini bundle adjustment shaped like the paper's (8 frames,
    6144 keypoints, 200 Levenberg-Marquardt iterations): eager launches and one
    CUDA graph holding all iterations."""
    from paper_2506_05558_gb300 import synth
    pr = synth.ba_problem()
    F, P = pr["xi"].shape[0], pr["X"].shape[0]
    W, H = pr["width"], pr["width"] * 9 // 16
    cx, cy = W / 2.0, H / 2.0
    f32 = lambda a: torch.tensor(np.asarray(a, np.float32), device=device).contiguous()
    ident = gs.cameras_tensor([synth.camera(np.eye(3), np.zeros(3), 1.0, 16, 16)] * F, device)
    cams_gt = torch.empty_like(ident)
    gs.gs_pose_apply(ident, f32(pr["xi"]), F, cams_gt)
    start_xi = pr["start_xi"].copy()
    start_xi[0] = 0.0  # frame 0 is the gauge
    cams_0 = torch.empty_like(ident)
    gs.gs_pose_apply(cams_gt, f32(start_xi), F, cams_0)
    rt = lambda c: c.view(torch.float32).view(F, 18)[:, :12].contiguous()
    pts_gt = f32(np.concatenate([pr["X"], np.zeros((P, 1))], 1))
    obs = torch.empty((P, F, 2), dtype=torch.float32, device=device)
    gs.gs_ba_project(f32([pr["fl"]]), rt(cams_gt), pts_gt, cx, cy, obs)
    obs += f32(pr["noise"])
    ws = gs.workspace(gs.gs_ba_workspace_size(F, P), device)
    failed = torch.zeros(1, dtype=torch.int32, device=device)
    hist = torch.zeros((iterations, 3), device=device)

    def state():
        return (f32([pr["fl"] * pr["start_fl"]]), rt(cams_0),
                f32(np.concatenate([pr["X"] * pr["start_X_scale"], np.zeros((P, 1))], 1)), f32([1e-5]))

    stream = torch.cuda.Stream()
    fl, poses, pts, lam = state()
    with torch.cuda.stream(stream):
        gs.gs_ba_lm(obs, cx, cy, fl, poses, pts, lam, 2, ws, failed, stream=stream)  # warm-up
    torch.cuda.synchronize()
    fl, poses, pts, lam = state()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        a.record(stream)
        gs.gs_ba_lm(obs, cx, cy, fl, poses, pts, lam, iterations, ws, failed, history=hist, stream=stream)
        b.record(stream)
    torch.cuda.synchronize()
    eager_ms = a.elapsed_time(b)
    fl, poses, pts, lam = state()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        gs.gs_ba_lm(obs, cx, cy, fl, poses, pts, lam, iterations, ws, failed, history=hist, stream=stream)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        a.record(stream)
        g.replay()
        b.record(stream)
    torch.cuda.synchronize()
    graph_ms = a.elapsed_time(b)
    h = hist.cpu().numpy()
    return {"frames": F, "points": P, "iterations": iterations, "graph_ms": graph_ms, "eager_ms": eager_ms,
            "ms_per_iteration": graph_ms / iterations, "cost_start": float(h[0, 0]),
            "cost_end": float(h[-1, 0]), "accepted": int(h[:, 2].sum()), "failed": int(failed.item()),
            "focal_end": float(fl.item()), "focal_true": pr["fl"],
            "paper": "145 ms with CUDA graphs, 625 ms without (bootstrapping optimisation, RTX 4090; context)"}


# ---------------------------------------------------------------------------
# oracle on the host cores
# ---------------------------------------------------------------------------
def measure_stream(torch, gs, synth, device, frames=100, size=(1920, 1080), n_gt=2_000_000, runs=None,
                   log_every=10):
    """The streaming workload at full size (Sec. 4.2-4.4): new 1920x1080 frames of
    a textured corridor along the standard path, spawn depths from a
    monocular-style estimate (true depth x a smooth 25% error field) for every
    mode, 3-frame window, anchors at 1 px / 40% with merging, opacity culling
    at 0.005. runs: (name, mode, iterations per frame, extra OnTheFly options).
    Per run: per-frame wall time, active set, Gaussians spawned in total, anchors
    and host bytes offloaded, PSNR of each new frame after its optimisation and
    of the last five frames rendered from the final active set."""
    from paper_2506_05558_gb300.stream import OnTheFly, render_depth, psnr
    if runs is None:
        runs = [("plain_30", "plain", 30, {}), ("plain_25", "plain", 25, {}), ("learned_30", "learned", 30, {}),
                ("learned_25", "learned", 25, {}),
                # the corridor keeps Gaussians above 1 px from the previous camera, so anchors
                # are also exercised with a 4 px size threshold
                ("learned_25_anchor_4px", "learned", 25, {"anchor_tau": 4.0})]
    W_, H_ = size
    sc, cams = synth.corridor_scene(n=n_gt, n_views=frames, size=size)
    g_true = gs.Gaussians.from_scene(sc, device)
    data = []
    for i, c in enumerate(cams):
        ct = gs.cameras_tensor([c], device)
        color, depth = render_depth(g_true, ct, size, gs.config(sh_degree=0), device)
        fac = torch.from_numpy(synth.monocular_factor(W_, H_, 300 + i)).to(device).reshape(-1)
        data.append((color, (depth * fac).contiguous(), ct))
    del g_true
    torch.cuda.synchronize()
    out = {"frames": frames, "size": [W_, H_], "ground_truth_gaussians": n_gt, "runs": {}}
    for name, mode, iters, kw in runs:
        opts = dict(anchor_tau=1.0, anchor_share=0.4, merge_radius=0.5, min_opacity=0.005)
        opts.update(kw)
        otf = OnTheFly(8_000_000, size, window=3, iters=iters, mode=mode, mlp_warmup_frames=3, mlp_steps=30,
                       device=device, **opts)
        per = []
        t_all = time.time()
        for i, (img, depth, cam) in enumerate(data):
            torch.cuda.synchronize()
            t0 = time.time()
            otf.add_frame(img, depth, cam, i)
            torch.cuda.synchronize()
            dt = time.time() - t0
            p_new = otf.evaluate([(img, cam)])
            e = otf.log[-1]
            per.append({"frame": i, "s": dt, "active": otf.store.n, "spawned": e["spawned"], "psnr": p_new,
                        "culled": e["culled"], "anchor": e["anchor"]})
            if i % log_every == 0:
                log(f"stream {name} frame {i}: {dt:.3f} s, active {otf.store.n}, spawned {e['spawned']}, "
                    f"psnr {p_new:.2f}")
        total_s = time.time() - t_all
        last = otf.evaluate([(img, cam) for img, _, cam in data[-5:]])
        out["runs"][name] = {
            "mode": mode, "iters_per_frame": iters, "total_s": total_s,
            "s_per_frame_median": float(np.median([q["s"] for q in per])),
            "peak_active": max(q["active"] for q in per), "final_active": otf.store.n,
            "spawned_total": sum(q["spawned"] for q in per), "anchors": len(otf.anchors),
            "offloaded_bytes": int(sum(a.n for a in otf.anchors) * 3 * 240),
            "psnr_new_frame_mean": float(np.mean([q["psnr"] for q in per])),
            "psnr_last5_final": last, "anchor_tau_px": opts["anchor_tau"],
            "merges": [q["anchor"] for q in per if q["anchor"]], "per_frame": per}
        del otf
        torch.cuda.empty_cache()
    return out


def ssim(torch, img, ref, window=11, sigma=1.5):
    """Mean SSIM of a [3][H][W] pair: 11x11 Gaussian window (sigma 1.5), zero
    padding, C1 = 0.01^2, C2 = 0.03^2 (the 720p workload's D-SSIM term; PyTorch
    turns the loss into dL/dC, which is all that crosses the library boundary)."""
    F = torch.nn.functional
    x = torch.arange(window, dtype=img.dtype, device=img.device) - window // 2
    k1 = torch.exp(-x * x / (2 * sigma * sigma))
    k1 = k1 / k1.sum()
    k = (k1[:, None] * k1[None, :]).expand(3, 1, window, window).contiguous()
    f = lambda t: F.conv2d(t[None], k, padding=window // 2, groups=3)[0]
    mu_x, mu_y = f(img), f(ref)
    sxx = f(img * img) - mu_x * mu_x
    syy = f(ref * ref) - mu_y * mu_y
    sxy = f(img * ref) - mu_x * mu_y
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    m = ((2 * mu_x * mu_y + c1) * (2 * sxy + c2)) / ((mu_x * mu_x + mu_y * mu_y + c1) * (sxx + syy + c2))
    return m.mean()


def config_scene(synth, which):
    """(scene, camera, rng, sh degree) of the 64x64 (which = 0) or 720p (1) workload."""
    if which == 0:
        sc, cam, rng = synth.tiny_scene()
        return sc, cam, rng, 0
    sc, cam, rng = synth.view_720p_scene()
    return sc, cam, rng, 3


def oracle_config_time(which, min_s=5.0):
    """Seconds per fwd+bwd (incl. pose) of the FP64 oracle on one view of the
    64x64 or 720p workload, repeated for at least min_s seconds (at least once),
    with the threads OMP_NUM_THREADS gives."""
    from oracle import build as ob
    from oracle import oracle as O
    from paper_2506_05558_gb300 import synth
    ob.build()
    sc, cam, rng, shd = config_scene(synth, which)
    cfg = O.Config(sh_degree=shd)
    H, W = cam["height"], cam["width"]
    dL = np.sign(rng.standard_normal((3, H, W))) / (3 * H * W)
    n, t0 = 0, time.perf_counter()
    while True:
        view = O.render_view(sc, cam, cfg)
        O.backward_view(sc, cam, cfg, view, dL)
        n += 1
        if time.perf_counter() - t0 >= min_s:
            break
    return (time.perf_counter() - t0) / n


def measure_configs(torch, gs, synth, device, reps=(400, 50)):
    """Iterations per second of the 64x64 and 720p workloads on the GPU (project,
    sort, forward, loss, adjoint with the pose gradient; no optimiser step; the
    720p loss is L1 + 0.2 (1 - SSIM) through PyTorch autograd into dL/dC), CUDA
    events over the repetitions after warm-up; and the FP64 oracle's time per
    iteration on one host thread and on all host cores (child processes)."""
    from paper_2506_05558_gb300.raster import Rasterizer
    out = {}
    for which in (0, 1):
        sc, cam, rng, shd = config_scene(synth, which)
        W_, H_ = cam["width"], cam["height"]
        cfg = gs.config(sh_degree=shd)
        g = gs.Gaussians.from_scene(sc, device)
        cams = gs.cameras_tensor([cam], device)
        r = Rasterizer(sc.n, [(W_, H_)], 1 << 20, cfg, device)
        r.fit_capacity(g, cams)
        r.forward(g, cams)
        tgt = (r.img.color.view(3, H_, W_) + 0.01 * torch.randn((3, H_, W_), device=device)).contiguous()
        dL = torch.zeros_like(r.img.color)
        loss = torch.zeros(1, device=device)
        ws = gs.workspace(4 * 4096, device)

        def step():
            r.forward(g, cams)
            if which == 0:
                gs.gs_l1_loss(r.img.color, tgt.view(-1), dL, loss, ws)
            else:
                img = r.img.color.view(3, H_, W_).detach().requires_grad_(True)
                lv = (img - tgt).abs().mean() + 0.2 * (1.0 - ssim(torch, img, tgt))
                lv.backward()
                dL.copy_(img.grad.view(-1))
            r.backward(g, cams, dL)

        for _ in range(5):
            step()
        ms = event_ms(torch, step, reps[which])
        assert r.status() == gs.GS_OK
        t1 = t_all = None
        for threads in (1, os.cpu_count() or 1):
            env = dict(os.environ, OMP_NUM_THREADS=str(threads))
            res = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-config", str(which)],
                                 capture_output=True, text=True, env=env)
            sec = float(res.stdout.strip().splitlines()[-1]) if res.returncode == 0 else None
            if threads == 1:
                t1 = sec
            else:
                t_all = sec
        name = "64x64, 1k Gaussians SH0, L1" if which == 0 else "1280x720, 200k Gaussians SH3, L1 + 0.2 D-SSIM"
        out[f"config{which}"] = {"workload": name, "gpu_ms_per_iter": ms, "gpu_iters_per_s": 1000.0 / ms,
                                 "oracle_s_per_iter_1_thread": t1, "oracle_s_per_iter_all_cores": t_all,
                                 "host_cores": os.cpu_count()}
    return out


def measure_peaks(torch, gs, device, sms, reps=5):
    """FP32 FMA and MUFU throughput measured by the library's probes (one
    CTA of 256 threads per 1/8 of an SM's threads, i.e. 8 per SM, long enough
    to time with CUDA events): best of reps, in TFLOP/s and T MUFU ops/s."""
    blocks = 8 * sms
    out = torch.empty(blocks * 256, dtype=torch.float32, device=device)
    res = {}
    for name, fn, per_iter, iters in (("fp32_tflops", gs.gs_probe_fma, 2 * 128, 2048),
                                      ("mufu_tops", gs.gs_probe_mufu, 64, 512)):
        fn(out, blocks, 16)  # warm-up
        best = None
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn(out, blocks, iters)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        res[name] = blocks * 256 * per_iter * iters / (best / 1000.0) / 1e12
        res[name.split("_")[0] + "_ms"] = best
    return res


def oracle_sample(n_views_sample=1, n=N_GAUSS):
    """Times the FP64 oracle's fwd+bwd (incl. pose) on n_views_sample of the
    workload's 1080p views over the full scene. Returns (iters/s, seconds, cores)."""
    from oracle import oracle as O
    from paper_2506_05558_gb300 import synth
    sc, cams, rng = synth.multiview_scene(seed=SEED, n=n, n_views=N_VIEWS)
    cfg = O.Config(sh_degree=3)
    dL = [np.sign(rng.standard_normal((3, HEIGHT, WIDTH))) / (3 * HEIGHT * WIDTH * N_VIEWS)
          for _ in range(n_views_sample)]
    t0 = time.perf_counter()
    for k in range(n_views_sample):
        view = O.render_view(sc, cams[k], cfg)
        O.backward_view(sc, cams[k], cfg, view, dL[k])
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return n_views_sample / dt, dt, cores


class Ranks:
    """Rank bookkeeping of a torchrun launch (one process per GPU, replicas):
    a barrier, the maximum of a per-rank time over all ranks, and the whole-job
    throughput from it. With one rank every call is local; the tensors of the
    collective live on `device` (a GPU under NCCL, the host under gloo)."""

    def __init__(self, world: int, rank: int, device, dist=None):
        self.world, self.rank, self.device, self.dist = world, rank, device, dist

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()

    def max(self, x: float) -> float:
        if self.world == 1:
            return x
        import torch
        t = torch.tensor([x], device=self.device, dtype=torch.float64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def throughput(self, units_per_rank: float, ms_local: float) -> tuple[float, float]:
        """(whole-job units per second, slowest rank's ms): every rank processed
        units_per_rank in its own timed region; the job took the longest one."""
        ms = self.max(ms_local)
        return self.world * units_per_rank / (ms / 1000.0), ms


def workload_name(n, views):
    return (f"joint pose+Gaussian optimisation step: {n} Gaussians SH3, {views} views {WIDTH}x{HEIGHT}, "
            "L1 + adjoint with SE(3) pose gradients + sparse Adam")


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step is one 1080p view's fwd+bwd
    (a bounded sample of the 8-view step) on the host cores."""
    if rank != 0:
        return 0
    from oracle import build as ob
    ob.build()
    for _ in range(args.warmup):
        oracle_sample(1)
    vals = []
    t_all = time.perf_counter()
    cores = 1
    for _ in range(args.steps):
        _, dt, cores = oracle_sample(1)
        vals.append(dt)
    total = time.perf_counter() - t_all
    value = len(vals) / sum(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(vals) / len(vals),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(N_GAUSS, N_VIEWS),
                       "step_sample": f"1 of the {N_VIEWS} views per step (FP64 oracle on the host cores); "
                                      "value in view iterations per second like the batched arm's"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "per step: fwd+bwd (incl. pose) of one 1080p view of the 1M-Gaussian scene"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": total}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# main
# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_GAUSS)
    ap.add_argument("--views", type=int, default=N_VIEWS)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-uneven", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-rows", action="store_true", help="skip the spawn / MLP / anchor measurements")
    ap.add_argument("--cpu-views", type=int, default=6, help="views of the oracle CPU sample")
    ap.add_argument("--oracle-config", type=int, default=None, help=argparse.SUPPRESS)
    ap.add_argument("--row", choices=["mini_ba", "pose_refine", "guided_matching", "stream", "configs", "mlp"],
                    default=None,
                    help="measure only this side row and print its numbers (for profiling)")
    ap.add_argument("--ba-iterations", type=int, default=200)
    ap.add_argument("--stream-frames", type=int, default=100)
    ap.add_argument("--stream-gt", type=int, default=2_000_000, help="ground-truth Gaussians of the streaming row")
    args = ap.parse_args()
    if args.warmup < 3:
        log("warm-up raised to 3 (timing rule)")
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.oracle_config is not None:  # child process of the configs row: the oracle alone
        print(oracle_config_time(args.oracle_config), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    from paper_2506_05558_gb300 import autotune, gs, synth
    from paper_2506_05558_gb300.raster import JointOptimizer

    torch.cuda.set_device(local_rank)
    device = f"cuda:{local_rank}"
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(device))

    ranks = Ranks(world, rank, device, dist)
    barrier, max_over_ranks = ranks.barrier, ranks.max

    gs.lib()
    if args.row is not None:  # one side row alone, rank 0 only
        if rank == 0:
            if args.row == "mini_ba":
                r = measure_ba(torch, gs, device, iterations=args.ba_iterations)
            elif args.row == "pose_refine":
                r = measure_ba_pose(torch, gs, device)
            elif args.row == "mlp":
                rng = np.random.default_rng(5)
                img = torch.tensor(rng.random(3 * WIDTH * HEIGHT).astype(np.float32), device=device)
                try:
                    bf16 = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
                except (OSError, KeyError, ValueError):
                    bf16 = 1900.0  # the pool's earlier GB300 measurement, used when the file is absent
                r = measure_mlp(torch, gs, device, {"bf16": bf16}, img, WIDTH, HEIGHT, rng)
            elif args.row == "configs":
                r = measure_configs(torch, gs, synth, device)
            elif args.row == "stream":
                r = measure_stream(torch, gs, synth, device, frames=args.stream_frames, n_gt=args.stream_gt)
            else:
                r = measure_guided(torch, gs, device, SMS * FP32_LANES * 2 * 2070.0 * 1e6 / 1e12)
            print(json.dumps({"row": args.row, **r}), flush=True)
        return 0
    W = make_workload(torch, gs, synth, device, args.n, args.views)
    capacity = int(W["pairs"] * 1.3) + 4096

    # ---------------- launch configuration ----------------
    tuned = None
    cfg = W["cfg"]
    if not args.no_autotune:
        cfg, table = autotune.tune(W["g"], W["cams"], W["sizes"], W["targets"], W["cfg"], steps=2, device=device,
                                   log=log)
        tuned = {"tile": cfg.tile, "fwd_batch": cfg.fwd_batch, "bwd_batch": cfg.bwd_batch,
                 "schedule": SCHEDULES[cfg.schedule],
                 "trials": [{"tile": t, "fwd_batch": fb, "bwd_batch": bb, "schedule": sc, "ms": ms}
                            for t, fb, bb, sc, ms in table]}
        reset(W)

    # ---------------- batched arm: per-stage CUDA graphs, events between them ----------------
    J = JointOptimizer(W["g"], W["cams"], W["sizes"], W["targets"], capacity, cfg, device=device)
    J.r.fit_capacity(W["g"], W["cams"])
    J.step()  # one-time set-up outside the capture
    torch.cuda.synchronize()
    reset(W)
    J.step_dev.fill_(1)
    launches_per_step = gs.gs_launch_count()
    J.step()
    torch.cuda.synchronize()
    launches_per_step = gs.gs_launch_count() - launches_per_step
    J.capture(per_stage=True)
    for _ in range(args.warmup):
        J.replay()
    torch.cuda.synchronize()
    assert J.r.status() == gs.GS_OK, "pair buffer overflow"
    n_ev = len(J.graphs) + 1
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(n_ev)] for _ in range(args.steps)]
    clocks = ClockSampler(local_rank)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.25)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record()
    for k in range(args.steps):
        J.replay(ev[k])
    t_end.record()
    torch.cuda.synchronize()
    barrier()
    time.sleep(0.1)
    clk = clocks.stop()
    value, ms = ranks.throughput(args.views * args.steps, t_start.elapsed_time(t_end))
    stage_ms = {name: float(np.mean([ev[k][i].elapsed_time(ev[k][i + 1]) for k in range(args.steps)]))
                for i, (name, _) in enumerate(J.graphs)}
    status = J.r.status()
    kept = (J.r.proj.n_tiles[:args.views * args.n] > 0).view(args.views, args.n)
    n_items_vis = int(kept.sum().item())
    n_seen = int(kept.any(0).sum().item())  # Gaussians kept in at least one view
    P = J.r.pair_count()
    K = int(J.r.img.n_contrib.to(torch.int64).sum().item())
    loss = float(J.loss.item())

    # ---------------- counted work (untimed) and measured peaks ----------------
    counts = torch.zeros(3, dtype=torch.int64, device=device)
    gs.gs_render_fwd_count(J.r.proj, J.r.pairs, J.r.f, J.r.cfg, J.r.img, counts, J.r.ws_render)
    torch.cuda.synchronize()
    warp_hits, lane_evals, K_c = (int(x) for x in counts.cpu().tolist())
    HW = sum(w * h for w, h in W["sizes"])
    n_tiles = int(J.r.f.tile_base[len(W["sizes"])])
    probe = measure_peaks(torch, gs, device, SMS)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    sm_clock = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak_tflops = probe["fp32_tflops"]
    mufu_peak_tops = probe["mufu_tops"]
    fp32_derived = SMS * FP32_LANES * 2 * sm_clock * 1e6 / 1e12
    # algorithmic work per stage: (bytes, flops, MUFU ops); bytes are what the
    # method must move (each input read once, each output written once)
    Vs, Vi, N, P = n_seen, n_items_vis, args.n, P
    work = {
        # cull read of every Gaussian, attributes of the Gaussians kept in any view read once,
        # 52 B per visible item and 12 B per culled one written
        "project": (16 * N + 224 * Vs + 52 * Vi + 12 * (N * args.views - Vi), PROJECT_FLOPS_PER_ITEM * Vi, 0),
        # visible depth keys + ids sorted, pair keys and ids written once, pairs sorted once, tile ranges
        "sort": (32 * Vi + 12 * P + 24 * P + 8 * P + 8 * n_tiles, 0, 0),
        # pair rows read once (id + mean2d + conic/opacity + rgb), colour + T + n_contrib written
        "render_fwd": (40 * P + 20 * HW, FWD_FLOPS_PER_EVAL * K_c, FWD_MUFU_PER_EVAL * K_c),
        # colour and target read, dL/dC written
        "loss": (36 * HW, 3 * HW, 0),
        # dL/dC, T, n_contrib read, pair rows read, one 9-float partial per pair written
        "composite_bwd": (20 * HW + 40 * P + 36 * P, BWD_FLOPS_PER_EVAL * K_c, BWD_MUFU_PER_EVAL * K_c),
        # parameters read, gradients written, item state and pair partials read
        "project_bwd": (480 * Vs + 48 * Vi + 36 * P, PROJECT_BWD_FLOPS_PER_ITEM * Vi, 0),
        # parameter, gradient, m, v read; parameter, m, v written, for the visible Gaussians; visibility flags
        "adam": (7 * 240 * Vs + N, 15 * 60 * Vs, 0),
        "pose": (0, 0, 0),
    }
    stages = {}
    floor_ms = 0.0
    for st, msv in stage_ms.items():
        by, fl, mu = work.get(st, (0, 0, 0))
        t_bytes = by / (hbm_peak * 1e9) * 1e3
        t_flops = fl / (fp32_peak_tflops * 1e12) * 1e3
        t_mufu = mu / (mufu_peak_tops * 1e12) * 1e3
        t_floor = max(t_bytes, t_flops, t_mufu)
        bound = ["hbm", "alu", "mufu"][int(np.argmax([t_bytes, t_flops, t_mufu]))]
        floor_ms += t_floor
        e = {"ms": msv, "floor_ms": t_floor, "bound": bound, "frac": t_floor / msv if msv > 0 else None,
             "bytes": by, "flops": fl, "mufu": mu}
        if bound == "hbm":
            e.update(achieved=by / (msv / 1e3) / 1e9, peak=hbm_peak, unit="GB/s")
        else:
            e.update(achieved=fl / (msv / 1e3) / 1e12, peak=fp32_peak_tflops, unit="TFLOP/s")
        stages[st] = e
    step_ms = ms / args.steps
    dom = max(stage_ms, key=lambda st: stage_ms[st])
    d = stages[dom]
    roof = {"kernel": dom, "bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"], "unit": d["unit"],
            "frac": d["achieved"] / d["peak"], "traffic": profiled_traffic(dom, args.views),
            "peak_source": ("FP32 FMA throughput measured by the library's probe (gs_probe_fma) in this run "
                            f"({fp32_peak_tflops:.1f} TFLOP/s; 152 SMs x 128 lanes x 2 x {sm_clock:.0f} MHz = "
                            f"{fp32_derived:.1f})" if d["bound"] == "alu"
                            else "MEASURED_PEAKS.json hbm_gbs (of measured)"),
            "work": "flops per compositing evaluation (63 adjoint, 20 forward; derivation in bench.py) x the "
                    "evaluations that composite, counted by an untimed instantiation of the forward kernel",
            "evaluations": {"composited": K_c, "live_lane_evaluations": lane_evals, "warp_hits": warp_hits,
                            "lane_slots": 32 * warp_hits, "list_entries_to_termination": K},
            "step_frac": floor_ms / step_ms, "step_floor_ms": floor_ms,
            "peaks": {"hbm_gbs": hbm_peak, "fp32_tflops": fp32_peak_tflops, "mufu_tops": mufu_peak_tops,
                      "fp32_tflops_derived": fp32_derived}}
    del J

    # ---------------- plain arm: per-view launches ----------------
    plain = None
    if not args.no_plain:
        reset(W)
        Pl = PlainStep(torch, gs, W, device)
        for _ in range(args.warmup):
            Pl.step()
        torch.cuda.synchronize()
        pms = max_over_ranks(timed(torch, Pl.step, args.steps, barrier))
        plain = {"value": world * args.views * args.steps / (pms / 1000.0), "unit": UNIT,
                 "ms_per_step": pms / args.steps, "status_ok": Pl.ok(),
                 "config": "tile 16, default batches, one CTA per tile, no graph"}
        del Pl

    # ---------------- end to end through the public API with host buffers ----------------
    reset(W)
    host_targets = W["targets"].cpu().pin_memory()
    host_loss = torch.zeros((1,), dtype=torch.float32).pin_memory()
    pipe = HostTargets(torch, host_targets, W["targets"])
    E = JointOptimizer(W["g"], W["cams"], W["sizes"], pipe.bufs[0], capacity, cfg, device=device)

    def e2e_step():
        E.set_targets(pipe.next())
        E.step()
        host_loss.copy_(E.loss, non_blocking=True)

    pipe.start(args.warmup)
    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    pipe.start(args.steps)
    ems = max_over_ranks(timed(torch, e2e_step, args.steps, barrier))
    e2e = {"value": world * args.views * args.steps / (ems / 1000.0), "unit": UNIT,
           "h2d_bytes_per_step": int(host_targets.numel() * 4), "d2h_bytes_per_step": 4,
           "path": "JointOptimizer.step() (C-ABI calls); every step's targets copied from pinned host memory, "
                   "double-buffered on a side stream so the copy for the next step overlaps this one"}
    del E, pipe

    # ---------------- the other rows, timed on their own ----------------
    rows = None
    if not args.no_rows and args.views >= 1:
        reset(W)
        bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
        rows = measure_rows(torch, gs, W, device, {"hbm": hbm_peak, "bf16": bf16_peak})
        rows["mini_ba"] = measure_ba(torch, gs, device)
        rows["pose_refine"] = measure_ba_pose(torch, gs, device)
        rows["guided_matching"] = measure_guided(torch, gs, device, fp32_peak_tflops)

    # ---------------- uneven views: 2M Gaussians, 16 views of mixed resolution ----------------
    uneven = None
    if not args.no_uneven:
        del W
        torch.cuda.empty_cache()
        rng_sz = np.random.Generator(np.random.PCG64(SEED + 1 + 7919))
        sizes_u = synth.uneven_sizes(rng_sz, 16)
        U = make_workload(torch, gs, synth, device, 2 * args.n, 16, sizes=sizes_u, seed=SEED + 1)
        cap_u = int(U["pairs"] * 1.3) + 4096
        cfg_u = U["cfg"]
        if not args.no_autotune:
            cfg_u, _ = autotune.tune(U["g"], U["cams"], U["sizes"], U["targets"], U["cfg"], steps=2, device=device,
                                     log=log)
            reset(U)
        Ju = JointOptimizer(U["g"], U["cams"], U["sizes"], U["targets"], cap_u, cfg_u, device=device)
        Ju.r.fit_capacity(U["g"], U["cams"])
        Ju.step()
        torch.cuda.synchronize()
        Ju.capture(per_stage=False)
        for _ in range(args.warmup):
            Ju.replay()
        torch.cuda.synchronize()
        ums = max_over_ranks(timed(torch, Ju.replay, args.steps, barrier))
        u_ok = Ju.r.status() == gs.GS_OK
        del Ju
        reset(U)
        Pu = PlainStep(torch, gs, U, device)
        for _ in range(args.warmup):
            Pu.step()
        torch.cuda.synchronize()
        pums = max_over_ranks(timed(torch, Pu.step, args.steps, barrier))
        pix = sum(w * h for w, h in sizes_u)
        uneven = {"workload": "2M Gaussians SH3, 16 views " + ",".join(f"{w}x{h}" for w, h in sizes_u),
                  "unit": "Mpix fwd+bwd/s",
                  "batched": {"value": world * pix * args.steps / (ums / 1000.0) / 1e6, "ms_per_step": ums / args.steps,
                              "config": {"tile": cfg_u.tile, "fwd_batch": cfg_u.fwd_batch,
                                         "bwd_batch": cfg_u.bwd_batch,
                                         "schedule": SCHEDULES[cfg_u.schedule],
                                         "graph": "whole step"}, "status_ok": u_ok},
                  "plain": {"value": world * pix * args.steps / (pums / 1000.0) / 1e6,
                            "ms_per_step": pums / args.steps, "status_ok": Pu.ok()}}
        del Pu, U

    # ---------------- oracle on the host cores ----------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, dt, cores = oracle_sample(args.cpu_views, args.n)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "seconds": dt,
               "sample": f"{args.cpu_views} of the 8 views: fwd+bwd (incl. pose) at 1920x1080 over the full "
                         f"{args.n}-Gaussian scene, FP64"}

    if rank == 0:
        # the full record (stages, side rows, autotune trials) goes to stderr; stdout carries one compact line
        detail = {"stages": stages, "rows": rows, "launch": tuned, "uneven": uneven, "plain": plain,
                  "work": {"visible_items": n_items_vis, "pairs": P, "evaluations_composited": K_c,
                           "list_entries": K, "loss": loss, "status": status}}
        log("detail " + json.dumps(detail))
        r3 = lambda x: None if x is None else float(f"{x:.4g}")
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(args.n, args.views),
                       "arm": "batched: all views per launch, CUDA graph per stage",
                       "launch": ({k: tuned[k] for k in ("tile", "fwd_batch", "bwd_batch", "schedule")}
                                  if tuned else "defaults"),
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (parameters + Adam state 0.7 GB, projected buffers "
                             f"{args.views * args.n * 52 / 1e9:.2f} GB)"},
            "plain": None if plain is None else {"value": r3(plain["value"]), "ms_per_step": r3(plain["ms_per_step"])},
            "uneven": None if uneven is None else {
                "unit": uneven["unit"], "batched": r3(uneven["batched"]["value"]),
                "plain": r3(uneven["plain"]["value"]), "schedule": uneven["batched"]["config"]["schedule"]},
            "stage_ms": {k: r3(v["ms"]) for k, v in stages.items()},
            "stage_frac": {k: r3(v["frac"]) for k, v in stages.items()},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches_per_step * args.steps),
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
