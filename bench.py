#!/usr/bin/env python
"""Throughput of the joint pose + Gaussian optimisation step on one GB300.

Workload (the headline configuration): 1,000,000 Gaussians with degree-3 SH
(fp32), 8 views of 1920x1080 on a smooth camera path (0.3 m / 5 degrees between
frames), poses perturbed by N(0, 0.01) rad/m. One step renders every view,
takes the L1 loss against the targets, runs the adjoint (Gaussian and SE(3)
pose gradients), a sparse Adam step on the visible Gaussians and an Adam +
retraction step on the poses. The metric counts view iterations: one
iteration = project + sort + render forward + render backward (with pose) of
one 1080p view. Inputs are synthetic (seeded), far larger than L2.

Two arms of the same step are timed: "batched" (all 8 views in each launch,
the value reported) and "plain" (one launch sequence per view).

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

# Algorithmic work per (pixel, Gaussian) evaluation, counted from the
# definitions of the compositing forward and its adjoint (FMA = 2 flops).
FWD_FLOPS_PER_EVAL = 22
BWD_FLOPS_PER_EVAL = 63
SMS = 152
FP32_LANES = 128


def log(*a):
    print(*a, file=sys.stderr, flush=True)


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
                                          "--format=csv,noheader,nounits", "-lms", "200"],
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
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
# workload
# ---------------------------------------------------------------------------
def make_workload(torch, gs, synth, device, n=N_GAUSS, n_views=N_VIEWS):
    from paper_2506_05558_gb300.raster import Rasterizer
    sc, cams, rng = synth.multiview_scene(seed=SEED, n=n, n_views=n_views)
    sizes = [(c["width"], c["height"]) for c in cams]
    cfg = gs.config(sh_degree=3)
    g_true = gs.Gaussians.from_scene(sc, device)
    cams_true = gs.cameras_tensor(cams, device)
    # targets: renders of the true scene from the true poses (setup, untimed)
    r = Rasterizer(n, sizes, capacity=1 << 20, cfg=cfg, device=device)
    p = r.fit_capacity(g_true, cams_true)
    r.forward(g_true, cams_true)
    targets = r.img.color.clone()
    # training state: jittered means, perturbed poses
    sc.mean_opa[:, :3] += rng.normal(0, 0.01, (n, 3)).astype(np.float32)
    g = gs.Gaussians.from_scene(sc, device)
    pert = []
    for c in cams:
        R, t = synth.perturb_pose(rng, c["R"].astype(np.float64), c["t"].astype(np.float64))
        pert.append(dict(c, R=R.astype(np.float32), t=t.astype(np.float32)))
    cams_train = gs.cameras_tensor(pert, device)
    del r
    torch.cuda.synchronize()
    return sc, sizes, cfg, g, cams_train, targets, p


class BatchedStep:
    """All views per launch (the library's multi-view path)."""

    STAGES = ("project", "sort", "render_fwd", "loss", "composite_bwd", "project_bwd", "adam", "pose")

    def __init__(self, torch, gs, g, cams, sizes, targets, cfg, capacity, device):
        from paper_2506_05558_gb300.raster import Rasterizer
        self.torch, self.gs = torch, gs
        self.g, self.cams, self.targets = g, cams, targets
        self.r = Rasterizer(g.n, sizes, capacity, cfg, device)
        self.m, self.v = gs.Gaussians.zeros(g.n, device), gs.Gaussians.zeros(g.n, device)
        nv = len(sizes)
        self.pm = torch.zeros((nv, 6), device=device)
        self.pv = torch.zeros((nv, 6), device=device)
        self.dL = torch.zeros_like(self.r.img.color)
        self.loss = torch.zeros((1,), device=device)
        self.ws_loss = gs.workspace(4 * 4096, device)
        self.adam = gs.adam_config()
        self.t = 0

    def step(self, ev=None):
        gs, r = self.gs, self.r
        self.t += 1
        rec = (lambda i: ev[i].record()) if ev is not None else (lambda i: None)
        rec(0)
        gs.gs_project(self.g, self.cams, r.f, r.cfg, r.proj)
        rec(1)
        gs.gs_sort(r.proj, r.n, r.f, r.pairs, r.ws_sort)
        rec(2)
        gs.gs_render_fwd(r.proj, r.pairs, r.f, r.cfg, r.img)
        rec(3)
        gs.gs_l1_loss(r.img.color, self.targets, self.dL, self.loss, self.ws_loss)
        rec(4)
        gs.gs_composite_bwd(r.proj, r.pairs, r.f, r.cfg, r.img, self.dL, r.n, r.ws_bwd)
        rec(5)
        gs.gs_project_bwd(self.g, self.cams, r.proj, r.pairs, r.f, r.cfg, r.grads, r.dpose, r.ws_bwd)
        rec(6)
        gs.gs_adam_step(self.g, r.grads, self.m, self.v, self.adam, self.t)
        rec(7)
        gs.gs_pose_step(self.cams, r.n_views, r.dpose, self.pm, self.pv, 1e-3, 1e-3, self.t)
        rec(8)
        return self.loss


class PlainStep:
    """One launch sequence per view (views rendered one after another); the
    gradients of all views are accumulated before the single optimiser step."""

    def __init__(self, torch, gs, g, cams, sizes, targets, cfg, capacity_per_view, device):
        from paper_2506_05558_gb300.raster import Rasterizer
        self.torch, self.gs = torch, gs
        self.g, self.targets = g, targets
        self.sizes = sizes
        nv = len(sizes)
        self.cams = cams
        cam_bytes = 72
        self.cam_views = [cams[v * cam_bytes:(v + 1) * cam_bytes] for v in range(nv)]
        self.rs = []
        for v in range(nv):
            cfg_v = gs.config(sh_degree=cfg.sh_degree, accumulate=1 if v > 0 else 0)
            self.rs.append(Rasterizer(g.n, [sizes[v]], capacity_per_view, cfg_v, device))
        self.grads = self.rs[0].grads
        for r in self.rs[1:]:
            r.grads = self.grads  # one accumulation buffer
        self.dpose = torch.zeros((nv, 6), device=device)
        self.m, self.v = gs.Gaussians.zeros(g.n, device), gs.Gaussians.zeros(g.n, device)
        self.pm = torch.zeros((nv, 6), device=device)
        self.pv = torch.zeros((nv, 6), device=device)
        self.dLs = [torch.zeros_like(r.img.color) for r in self.rs]
        self.loss = torch.zeros((nv,), device=device)
        self.ws_loss = gs.workspace(4 * 4096, device)
        offs = np.cumsum([0] + [3 * w * h for w, h in sizes])
        self.tgt = [targets[offs[v]:offs[v + 1]] for v in range(nv)]
        self.adam = gs.adam_config()
        self.t = 0

    def step(self):
        gs = self.gs
        self.t += 1
        for v, r in enumerate(self.rs):
            cam = self.cam_views[v]
            gs.gs_project(self.g, cam, r.f, r.cfg, r.proj)
            gs.gs_sort(r.proj, r.n, r.f, r.pairs, r.ws_sort)
            gs.gs_render_fwd(r.proj, r.pairs, r.f, r.cfg, r.img)
            gs.gs_l1_loss(r.img.color, self.tgt[v], self.dLs[v], self.loss[v:v + 1], self.ws_loss)
            gs.gs_render_bwd(self.g, cam, r.proj, r.pairs, r.f, r.cfg, r.img, self.dLs[v], self.grads,
                             self.dpose[v:v + 1], r.ws_bwd)
        gs.gs_adam_step(self.g, self.grads, self.m, self.v, self.adam, self.t)
        gs.gs_pose_step(self.cams, len(self.rs), self.dpose, self.pm, self.pv, 1e-3, 1e-3, self.t)
        return self.loss


# ---------------------------------------------------------------------------
# oracle on the host cores
# ---------------------------------------------------------------------------
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


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state beyond the first build
    from oracle import build as ob
    ob.build()
    vals = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        v, dt, cores = oracle_sample(1)
        vals.append(dt)
    total = time.perf_counter() - t_all
    value = len(vals) / sum(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(vals) / len(vals),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "joint optimisation view iteration, 1M Gaussians SH3, 1920x1080",
                       "step_sample": "1 of the 8 views per step (FP64 oracle on the host cores)"},
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
    ap.add_argument("--cpu-views", type=int, default=3, help="views of the oracle CPU sample")
    args = ap.parse_args()
    if args.warmup < 3:
        log("warm-up raised to 3 (timing rule)")
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    from paper_2506_05558_gb300 import gs, synth

    torch.cuda.set_device(local_rank)
    device = f"cuda:{local_rank}"
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(device))

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x):
        if world == 1:
            return x
        t = torch.tensor([x], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    gs.lib()
    sc, sizes, cfg, g, cams, targets, pairs_true = make_workload(torch, gs, synth, device, args.n, args.views)
    g0 = [t.clone() for t in (g.mean_opa, g.scale, g.quat, g.sh)]
    cams0 = cams.clone()
    capacity = int(pairs_true * 1.3) + 4096

    # ---------------- batched arm ----------------
    B = BatchedStep(torch, gs, g, cams, sizes, targets, cfg, capacity, device)
    B.r.fit_capacity(g, cams)
    for _ in range(args.warmup):
        B.step()
    torch.cuda.synchronize()
    assert B.r.status() == gs.GS_OK, "pair buffer overflow"
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(9)] for _ in range(args.steps)]
    clocks = ClockSampler(local_rank)
    launches0 = gs.gs_launch_count()
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record()
    for k in range(args.steps):
        B.step(ev[k])
    t_end.record()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = gs.gs_launch_count() - launches0
    ms_local = t_start.elapsed_time(t_end)
    ms = max_over_ranks(ms_local)
    stage_ms = {s: float(np.mean([ev[k][i].elapsed_time(ev[k][i + 1]) for k in range(args.steps)]))
                for i, s in enumerate(BatchedStep.STAGES)}
    value = world * args.views * args.steps / (ms / 1000.0)
    status = B.r.status()
    # work counts of the last step (untimed accounting)
    n_items_vis = int((B.r.proj.n_tiles > 0).sum().item())
    P = B.r.pair_count()
    K = int(B.r.img.n_contrib.to(torch.int64).sum().item())
    loss = float(B.loss.item())

    # ---------------- roofline of the dominant kernel ----------------
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    sm_clock = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak_tflops = SMS * FP32_LANES * 2 * sm_clock * 1e6 / 1e12
    algo = {
        "render_fwd": ("alu", FWD_FLOPS_PER_EVAL * K / 1e12, "TFLOP/s"),
        "composite_bwd": ("alu", BWD_FLOPS_PER_EVAL * K / 1e12, "TFLOP/s"),
        "project": ("hbm", (16 * args.n * args.views + (224 + 56) * n_items_vis) / 1e9, "GB/s"),
        "project_bwd": ("hbm", ((240 + 240) * args.n + (36 + 16) * n_items_vis + 36 * P) / 1e9, "GB/s"),
        "adam": ("hbm", 7 * 240 * args.n / 1e9, "GB/s"),
    }
    stages = {}
    for s, msv in stage_ms.items():
        e = {"ms": msv}
        if s in algo:
            bound, work, unit = algo[s]
            ach = work / (msv / 1000.0)
            peak = fp32_peak_tflops if bound == "alu" else hbm_peak
            e.update({"bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak})
        stages[s] = e
    dom = max(stage_ms, key=lambda s: stage_ms[s])
    if dom in algo:
        d = stages[dom]
        roof = {"kernel": dom, "bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"], "unit": d["unit"],
                "frac": d["frac"], "traffic": None,
                "peak_source": ("FP32: 152 SMs x 128 lanes x 2 flop x median SM clock under load"
                                if d["bound"] == "alu" else "MEASURED_PEAKS.json hbm_gbs (of measured)")}
    else:
        roof = {"kernel": dom, "bound": None, "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": None}

    # ---------------- plain arm ----------------
    plain = None
    if not args.no_plain:
        for t, s in zip((g.mean_opa, g.scale, g.quat, g.sh), g0):
            t.copy_(s)
        cams.copy_(cams0)
        cap_v = int(capacity / args.views * 1.6) + 4096
        Pl = PlainStep(torch, gs, g, cams, sizes, targets, cfg, cap_v, device)
        for r, cam in zip(Pl.rs, Pl.cam_views):
            r.fit_capacity(g, cam)
        for _ in range(args.warmup):
            Pl.step()
        torch.cuda.synchronize()
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            Pl.step()
        b.record()
        torch.cuda.synchronize()
        barrier()
        pms = max_over_ranks(a.elapsed_time(b))
        plain = {"value": world * args.views * args.steps / (pms / 1000.0), "unit": UNIT, "ms_per_step": pms / args.steps,
                 "status_ok": all(r.status() == gs.GS_OK for r in Pl.rs)}
        del Pl

    # ---------------- end to end through the public API with host buffers ----------------
    for t, s in zip((g.mean_opa, g.scale, g.quat, g.sh), g0):
        t.copy_(s)
    cams.copy_(cams0)
    host_targets = targets.cpu().pin_memory()
    host_loss = torch.zeros((1,), dtype=torch.float32).pin_memory()
    E = BatchedStep(torch, gs, g, cams, sizes, torch.empty_like(targets), cfg, capacity, device)
    for _ in range(args.warmup):
        E.targets.copy_(host_targets, non_blocking=True)
        E.step()
        host_loss.copy_(E.loss, non_blocking=True)
    torch.cuda.synchronize()
    barrier()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        E.targets.copy_(host_targets, non_blocking=True)
        E.step()
        host_loss.copy_(E.loss, non_blocking=True)
    b.record()
    torch.cuda.synchronize()
    barrier()
    ems = max_over_ranks(a.elapsed_time(b))
    e2e = {"value": world * args.views * args.steps / (ems / 1000.0), "unit": UNIT,
           "h2d_bytes_per_step": int(host_targets.numel() * 4), "d2h_bytes_per_step": 4}
    del E

    # ---------------- oracle on the host cores ----------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, dt, cores = oracle_sample(args.cpu_views, args.n)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "seconds": dt,
               "sample": f"{args.cpu_views} of the 8 views: fwd+bwd (incl. pose) at 1920x1080 over the full "
                         f"{args.n}-Gaussian scene, FP64"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"joint pose+Gaussian optimisation step: {args.n} Gaussians SH3, {args.views} "
                                   f"views {WIDTH}x{HEIGHT}, L1 + adjoint with SE(3) pose gradients + sparse Adam",
                       "arm": "batched (all views per launch)", "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (parameters+Adam state 0.7 GB, projected buffers "
                             f"{args.views * args.n * 56 / 1e9:.2f} GB)"},
            "plain": plain,
            "roofline": roof,
            "stages": stages,
            "work": {"visible_items": n_items_vis, "pairs": P, "evaluations": K, "loss": loss,
                     "status": status},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
