"""End-to-end streaming checks (Sec. 4.2-4.4): the learned spawn proposal
against plain direct sampling (the fallback it is measured against), anchors,
the training-schedule variants and guided matching in the loop."""
import json
import os

import numpy as np
import pytest
import torch

from paper_2506_05558_gb300 import gs, synth
from paper_2506_05558_gb300.stream import OnTheFly, render_depth

pytestmark = pytest.mark.gpu

# where the streaming comparisons write their JSON reports
REPORT_DIR = os.environ.get("GS_REPORT_DIR", "test_reports")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2506_05558_gb300 import build
    build.build()


def make_stream(n_gt=60_000, n_frames=10, size=(256, 144), seed=21):
    sc, cams, _ = synth.multiview_scene(seed=seed, n=n_gt, n_views=n_frames, sizes=[size] * n_frames)
    sc.sh[:, 3:] = 0.0
    sc.scale[:, :3] += 2.0  # dense enough to cover most of a small frame
    g = gs.Gaussians.from_scene(sc)
    cfg = gs.config(sh_degree=0)
    frames = []
    for c in cams:
        ct = gs.cameras_tensor([c])
        color, depth = render_depth(g, ct, size, cfg)
        frames.append((color, depth, ct))
    return frames


def run(mode, frames, size, iters=20):
    otf = OnTheFly(2_000_000, size, window=3, iters=iters, mode=mode, mlp_warmup_frames=3, mlp_steps=30,
                   anchor_tau=0.0)  # spawning comparison without anchors
    for i, (img, depth, cam) in enumerate(frames):
        otf.add_frame(img, depth, cam, i)
    ev = [(img, cam) for img, _, cam in frames[-3:]]
    return otf.evaluate(ev), otf


def mono_depth(depth, size, seed, sd=0.1):
    """A monocular-style estimate: the true depth times exp(sd x a smooth random
    field) with a little per-pixel noise; uncovered pixels stay 0."""
    W, H = size
    gen = torch.Generator(device="cpu").manual_seed(seed)
    coarse = torch.randn((1, 1, 4, 6), generator=gen)
    field = torch.nn.functional.interpolate(coarse, size=(H, W), mode="bilinear", align_corners=True)[0, 0]
    fine = 0.02 * torch.randn((H, W), generator=gen)
    d = depth.reshape(H, W) * torch.exp(sd * field.cuda() + fine.cuda())
    return d.reshape(depth.shape).contiguous()


def test_learned_proposal_reaches_plain_psnr_in_fewer_iterations():
    """The learned proposal's target relation on a room of textured opaque
    surfaces (16 frames of 256x144 on the standard path) where both modes take
    spawn depths from a monocular-style estimate with a smooth 25% error (the
    paper's setting, Sec. 4.2; no mode sees the true depth): with 25 iterations
    per frame the learned proposal must come within 0.2 dB of plain direct
    sampling with 30. Budgets 15-30 are recorded for both modes, with the
    Gaussians each spawned, and the same comparison with the true depth."""
    size = (256, 144)
    n_frames = 16
    sc, cams = synth.surface_scene(n_views=n_frames, size=size)
    g = gs.Gaussians.from_scene(sc)
    cts = [gs.cameras_tensor([c]) for c in cams]
    rendered = [render_depth(g, ct, size, gs.config(sh_degree=0)) for ct in cts]
    monos = [mono_depth(d, size, 100 + i, sd=0.25) for i, (_, d) in enumerate(rendered)]
    empty = 10 * np.log10(1.0 / torch.mean(rendered[-1][0] ** 2).item())
    report = {"frames": n_frames, "size": size, "empty_render_psnr": empty, "mono": {}, "true_depth": {}}
    for depth_kind, budgets in (("mono", (15, 20, 25, 30)), ("true_depth", (20, 30))):
        frames = [(img, monos[i] if depth_kind == "mono" else d, cts[i]) for i, (img, d) in enumerate(rendered)]
        for iters in budgets:
            p_plain, a = run("plain", frames, size, iters)
            p_learn, b = run("learned", frames, size, iters)
            report[depth_kind][iters] = {"psnr_plain": p_plain, "psnr_learned": p_learn,
                                         "gaussians_plain": a.store.n, "gaussians_learned": b.store.n}
    os.makedirs(REPORT_DIR, exist_ok=True)
    with open(os.path.join(REPORT_DIR, "stream_learned_report.json"), "w") as f:
        json.dump(report, f, indent=1)
    print(json.dumps(report))
    m = report["mono"]
    assert m[25]["psnr_learned"] >= m[30]["psnr_plain"] - 0.2, report
    assert m[30]["psnr_plain"] > empty + 5, report


def test_learned_vs_plain_spawning_random_scene():
    """The same comparison on a scene of random small Gaussians, spawning from
    the true depth: recorded (the proposal loses here; no relation is
    asserted beyond both modes reconstructing)."""
    size = (256, 144)
    frames = make_stream(size=size)
    empty = 10 * np.log10(1.0 / torch.mean(frames[-1][0] ** 2).item())
    report = {"empty_render_psnr": empty, "frames": len(frames), "size": size, "budgets": {}}
    for iters in (10, 20, 30):
        p_plain, a = run("plain", frames, size, iters)
        p_learn, b = run("learned", frames, size, iters)
        report["budgets"][iters] = {"psnr_plain": p_plain, "psnr_learned": p_learn, "gaussians_plain": a.store.n,
                                    "gaussians_learned": b.store.n, "iterations": a.iter_count,
                                    "spawned_learned": [e["spawned"] for e in b.log],
                                    "spawned_plain": [e["spawned"] for e in a.log]}
        assert p_plain > empty + 5 and p_learn > empty + 3, report
    os.makedirs(REPORT_DIR, exist_ok=True)
    with open(os.path.join(REPORT_DIR, "stream_report.json"), "w") as f:
        json.dump(report, f, indent=1)


def test_anchors_in_the_stream():
    """With a 50-pixel size threshold anchors trigger: each stores the active set
    on the host and the merge shrinks it; the final set is stored in a last
    anchor and a training view rendered from the anchors (closest or blended)
    still reconstructs the frame."""
    size = (256, 144)
    frames = make_stream(size=size)
    empty = 10 * np.log10(1.0 / torch.mean(frames[-1][0] ** 2).item())
    otf = OnTheFly(2_000_000, size, window=3, iters=20, mode="plain", anchor_tau=50.0, merge_radius=0.5)
    for i, (img, depth, cam) in enumerate(frames):
        otf.add_frame(img, depth, cam, i)
    merges = [e["anchor"] for e in otf.log if e["anchor"]]
    assert merges, otf.log
    for a in merges:
        assert a["after"] < a["before"] and a["too_fine"] > 0.4 * a["before"]
    otf.finish(frames[-1][2])
    assert len(otf.anchors) == len(merges) + 1
    from paper_2506_05558_gb300.stream import psnr
    img, _, cam = frames[-1]
    p_active = otf.evaluate([(img, cam)])
    p_anchor = psnr(otf.render_anchors(cam), img)
    report = {"merges": merges, "psnr_active": p_active, "psnr_from_anchors": p_anchor, "empty": empty,
              "anchors": [dict(location=a.location.tolist(), n=a.n) for a in otf.anchors]}
    os.makedirs(REPORT_DIR, exist_ok=True)
    with open(os.path.join(REPORT_DIR, "stream_anchor_report.json"), "w") as f:
        json.dump(report, f, indent=1)
    assert p_active > empty + 3 and p_anchor > empty + 3, report


def test_training_schedule_variants():
    """The schedule variants of the joint optimisation (Sec. 4.3, App. A.3):
    coarse-to-fine from 2^3 downsampling with the integral-keeping filter,
    per-Gaussian rate decay and opacity culling, each on its own and together,
    against the plain schedule at 20 iterations per frame."""
    size = (256, 144)
    frames = make_stream(size=size)
    empty = 10 * np.log10(1.0 / torch.mean(frames[-1][0] ** 2).item())
    # culling bound 0.05 (3DGS uses 0.005, which nothing reaches in these short runs)
    variants = {"plain": {}, "coarse_to_fine": dict(coarse_to_fine=3, mip_filter=True),
                "lr_decay": dict(lr_decay=0.995), "cull": dict(min_opacity=0.05),
                "all": dict(coarse_to_fine=3, mip_filter=True, lr_decay=0.995, min_opacity=0.05)}
    report = {"empty_render_psnr": empty}
    for name, kw in variants.items():
        otf = OnTheFly(2_000_000, size, window=3, iters=20, mode="plain", anchor_tau=0.0, **kw)
        for i, (img, depth, cam) in enumerate(frames):
            otf.add_frame(img, depth, cam, i)
        p = otf.evaluate([(img, cam) for img, _, cam in frames[-3:]])
        report[name] = {"psnr": p, "gaussians": otf.store.n, "culled": sum(e["culled"] for e in otf.log)}
    os.makedirs(REPORT_DIR, exist_ok=True)
    with open(os.path.join(REPORT_DIR, "stream_schedule_report.json"), "w") as f:
        json.dump(report, f, indent=1)
    for name in variants:
        assert report[name]["psnr"] > empty + 5, (name, report)
    assert report["cull"]["culled"] > 0 and report["all"]["culled"] > 0, report


C0 = 0.28209479177387814


def render_features(sc, cams, size, channels=16, seed=3, period=(0.3, 1.0)):
    """Multi-view feature maps of the ground-truth scene, standing in for the
    dense feature network: every Gaussian carries the values in [0, 1] of a
    smooth random field of its position (mixtures of 8 sinusoids with periods
    in `period` metres), rendered three channels at a time as colours; per
    pixel the vector is centred and normalised, then rounded to bfloat16."""
    import copy
    rng = np.random.default_rng(seed)
    passes = (channels + 2) // 3
    dirs = rng.normal(size=(8, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    omega = dirs * (2 * np.pi / rng.uniform(*period, 8))[:, None]
    field = np.sin(sc.mean_opa[:, :3].astype(np.float64) @ omega.T + rng.uniform(0, 2 * np.pi, 8))
    vals = field @ rng.normal(size=(8, 3 * passes))
    vals = (1.0 / (1.0 + np.exp(-vals))).astype(np.float32)  # into [0, 1]
    W, H = size
    maps = [[] for _ in cams]
    cfg = gs.config(sh_degree=0)
    for p in range(passes):
        sp = copy.deepcopy(sc)
        sp.sh[:, :3] = (vals[:, 3 * p:3 * p + 3] - 0.5) / C0
        g = gs.Gaussians.from_scene(sp)
        for i, ct in enumerate(cams):
            color, _ = render_depth(g, ct, size, cfg)
            maps[i].append(color.reshape(3, H, W))
    out = []
    for m in maps:
        f = torch.cat(m)[:channels].permute(1, 2, 0)  # [H][W][C]
        f = f - f.mean(-1, keepdim=True)
        f = f / f.norm(dim=-1, keepdim=True).clamp_min(1e-6)
        out.append(f.to(torch.bfloat16).view(torch.int16).contiguous())
    return out


def test_guided_matching_refines_the_spawn_depth():
    """Guided matching in the loop (Sec. 4.2, App. A.2) on a room of textured
    surfaces: spawning from a smooth 25%-error monocular depth, from that depth
    refined against the previous frames' feature maps, and from the true depth.
    The refined depth (two previous frames as neighbours) is closer to the
    truth than the monocular one - most frames reach 0.006-0.015 in inverse
    depth, a few stay near their monocular error where the matching fails -
    and the PSNR each reaches is recorded (the optimisation corrects spawn
    depth errors, so it differs little)."""
    size = (256, 144)
    n_frames = 10
    # textured opaque surfaces (the matching assumes them): rendered images and
    # feature maps agree across views
    sc, cams = synth.surface_scene(n_views=n_frames, size=size)
    g = gs.Gaussians.from_scene(sc)
    cts = [gs.cameras_tensor([c]) for c in cams]
    frames = [render_depth(g, ct, size, gs.config(sh_degree=0)) for ct in cts]
    feats = render_features(sc, cts, size)
    monos = [mono_depth(d, size, 100 + i, sd=0.25) for i, (_, d) in enumerate(frames)]
    # depth quality on the frames that have neighbours
    W, H = size
    errs = {"mono": [], "guided": []}
    for i in range(1, n_frames):
        prev = list(range(max(0, i - 2), i))
        stack = torch.stack([feats[i]] + [feats[j] for j in prev[::-1]]).contiguous()
        camst = torch.cat([cts[i]] + [cts[j] for j in prev[::-1]])
        ref = gs.gs_guided_depth(stack, camst, monos[i].reshape(H, W).contiguous()).reshape(-1)
        gt = frames[i][1].reshape(-1)
        v = gt > 0
        errs["mono"].append(torch.median((1 / monos[i][v] - 1 / gt[v]).abs()).item())
        errs["guided"].append(torch.median((1 / ref[v] - 1 / gt[v]).abs()).item())
    report = {k: float(np.mean(v)) for k, v in errs.items()}
    psnr = {}
    for name in ("gt", "mono", "guided"):
        otf = OnTheFly(2_000_000, size, window=3, iters=20, mode="plain", anchor_tau=0.0,
                       guided_neighbours=2 if name == "guided" else 0)
        for i, (img, depth) in enumerate(frames):
            d = depth if name == "gt" else monos[i]
            otf.add_frame(img, d, cts[i], i, feats=feats[i] if name == "guided" else None)
        psnr[name] = otf.evaluate([(img, cts[i]) for i, (img, _) in enumerate(frames)][-3:])
    report.update({f"psnr_{k}": v for k, v in psnr.items()})
    os.makedirs(REPORT_DIR, exist_ok=True)
    with open(os.path.join(REPORT_DIR, "stream_guided_report.json"), "w") as f:
        json.dump(report, f, indent=1)
    print(report)
    assert report["guided"] < 0.9 * report["mono"], report
    assert psnr["guided"] > psnr["mono"] - 0.3, report
