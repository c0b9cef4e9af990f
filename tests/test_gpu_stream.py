"""End-to-end streaming check of the learned spawn proposal against plain
direct sampling (Sec. 4.2 as the fallback and judge): both reconstruct a
synthetic scene frame by frame with the same iteration budget; the test
records the PSNR each reaches and the Gaussians each spawned, and requires both
to reconstruct (PSNR well above the empty render)."""
import json
import os

import numpy as np
import pytest
import torch

from paper_2506_05558_gb300 import gs, synth
from paper_2506_05558_gb300.stream import OnTheFly, render_depth

pytestmark = pytest.mark.gpu


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


def test_learned_vs_plain_spawning():
    """Both modes at 10, 20 and 30 iterations per frame; the report records
    PSNR and set size per budget."""
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
    os.makedirs("gpurun_out", exist_ok=True)
    with open("gpurun_out/stream_report.json", "w") as f:
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
    os.makedirs("gpurun_out", exist_ok=True)
    with open("gpurun_out/stream_anchor_report.json", "w") as f:
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
    os.makedirs("gpurun_out", exist_ok=True)
    with open("gpurun_out/stream_schedule_report.json", "w") as f:
        json.dump(report, f, indent=1)
    for name in variants:
        assert report[name]["psnr"] > empty + 5, (name, report)
    assert report["cull"]["culled"] > 0 and report["all"]["culled"] > 0, report
