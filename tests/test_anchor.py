"""Anchor trigger (Sec. 4.4): the oracle's on-screen size against the
independently coded EWA projection (CPU), then the GPU flags, count and the
host offload / reload round trip (GPU)."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2506_05558_gb300 import gs, synth


def test_anchor_size_equals_projected_sigma_on_axis():
    """An isotropic Gaussian on the optical axis at depth z projects (EWA, no
    dilation) to a circle of standard deviation fx S / z pixels: the anchor size
    with D = z."""
    cam = synth.camera(np.eye(3), np.zeros(3), 700.0, 640, 480, dtype=np.float64)
    for z, S in ((3.0, 0.01), (12.0, 0.002), (40.0, 0.05)):
        mo = np.array([[0.0, 0.0, z, 0.0]])
        sc = synth.Scene(mo, np.array([[math.log(S)] * 3 + [0.0]]), np.array([[1.0, 0, 0, 0]]), np.zeros((1, 48)), 0)
        p = O.project(sc, cam, O.Config(sh_degree=0, dilation=0.0))
        a, b, c = p["conic"][0]
        sigma_px = math.sqrt(c / (a * c - b * b))
        assert abs(O.anchor_sizes(sc, cam)[0] - sigma_px) < 1e-9 * sigma_px


def test_anchor_rule_forty_percent():
    rng = np.random.default_rng(0)
    sc, cams, _ = synth.multiview_scene(seed=4, n=2000, n_views=2)
    res = O.anchor_check(sc, cams[0])
    assert res["due"] == (res["count"] > 0.4 * sc.n)
    # shrinking every Gaussian makes most of them too fine
    sc.scale[:, :3] -= 3.0
    assert O.anchor_check(sc, cams[0])["due"]


@pytest.mark.gpu
def test_anchor_check_and_offload_on_gpu():
    from paper_2506_05558_gb300 import build
    build.build()
    sc, cams, _ = synth.multiview_scene(seed=4, n=300_000, n_views=2)
    g = gs.Gaussians.from_scene(sc)
    cam = gs.cameras_tensor([cams[1]])
    fine = torch.zeros(sc.n, dtype=torch.uint8, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    gs.gs_anchor_check(g, cam, 1.0, fine, count)
    torch.cuda.synchronize()
    ref = O.anchor_check(sc, cams[1])
    got = fine.cpu().numpy().astype(bool)
    ok = ~ref["amb"]
    assert np.array_equal(got[ok], ref["too_fine"][ok])
    assert abs(int(count.item()) - ref["count"]) <= int(ref["amb"].sum())
    assert int(count.item()) == int(got.sum())
    # offload the set and two Adam-like states, scramble the device copies, load back
    m = gs.Gaussians.from_scene(synth.scene_subset(sc, np.arange(sc.n)[::-1].copy()))
    host = [gs.pinned_gaussians(sc.n) for _ in range(3)]
    gs.gs_anchor_offload(g, m, m, host[0], host[1], host[2])
    torch.cuda.synchronize()
    want = [t.cpu().clone() for t in (g.mean_opa, g.scale, g.quat, g.sh, m.sh)]
    for t in (g.mean_opa, g.scale, g.quat, g.sh, m.sh):
        t.zero_()
    gs.gs_anchor_load(host[0], host[1], None, g, m, None)
    torch.cuda.synchronize()
    for a, b in zip((g.mean_opa, g.scale, g.quat, g.sh, m.sh), want):
        assert torch.equal(a.cpu(), b)
