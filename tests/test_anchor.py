"""Anchor trigger (Sec. 4.4): the oracle's on-screen size against the
independently coded EWA projection (CPU), then the GPU flags, count and the
host offload / reload round trip (GPU)."""
import math

import numpy as np
import pytest
import torch

from helpers import assert_close
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


# ---------------------------------------------------------------------------
# Merging at an anchor and the blending weight (oracle pins, CPU)
# ---------------------------------------------------------------------------

def _rot_quat(rng):
    q = rng.standard_normal(4)
    return q / np.linalg.norm(q)


def test_merge_group_single_and_duplicate():
    rng = np.random.default_rng(2)
    mo = np.array([[0.3, -1.0, 4.0, 0.2]])
    sc = np.array([[-3.0, -2.5, -3.4, 0.0]])
    q = np.array([_rot_quat(rng)])
    sh = rng.standard_normal((1, 48))
    mu, cov, op, shm = O.merge_group(mo, sc, q, sh)
    o = 1 / (1 + math.exp(-0.2))
    np.testing.assert_allclose(mu, mo[0, :3], rtol=1e-14)
    np.testing.assert_allclose(cov, O.covariance(sc[0], q[0]), rtol=1e-12, atol=1e-18)
    assert abs(op - o) < 1e-12
    np.testing.assert_allclose(shm, sh[0], rtol=1e-14)
    # two copies: same geometry and colour, opacity doubled (total o * area kept)
    mu2, cov2, op2, _ = O.merge_group(np.repeat(mo, 2, 0), np.repeat(sc, 2, 0), np.repeat(q, 2, 0),
                                      np.repeat(sh, 2, 0))
    np.testing.assert_allclose(cov2, cov, rtol=1e-12, atol=1e-18)
    assert abs(op2 - min(0.99, 2 * o)) < 1e-12


def test_merge_group_symmetric_pair_closed_form():
    """Two equal isotropic Gaussians at +-d on x: mean 0, covariance
    sigma^2 I + diag(d^2, 0, 0)."""
    sig, d = 0.05, 0.2
    mo = np.array([[d, 0, 5, 0.0], [-d, 0, 5, 0.0]])
    sc = np.log(np.array([[sig, sig, sig, 1.0]] * 2))
    q = np.array([[1.0, 0, 0, 0]] * 2)
    mu, cov, op, _ = O.merge_group(mo, sc, q, np.zeros((2, 48)))
    np.testing.assert_allclose(mu, [0, 0, 5], atol=1e-15)
    np.testing.assert_allclose(cov, np.diag([sig ** 2 + d ** 2, sig ** 2, sig ** 2]), rtol=1e-12)
    # opacity keeps sum o a: 2 * 0.5 * sig^2 = o * sig * sqrt(sig^2 + d^2)
    assert abs(op - min(0.99, sig / math.sqrt(sig ** 2 + d ** 2))) < 1e-12


def test_merge_group_matches_the_mixture_moments():
    """Monte Carlo: samples of the w-weighted mixture of the group's Gaussians
    have the merged mean and covariance (law of total covariance)."""
    rng = np.random.default_rng(3)
    g = 4
    mo = np.concatenate([rng.normal(0, 0.3, (g, 3)), rng.normal(0, 1, (g, 1))], 1)
    sc = np.concatenate([rng.normal(-2.5, 0.4, (g, 3)), np.zeros((g, 1))], 1)
    q = np.array([_rot_quat(rng) for _ in range(g)])
    mu, cov, _, _ = O.merge_group(mo, sc, q, np.zeros((g, 48)))
    o = 1 / (1 + np.exp(-mo[:, 3]))
    ss = np.sort(np.exp(sc[:, :3]), 1)
    w = o * ss[:, 1] * ss[:, 2]
    counts = np.round(400_000 * w / w.sum()).astype(int)
    pts = np.concatenate([rng.multivariate_normal(mo[i, :3], O.covariance(sc[i], q[i]), counts[i])
                          for i in range(g)])
    np.testing.assert_allclose(pts.mean(0), mu, atol=4e-3)
    np.testing.assert_allclose(np.cov(pts.T), cov, atol=0.02 * np.abs(cov).max())


def test_anchor_merge_neighbours_claims_and_counts():
    """Proposals are the k nearest non-selected too-fine Gaussians within the
    radius (checked with scipy's k-d tree); each claimed Gaussian goes to the
    lowest selected index; the output drops exactly the claimed ones."""
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(5)
    n = 3000
    sc, _, _ = synth.multiview_scene(seed=9, n=n, n_views=1, sizes=[(64, 48)])
    fine = rng.random(n) < 0.6
    radius = 1.5
    r = O.anchor_merge(sc, fine, seed=17, radius=radius, k=3)
    sel = r["selected"]
    assert 0.15 < sel.sum() / fine.sum() < 0.35
    cand = np.nonzero(fine & ~sel)[0]
    tree = spatial.cKDTree(np.asarray(sc.mean_opa)[cand, :3])
    claim_ref = np.full(n, -1)
    for s in np.nonzero(sel)[0]:
        d, j = tree.query(np.asarray(sc.mean_opa)[s, :3], k=3, distance_upper_bound=radius)
        for dd, jj in zip(d, j):
            if np.isfinite(dd):
                c = cand[jj]
                if claim_ref[c] < 0:
                    claim_ref[c] = s  # selected Gaussians are visited in increasing index
    np.testing.assert_array_equal(r["claim"], claim_ref)
    assert len(r["src"]) == n - (claim_ref >= 0).sum()
    np.testing.assert_array_equal(r["src"], np.nonzero(claim_ref < 0)[0])
    np.testing.assert_array_equal(r["kind"], sel[r["src"]].astype(int))


def test_anchor_blend_weight():
    """w = 1 for r < 1 - o, 0.5 at r = 1, continuous at r = 1 - o, linear between."""
    o = 0.1
    assert O.anchor_blend_weight(1.0, 2.0, o) == 1.0
    assert abs(O.anchor_blend_weight(0.9, 1.0, o) - 1.0) < 1e-12
    assert abs(O.anchor_blend_weight(1.0, 1.0, o) - 0.5) < 1e-12
    assert abs(O.anchor_blend_weight(0.95, 1.0, o) - 0.75) < 1e-12


@pytest.mark.gpu
@pytest.mark.parametrize("with_moments", [False, True])
def test_anchor_merge_matches_oracle(with_moments):
    """GPU merge against the oracle on 20k Gaussians (60% too fine): the output
    count and the kept rows bit-exact (with their Adam moments), merged rows'
    mean, covariance, opacity and SH within tolerance, merged moments zero."""
    from paper_2506_05558_gb300 import build
    build.build()
    rng = np.random.default_rng(8)
    n, radius, seed = 20000, 1.2, 4243  # a seed with no neighbour decision within the FP32 margin
    sc, _, _ = synth.multiview_scene(seed=12, n=n, n_views=1, sizes=[(64, 48)])
    sc.mean_opa[:, 3] = rng.normal(0, 1, n)
    fine = (rng.random(n) < 0.6)
    ref = O.anchor_merge(sc, fine, seed=seed, radius=radius, k=3)
    assert ref["amb"].sum() == 0
    g = gs.Gaussians.from_scene(sc)
    out = gs.Gaussians.zeros(n)
    n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = gs.workspace(gs.gs_anchor_merge_workspace_size(n, 3))
    kw = {}
    if with_moments:
        m = gs.Gaussians(*[t.clone().normal_() for t in (g.mean_opa, g.scale, g.quat, g.sh)])
        v = gs.Gaussians(*[t.clone().uniform_() for t in (g.mean_opa, g.scale, g.quat, g.sh)])
        kw = dict(m=m, v=v, m_out=gs.Gaussians.zeros(n), v_out=gs.Gaussians.zeros(n),
                  lr=torch.rand(n, device="cuda") * 0.5 + 0.25, lr_out=torch.zeros(n, device="cuda"))
    gs.gs_anchor_merge(g, torch.tensor(fine.astype(np.uint8), device="cuda"), radius, seed, out, n_out, ws, **kw)
    torch.cuda.synchronize()
    k = int(n_out.item())
    assert k == len(ref["src"]) and k < n
    kept = ref["kind"] == 0
    src = ref["src"]
    for name in ("mean_opa", "scale", "quat", "sh"):
        got = getattr(out, name)[:k].cpu().numpy()
        want = getattr(g, name).cpu().numpy()[src]
        assert np.array_equal(got[kept], want[kept]), name
        if with_moments:
            for st, so in ((kw["m"], kw["m_out"]), (kw["v"], kw["v_out"])):
                mo_ = getattr(so, name)[:k].cpu().numpy()
                assert np.array_equal(mo_[kept], getattr(st, name).cpu().numpy()[src][kept])
                assert not mo_[~kept].any()
    mrg = ~kept
    assert mrg.sum() > 500
    if with_moments:
        lr_out = kw["lr_out"][:k].cpu().numpy()
        assert np.array_equal(lr_out[kept], kw["lr"].cpu().numpy()[src][kept]) and (lr_out[mrg] == 1.0).all()
    mo = out.mean_opa[:k].cpu().numpy()[mrg]
    assert_close(mo[:, :3], ref["mean"][mrg], 1e-5, what="merged mean")
    assert_close(1 / (1 + np.exp(-mo[:, 3].astype(np.float64))), ref["opacity"][mrg], 1e-4, what="merged opacity")
    ls = out.scale[:k].cpu().numpy()[mrg]
    q = out.quat[:k].cpu().numpy()[mrg]
    cov = np.array([O.covariance(ls[i], q[i]) for i in range(len(ls))])
    for i in range(len(ls)):
        assert_close(cov[i], ref["cov"][mrg][i], 1e-3, what=f"merged covariance {i}")
    assert_close(out.sh[:k].cpu().numpy()[mrg], ref["sh"][mrg], 1e-4, what="merged SH")


@pytest.mark.gpu
def test_anchor_blend_weight_and_opacity_scaling():
    from paper_2506_05558_gb300 import build
    build.build()
    for d1, d2 in ((1.0, 2.0), (0.95, 1.0), (1.0, 1.0), (0.9, 1.0)):
        assert abs(gs.gs_anchor_blend_weight(d1, d2, 0.1) - O.anchor_blend_weight(d1, d2, 0.1)) < 1e-6
    assert math.isnan(gs.gs_anchor_blend_weight(2.0, 1.0, 0.1))
    logit = torch.tensor([[0, 0, 0, 1.5], [0, 0, 0, -2.0], [0, 0, 0, 0.0]], device="cuda")
    o = 1 / (1 + np.exp(-logit[:, 3].cpu().numpy().astype(np.float64)))
    gs.gs_scale_opacity(logit, 0.25)
    torch.cuda.synchronize()
    got = 1 / (1 + np.exp(-logit[:, 3].cpu().numpy().astype(np.float64)))
    np.testing.assert_allclose(got, 0.25 * o, rtol=1e-5)



def test_cull_opacity_hand_case():
    logits = np.array([-6.0, -4.0, 0.0, -5.2933, 3.0, -10.0])  # sigmoid: 0.00247, 0.018, 0.5, 0.00500.., 0.95, 4.5e-5
    mo = np.zeros((6, 4))
    mo[:, 3] = logits
    kept, amb = O.cull_opacity(mo, 0.005)
    o = 1 / (1 + np.exp(-logits))
    np.testing.assert_array_equal(kept, [i for i in range(6) if o[i] >= 0.005])
    np.testing.assert_array_equal(kept, [1, 2, 3, 4])
    assert not amb.any()



@pytest.mark.gpu
def test_cull_opacity_matches_oracle():
    """Kept rows, their order, Adam moments and rate multipliers bit-exact."""
    from paper_2506_05558_gb300 import build
    build.build()
    rng = np.random.default_rng(3)
    n = 50_000
    sc, _, _ = synth.multiview_scene(seed=2, n=n, n_views=1, sizes=[(64, 48)])
    sc.mean_opa[:, 3] = rng.normal(-4, 2, n)
    kept, amb = O.cull_opacity(sc.mean_opa.astype(np.float32).astype(np.float64), 0.005, margin=1e-5)
    assert not amb.any()
    g = gs.Gaussians.from_scene(sc)
    m = gs.Gaussians(*[t.clone().normal_() for t in (g.mean_opa, g.scale, g.quat, g.sh)])
    v = gs.Gaussians(*[t.clone().uniform_() for t in (g.mean_opa, g.scale, g.quat, g.sh)])
    lr = torch.rand(n, device="cuda")
    out, mo, vo = gs.Gaussians.zeros(n), gs.Gaussians.zeros(n), gs.Gaussians.zeros(n)
    lr_out = torch.zeros(n, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = gs.workspace(gs.gs_cull_opacity_workspace_size(n))
    gs.gs_cull_opacity(g, 0.005, out, n_out, ws, m=m, v=v, m_out=mo, v_out=vo, lr=lr, lr_out=lr_out)
    torch.cuda.synchronize()
    k = int(n_out.item())
    assert k == len(kept) and 0.2 * n < k < 0.9 * n
    for src_set, dst_set in ((g, out), (m, mo), (v, vo)):
        for name in ("mean_opa", "scale", "quat", "sh"):
            assert np.array_equal(getattr(dst_set, name)[:k].cpu().numpy(),
                                  getattr(src_set, name).cpu().numpy()[kept]), name
    assert np.array_equal(lr_out[:k].cpu().numpy(), lr.cpu().numpy()[kept])
