"""Guided-matching depth refinement on the GPU (App. A.2) against the FP64
oracle on the same bfloat16 feature maps: neighbour choice bit-exact, refined
inverse depth within a tolerance set by the parabola's conditioning,
correlation within 1e-4 (unit-length features), pass-through pixels exact; all
channel counts, ragged sizes, a sampled check at 1920x1080, degenerate pixels,
determinism and argument checks."""
import numpy as np
import pytest
import torch

from oracle import guided as G
from paper_2506_05558_gb300 import gs, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2506_05558_gb300 import build
    build.build()


def run_gpu(sc, n_cand=32, window=0.1):
    feats = torch.from_numpy(sc["feats"].view(np.int16)).cuda()
    cams = gs.cameras_tensor(sc["cams"])
    z = torch.from_numpy(sc["z_mono"]).cuda()
    H, W = sc["z_mono"].shape
    nb = torch.empty((H, W), dtype=torch.int32, device="cuda")
    corr = torch.empty((H, W), dtype=torch.float32, device="cuda")
    depth = gs.gs_guided_depth(feats, cams, z, n_cand=n_cand, window=window, nb=nb, corr=corr)
    torch.cuda.synchronize()
    return depth.cpu().numpy(), nb.cpu().numpy(), corr.cpu().numpy()


def oracle(sc, n_cand=32, window=0.1, pixels=None):
    # the values the device reads: float32 poses and intrinsics
    f32 = lambda k, v: np.asarray(v, np.float32).astype(np.float64) if k in ("R", "t") else (
        float(np.float32(v)) if k in ("fx", "fy", "cx", "cy") else v)
    cams = [{k: f32(k, v) for k, v in c.items()} for c in sc["cams"]]
    return G.guided_depth(sc["feats"][0], sc["feats"][1:], cams[0], cams[1:], sc["z_mono"], n_cand=n_cand,
                          window=window, margins=True, pixels=pixels)


def compare(depth, nb, corr, z_mono, ref, max_flag=0.1):
    """Neighbour output bit-exact except where the FP32 path may decide the
    usability or the ranking the other way; the refined inverse depth within
    (1e-3 + 3e-5 / |curvature|) candidate steps of the oracle's (the parabola's
    offset moves by about the correlation error over its curvature). Where the
    two best correlations are within 1e-4 either may be the maximum, so the
    runner-up's outputs (neighbour, depth, curvature) are accepted too."""
    flag_nb = (ref["score_gap"] < 1e-4) | (ref["edge"] < 2e-3) | (ref["front"] < 1e-5)
    assert flag_nb.mean() <= max_flag, flag_nb.mean()
    ok = ~flag_nb
    tie = ref["arg_gap"] < 1e-4
    first = nb == ref["nb"]
    second = tie & (nb == ref["nb_alt"])
    assert (first | second)[ok].all(), np.count_nonzero(~(first | second)[ok])
    keep = ok & (nb < 0)
    assert np.array_equal(depth[keep], z_mono[keep].astype(np.float32), equal_nan=True)
    assert np.all(corr[keep] == 0)
    m = ok & (nb >= 0)
    step = ref["inv_step"]
    tol = (1e-3 + 3e-5 / np.maximum(np.abs(ref["den"]), 1e-12)) * step
    tol2 = (1e-3 + 3e-5 / np.maximum(np.abs(ref["den_alt"]), 1e-12)) * step
    with np.errstate(divide="ignore", invalid="ignore"):
        e1 = np.abs(1.0 / depth - 1.0 / ref["depth"])
        e2 = np.abs(1.0 / depth - 1.0 / ref["depth_alt"])
    good = (first & (e1 <= tol)) | (second & (e2 <= tol2))
    assert good[m].all(), (np.count_nonzero(~good[m]), (e1 / step)[m & ~good][:5])
    cerr = np.abs(corr - ref["cbest"])
    assert (cerr[m] < np.where(tie[m], 2e-4, 1e-4)).all(), cerr[m].max()
    return m.sum(), tie[m].mean()


@pytest.mark.parametrize("C,W,H,n_nb", [(32, 160, 120, 3), (16, 157, 118, 4), (8, 96, 70, 2), (64, 101, 67, 3)])
def test_parity_small(C, W, H, n_nb):
    sc = synth.guided_scene(seed=50 + C, width=W, height=H, f=W * 0.78, n_nb=n_nb, channels=C)
    depth, nb, corr = run_gpu(sc)
    ref = oracle(sc)
    n, ties = compare(depth, nb, corr, sc["z_mono"], ref)
    assert n > 0.7 * W * H  # most pixels are refined


def test_parity_candidate_counts_and_window():
    sc = synth.guided_scene(seed=61, width=128, height=96, f=100.0, n_nb=2, channels=32)
    for n_cand, window in ((3, 0.1), (17, 0.05), (64, 0.2)):
        depth, nb, corr = run_gpu(sc, n_cand, window)
        compare(depth, nb, corr, sc["z_mono"], oracle(sc, n_cand, window))


def test_full_size_sampled():
    """1920x1080, four neighbours, 32 channels, 32 candidates (the benchmark
    workload): 3000 sampled pixels against the oracle."""
    sc = synth.guided_scene()
    depth, nb, corr = run_gpu(sc)
    H, W = sc["z_mono"].shape
    pix = np.random.default_rng(0).choice(H * W, 3000, replace=False)
    ref = oracle(sc, pixels=pix)
    compare(depth.reshape(-1)[pix], nb.reshape(-1)[pix], corr.reshape(-1)[pix], sc["z_mono"].reshape(-1)[pix], ref)
    # the refinement helps: median inverse-depth error well below the monocular input's
    v = nb >= 0
    zt = sc["z_true"]
    assert np.median(np.abs(1 / depth[v] - 1 / zt[v])) < 0.5 * np.median(np.abs(1 / sc["z_mono"][v] - 1 / zt[v]))


def test_degenerate_pixels_and_determinism():
    sc = synth.guided_scene(seed=70, width=64, height=48, f=50.0, n_nb=2, channels=16)
    z = sc["z_mono"]
    z[3, 5], z[3, 6], z[3, 7], z[3, 8] = 0.0, np.nan, -2.0, np.inf
    a = run_gpu(sc)
    b = run_gpu(sc)
    for x, y in zip(a, b):
        assert np.array_equal(x, y, equal_nan=True)
    depth, nb, corr = a
    assert (nb[3, 5:9] == -1).all() and depth[3, 5] == 0 and np.isnan(depth[3, 6]) and depth[3, 7] == -2
    assert np.isinf(depth[3, 8])
    ref = oracle(sc)
    compare(depth, nb, corr, z, ref)
    # a neighbour turned around sees no segment: every pixel keeps its monocular depth
    sc2 = dict(sc)
    back = dict(sc["cams"][1])
    back["R"] = (np.diag([-1.0, 1.0, -1.0]) @ sc["cams"][0]["R"].astype(np.float64)).astype(np.float32)
    back["t"] = (np.diag([-1.0, 1.0, -1.0]) @ sc["cams"][0]["t"].astype(np.float64)).astype(np.float32)
    sc2["cams"] = [sc["cams"][0], back]
    sc2["feats"] = sc["feats"][:2]
    depth, nb, corr = run_gpu(sc2)
    assert (nb == -1).all() and np.array_equal(depth, z, equal_nan=True)


def test_invalid_arguments():
    sc = synth.guided_scene(seed=71, width=32, height=16, f=30.0, n_nb=2, channels=16)
    feats = torch.from_numpy(sc["feats"].view(np.int16)).cuda()
    cams = gs.cameras_tensor(sc["cams"])
    z = torch.from_numpy(sc["z_mono"]).cuda()
    with pytest.raises(RuntimeError):
        gs.gs_guided_depth(feats, cams, z, n_cand=2)
    with pytest.raises(RuntimeError):
        gs.gs_guided_depth(feats, cams, z, window=0.0)
    with pytest.raises(RuntimeError):
        gs.gs_guided_depth(feats[:, :, :, :12].contiguous(), cams, z)  # 12 channels
    with pytest.raises(RuntimeError):
        gs.gs_guided_depth(feats[:1], cams, z)  # no neighbour
    big = feats.new_zeros((10, 16, 32, 16))
    with pytest.raises(RuntimeError):
        gs.gs_guided_depth(big, cams, z)  # 9 neighbours
    buf = feats.new_zeros(feats.numel() + 8)
    with pytest.raises(RuntimeError):  # feature base not 16-byte aligned
        gs.gs_guided_depth(buf[1:1 + feats.numel()].reshape(feats.shape), cams, z)
