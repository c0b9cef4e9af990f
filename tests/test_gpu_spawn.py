"""GPU direct spawn sampling against the FP64 oracle (Sec. 4.2, Eq. 1-3):
per-pixel maps at 1e-5, the mask bit-exact except where the oracle flags
|u - P_s| within the FP32 margin, the spawned Gaussians at 1e-5."""
import numpy as np
import pytest
import torch

from helpers import assert_close
from oracle import oracle as O
from paper_2506_05558_gb300 import gs, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2506_05558_gb300 import build
    from oracle import build as ob
    build.build()
    ob.build()


def t32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def smooth_image(rng, W, H, k=6):
    """Random image with structure at several scales, values in [0, 1]."""
    im = np.zeros((3, H, W))
    y, x = np.mgrid[0:H, 0:W]
    for _ in range(k):
        fx, fy = rng.uniform(0.01, 0.3, 2)
        ph = rng.uniform(0, 6.3, 3)
        im += np.sin(fx * x[None] + fy * y[None] + ph[:, None, None])
    im += 0.3 * rng.standard_normal((3, H, W))
    im = (im - im.min()) / (im.max() - im.min())
    return im.astype(np.float32)


@pytest.mark.parametrize("W,H,sigma,with_render", [(203, 131, 1.0, True), (96, 64, 2.0, False),
                                                   (1920, 1080, 1.0, True)])
def test_spawn_matches_oracle(W, H, sigma, with_render):
    rng = np.random.default_rng(W)
    im = smooth_image(rng, W, H)
    rd = np.clip(im + 0.05 * rng.standard_normal(im.shape), 0, 1).astype(np.float32) if with_render else None
    depth = rng.uniform(1.0, 20.0, (H, W)).astype(np.float32)
    depth[::17, ::13] = 0.0  # no depth there: never spawns
    R, t = O.retract_pose(np.eye(3), np.zeros(3), [0.1, 0.2, -0.1, 0.05, -0.02, 0.03])
    cam = synth.camera(R.astype(np.float32), t.astype(np.float32), 0.8 * W, W, H)
    seed, frame = 0x1234_5678_9ABC, 17
    cap = W * H
    out = gs.Spawned.alloc(cap, W * H)
    ws = gs.workspace(gs.gs_spawn_workspace_size(W, H))
    gs.gs_spawn_propose(t32(im), None if rd is None else t32(rd), t32(depth), W, H, gs.cameras_tensor([cam]),
                        sigma, seed, frame, out, ws)
    torch.cuda.synchronize()
    assert int(out.status.item()) == gs.GS_OK
    ref = O.spawn(im.astype(np.float64), None if rd is None else rd.astype(np.float64), depth, cam, sigma, seed,
                  frame, margin=1e-5)
    m = ref["maps"]
    for k in ("p_l", "p_pen"):
        assert_close(getattr(out, k).cpu().numpy().reshape(H, W), m[k], 1e-5, what=k)
    # P_s = max(P_L - P~, 0) cancels: its error scale is that of its operands
    ps = out.p_s.cpu().numpy().reshape(H, W)
    scale_l = np.abs(m["p_l"]) + np.sqrt(np.mean(m["p_l"] ** 2))
    assert np.all(np.abs(ps - m["p_s"]) <= 1e-5 * scale_l), np.abs(ps - m["p_s"]).max()
    n = int(out.count.item())
    pix = out.pixel[:n].cpu().numpy()
    assert np.all(np.diff(pix) > 0)  # compacted in pixel order
    amb = set(np.nonzero(m["amb"].reshape(-1))[0].tolist())
    got, want = set(pix.tolist()), set(ref["pixel"].tolist())
    assert (got ^ want) <= amb, len(got ^ want)
    assert len(amb) <= 1e-4 * W * H + 3
    common = np.array(sorted(got & want))
    gi = np.searchsorted(pix, common)
    oi = np.searchsorted(ref["pixel"], common)
    mo = out.g.mean_opa[:n].cpu().numpy()[gi]
    assert_close(mo[:, :3], ref["mean"][oi], 1e-5, what="mean")
    assert np.all(mo[:, 3] == 0)
    assert_close(out.g.scale[:n].cpu().numpy()[gi][:, :3], ref["log_scale"][oi], 1e-5, what="log scale")
    assert np.all(out.g.quat[:n].cpu().numpy()[gi] == np.array([1, 0, 0, 0], np.float32))
    shg = out.g.sh[:n].cpu().numpy()[gi]
    assert_close(shg[:, :3], ref["sh_dc"][oi], 1e-5, what="sh dc")
    assert np.all(shg[:, 3:] == 0)


def test_spawn_capacity_overflow():
    rng = np.random.default_rng(3)
    W, H = 64, 64
    im = smooth_image(rng, W, H)
    depth = np.ones((H, W), np.float32)
    out = gs.Spawned.alloc(4)
    ws = gs.workspace(gs.gs_spawn_workspace_size(W, H))
    cam = synth.camera(np.eye(3), np.zeros(3), 50.0, W, H)
    gs.gs_spawn_propose(t32(im), None, t32(depth), W, H, gs.cameras_tensor([cam]), 1.0, 5, 0, out, ws)
    torch.cuda.synchronize()
    assert int(out.count.item()) > 4 and int(out.status.item()) == gs.GS_ERR_CAPACITY
