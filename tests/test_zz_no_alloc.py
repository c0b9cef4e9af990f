"""The allocation-free spawn proposal (for callers that cannot allocate device
memory, e.g. a host application that owns the allocator) must give exactly
what the workspace-based gs_spawn_propose gives, call after call, although its
scratch is one array inside the library shared by all calls.

Collected last on purpose: it runs after every other test in a full run, and
must also pass alone in a fresh process."""
import numpy as np
import pytest
import torch

from paper_2506_05558_gb300 import gs, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2506_05558_gb300 import build
    build.build()


def t32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _frame(seed, W, H):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:H, 0:W]
    im = np.stack([0.5 + 0.4 * np.sin(0.07 * (c + 1) * x + 0.05 * y + seed) for c in range(3)])
    im = np.clip(im + 0.1 * rng.standard_normal(im.shape), 0, 1)
    rd = np.clip(im + 0.05 * rng.standard_normal(im.shape), 0, 1)
    depth = rng.uniform(1, 10, (H, W))
    return t32(im), t32(rd), t32(depth)


def test_noalloc_matches_workspace_entry_point_twice():
    W, H = 640, 360
    cam = gs.cameras_tensor([synth.camera(np.eye(3), np.zeros(3), 500.0, W, H)])
    ws = gs.workspace(gs.gs_spawn_workspace_size(W, H))
    for call, seed in enumerate((11, 12)):  # two calls in a row: the shared scratch holds the previous call's data
        im, rd, depth = _frame(seed, W, H)
        ref = gs.Spawned.alloc(W * H, W * H)
        got = gs.Spawned.alloc(W * H, W * H)
        gs.gs_spawn_propose(im, rd, depth, W, H, cam, 1.0, 77, call, ref, ws)
        assert gs.gs_spawn_propose_noalloc(im, rd, depth, W, H, cam, 1.0, 77, call, got) == gs.GS_OK
        torch.cuda.synchronize()
        assert int(got.status.item()) == gs.GS_OK
        n = int(ref.count.item())
        assert n > 1000 and int(got.count.item()) == n
        for a, b in ((got.p_l, ref.p_l), (got.p_pen, ref.p_pen), (got.p_s, ref.p_s), (got.pixel[:n], ref.pixel[:n]),
                     (got.g.mean_opa[:n], ref.g.mean_opa[:n]), (got.g.scale[:n], ref.g.scale[:n]),
                     (got.g.quat[:n], ref.g.quat[:n]), (got.g.sh[:n], ref.g.sh[:n])):
            a, b = a.cpu().numpy(), b.cpu().numpy()
            assert np.allclose(a, b, rtol=1e-5, atol=1e-7)


def test_noalloc_rejects_frames_over_its_limit():
    W, H = 2048, 1100  # 2,252,800 pixels > 2,097,152
    cam = gs.cameras_tensor([synth.camera(np.eye(3), np.zeros(3), 500.0, W, H)])
    im = torch.zeros((3 * W * H,), device="cuda")
    depth = torch.ones((W * H,), device="cuda")
    out = gs.Spawned.alloc(16)
    assert gs.gs_spawn_propose_noalloc(im, None, depth, W, H, cam, 1.0, 1, 0, out) == gs.GS_ERR_INVALID_ARG
