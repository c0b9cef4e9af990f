"""The allocation-free spawn proposal (for callers that cannot allocate device
memory, e.g. a host application that owns the allocator) must give exactly
what the workspace-based gs_spawn_propose gives - bit for bit, since both run
the same kernels - call after call and across frame sizes, although its
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


def _check(W, H, seed, call, ws_cache):
    """One call of each entry point on the same frame: identical outputs, bit for bit
    (both run the same kernels; only the scratch memory differs)."""
    cam = gs.cameras_tensor([synth.camera(np.eye(3), np.zeros(3), 0.8 * W, W, H)])
    if (W, H) not in ws_cache:
        ws_cache[(W, H)] = gs.workspace(gs.gs_spawn_workspace_size(W, H))
    im, rd, depth = _frame(seed, W, H)
    ref = gs.Spawned.alloc(W * H, W * H)
    got = gs.Spawned.alloc(W * H, W * H)
    gs.gs_spawn_propose(im, rd, depth, W, H, cam, 1.0, 77, call, ref, ws_cache[(W, H)])
    assert gs.gs_spawn_propose_noalloc(im, rd, depth, W, H, cam, 1.0, 77, call, got) == gs.GS_OK
    torch.cuda.synchronize()
    assert int(got.status.item()) == gs.GS_OK
    n = int(ref.count.item())
    assert n > 100 and int(got.count.item()) == n
    for a, b in ((got.p_l, ref.p_l), (got.p_pen, ref.p_pen), (got.p_s, ref.p_s), (got.pixel[:n], ref.pixel[:n]),
                 (got.g.mean_opa[:n], ref.g.mean_opa[:n]), (got.g.scale[:n], ref.g.scale[:n]),
                 (got.g.quat[:n], ref.g.quat[:n]), (got.g.sh[:n], ref.g.sh[:n])):
        assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
    return im, rd, got


def test_noalloc_matches_workspace_entry_point_call_after_call():
    """Calls in a row share the library's scratch array, which keeps the previous
    call's contents: two frames of one size, then a smaller frame (the words past
    its pixel count still hold the larger frame's data and must not be read),
    then the larger size again."""
    ws = {}
    for call, (W, H, seed) in enumerate(((640, 360, 11), (640, 360, 12), (320, 200, 13), (640, 360, 14))):
        _check(W, H, seed, call, ws)


def test_noalloc_maps_match_the_oracle():
    """The allocation-free call's probability maps against the FP64 oracle's
    (Sec. 4.2, Eq. 1-3), at the spawn tests' 1e-5, on a frame that follows a
    larger one."""
    from helpers import assert_close
    from oracle import build as ob
    from oracle import oracle as O
    ob.build()
    ws = {}
    _check(640, 360, 21, 0, ws)
    W, H = 200, 120
    im, rd, got = _check(W, H, 22, 1, ws)
    ref = O.spawn_maps(im.cpu().numpy().reshape(3, H, W).astype(np.float64),
                       rd.cpu().numpy().reshape(3, H, W).astype(np.float64), 1.0, 77, 1)
    assert_close(got.p_l.cpu().numpy().reshape(H, W), ref["p_l"], 1e-5, what="P_L")
    assert_close(got.p_pen.cpu().numpy().reshape(H, W), ref["p_pen"], 1e-5, what="P~")
    assert_close(got.p_s.cpu().numpy().reshape(H, W), ref["p_s"], 1e-5, what="P_s")


def test_noalloc_rejects_frames_over_its_limit():
    W, H = 2048, 1100  # 2,252,800 pixels > 2,097,152
    cam = gs.cameras_tensor([synth.camera(np.eye(3), np.zeros(3), 500.0, W, H)])
    im = torch.zeros((3 * W * H,), device="cuda")
    depth = torch.ones((W * H,), device="cuda")
    out = gs.Spawned.alloc(16)
    assert gs.gs_spawn_propose_noalloc(im, None, depth, W, H, cam, 1.0, 1, 0, out) == gs.GS_ERR_INVALID_ARG
