"""Learned spawn proposal on the GPU against the FP64 oracle (oracle/mlp.py),
for both tensor-core paths (0: mma.sync tiles, 1: tcgen05.mma with the
accumulator in tensor memory): the bf16 GEMM against NumPy, the forward pass
at 1e-3, the training step's loss at 1e-3 and weight gradients at 1e-2, one
Adam step."""
import numpy as np
import pytest
import torch

from helpers import assert_close
from oracle import mlp as OM
from paper_2506_05558_gb300 import gs

pytestmark = pytest.mark.gpu
PATHS = [0, 1]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2506_05558_gb300 import build
    build.build()


def bf16_pair(rng, M, N, K):
    A = torch.tensor(rng.standard_normal((M, K)), dtype=torch.float32).to(torch.bfloat16)
    B = torch.tensor(rng.standard_normal((N, K)), dtype=torch.float32).to(torch.bfloat16)
    ref = A.double() @ B.double().T
    return A.cuda(), B.cuda(), ref.numpy()


@pytest.mark.parametrize("PATH", PATHS)
@pytest.mark.parametrize("M,N,K", [(300, 128, 208), (100, 16, 128), (128, 208, 4096), (1000, 128, 16), (7, 32, 32)])
def test_gemm_matches_numpy(M, N, K, PATH):
    rng = np.random.default_rng(M + N + K)
    A, B, ref = bf16_pair(rng, M, N, K)
    C = torch.full((M, N), float("nan"), device="cuda")
    gs.gs_mlp_gemm_bf16(A, B, C, PATH)
    torch.cuda.synchronize()
    assert_close(C.cpu().numpy(), ref, 1e-5, what=f"gemm path {PATH}")
    if PATH == 1:
        assert gs.gs_mlp_tc_error() == 0


def mlp_case(seed, W=96, H=64):
    rng = np.random.default_rng(seed)
    layers = OM.init_params(rng)
    image = rng.random((3, H, W))
    n = (W // 8) * (H // 8)
    targets = np.stack([rng.random(n), rng.uniform(2, 10, n), rng.normal(-4, 0.5, n),
                        (rng.random(n) < 0.6).astype(float)], 1)
    return rng, layers, image, targets


def run_train(layers, image, targets, path, with_adam=False, lr=1e-3):
    H, W = image.shape[1:]
    n = gs.gs_mlp_patches(W, H)
    p = gs.MlpParams.from_numpy(layers)
    m = gs.MlpParams.zeros() if with_adam else None
    v = gs.MlpParams.zeros() if with_adam else None
    ws = gs.workspace(gs.gs_mlp_workspace_size(n))
    loss = torch.zeros(1, device="cuda")
    out = torch.zeros((n, 3), device="cuda")
    grads = torch.zeros(gs.gs_mlp_param_count(), device="cuda")
    img = torch.tensor(image, dtype=torch.float32, device="cuda")
    tg = torch.tensor(targets, dtype=torch.float32, device="cuda")
    cfg = gs.mlp_config(tensor_path=path, lr=lr)
    gs.gs_mlp_train_step(p, m, v, img, W, H, tg, cfg, 1, loss, ws, out=out, grads=grads)
    torch.cuda.synchronize()
    return p, loss.item(), out.cpu().numpy(), grads.cpu().numpy()


def oracle_train(layers, image, targets):
    X = OM.patch_features(image)
    Y, cache = OM.forward(layers, X)
    L, dY = OM.loss(Y, targets[:, 0], targets[:, 1], targets[:, 2], targets[:, 3])
    grads = OM.backward(layers, cache, dY)
    flat = np.concatenate([np.concatenate([dW.reshape(-1), db]) for dW, db in grads])
    return Y, L, grads, flat


@pytest.mark.parametrize("PATH", PATHS)
def test_forward_matches_oracle(PATH):
    rng, layers, image, targets = mlp_case(1)
    H, W = image.shape[1:]
    n = gs.gs_mlp_patches(W, H)
    out = torch.zeros((n, 3), device="cuda")
    ws = gs.workspace(gs.gs_mlp_workspace_size(n))
    gs.gs_mlp_forward(gs.MlpParams.from_numpy(layers), torch.tensor(image, dtype=torch.float32, device="cuda"), W, H,
                      out, gs.mlp_config(tensor_path=PATH), ws)
    torch.cuda.synchronize()
    Y, _, _, _ = oracle_train(layers, image, targets)
    assert_close(out.cpu().numpy(), Y, 1e-3, what="mlp forward")


@pytest.mark.parametrize("PATH", PATHS)
def test_forward_full_frame_matches_oracle(PATH):
    """A 1920x1080 frame: 32,400 patches = 253 tiles of 128 with a ragged last
    tile, more tiles than SMs (the tcgen05 path runs the fused persistent
    kernel, so CTAs take several tiles)."""
    rng, layers, image, targets = mlp_case(5, W=1920, H=1080)
    n = gs.gs_mlp_patches(1920, 1080)
    assert n == 32400
    out = torch.zeros((n, 3), device="cuda")
    ws = gs.workspace(gs.gs_mlp_workspace_size(n))
    gs.gs_mlp_forward(gs.MlpParams.from_numpy(layers), torch.tensor(image, dtype=torch.float32, device="cuda"), 1920,
                      1080, out, gs.mlp_config(tensor_path=PATH), ws)
    torch.cuda.synchronize()
    assert gs.gs_mlp_tc_error() == 0
    Y, _ = OM.forward(layers, OM.patch_features(image))
    assert_close(out.cpu().numpy(), Y, 1e-3, what="mlp forward 1080p")


@pytest.mark.parametrize("PATH", PATHS)
def test_train_step_loss_and_gradients_match_oracle(PATH):
    rng, layers, image, targets = mlp_case(2)
    _, loss, out, grads = run_train(layers, image, targets, PATH)
    Y, L, g, flat = oracle_train(layers, image, targets)
    assert_close(out, Y, 1e-3, what="outputs")
    assert abs(loss - L) <= 1e-3 * abs(L)
    off = 0
    for l, (dW, db) in enumerate(g):
        for name, ref in ((f"dW{l + 1}", dW), (f"db{l + 1}", db)):
            got = grads[off:off + ref.size].reshape(ref.shape)
            assert_close(got, ref, 1e-2, what=name)
            off += ref.size


@pytest.mark.parametrize("PATH", PATHS)
def test_adam_step_matches_oracle(PATH):
    rng, layers, image, targets = mlp_case(3)
    p, _, _, grads = run_train(layers, image, targets, PATH, with_adam=True, lr=1e-3)
    # Adam's first step from zero moments moves each parameter by lr * sign(g)
    got = p.numpy()
    off = 0
    for (W, b), (W2, b2) in zip(layers, got):
        for ref, new in ((W, W2), (b, b2)):
            g = grads[off:off + ref.size].reshape(ref.shape)
            off += ref.size
            want = ref - 1e-3 * g / (np.abs(g) + 1e-8)
            assert_close(new, want, 1e-5, what="adam")


def test_targets_from_kept_spawns_match_oracle():
    """The keep decision (sigmoid of the optimised logit above the threshold),
    camera depth and log-scale change of every spawn, summed per patch, against
    the FP64 oracle. Logits stay 1e-3 away from the threshold's logit, so FP32
    takes the same keep decisions."""
    from paper_2506_05558_gb300 import synth
    from oracle import oracle as O
    rng = np.random.default_rng(5)
    W, H = 120, 64
    n = 2000
    thr = 0.05
    pixel = np.sort(rng.choice(W * H, n, replace=False)).astype(np.int32)
    mean_opa = np.zeros((n, 4), np.float32)
    mean_opa[:, :3] = rng.uniform(-3, 3, (n, 3))
    mean_opa[:, 2] += 8.0
    logit = rng.normal(-3.0, 1.5, n)
    l_thr = np.log(thr / (1 - thr))
    logit = np.where(np.abs(logit - l_thr) < 1e-3, l_thr + 2e-3, logit)
    mean_opa[:, 3] = logit
    scale = np.zeros((n, 4), np.float32)
    scale[:, :3] = rng.normal(-4, 1, (n, 3))
    scale0 = np.repeat(rng.normal(-4, 0.5, (n, 1)), 4, 1).astype(np.float32)
    R, t = O.retract_pose(np.eye(3), np.zeros(3), [0.2, -0.1, 0.3, 0.05, 0.1, -0.08])
    cam = synth.camera(R.astype(np.float32), t.astype(np.float32), 100.0, W, H)
    tg = torch.zeros(((W // 8) * (H // 8), 4), device="cuda")
    ws = gs.workspace(gs.gs_mlp_targets_workspace_size(W, H))
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    gs.gs_mlp_targets(c(pixel), c(mean_opa), c(scale), c(scale0), gs.cameras_tensor([cam]), thr, n, W, H, tg, ws)
    torch.cuda.synchronize()
    ref, opa = OM.targets_from_rows(pixel, mean_opa.astype(np.float64), scale.astype(np.float64),
                                    scale0.astype(np.float64), cam, thr, W, H)
    assert 0.2 < np.mean(opa > thr) < 0.8
    assert_close(tg.cpu().numpy(), ref, 1e-5, what="targets")


@pytest.mark.parametrize("with_depth,with_render", [(False, False), (True, False), (True, True)])
def test_learned_spawn_matches_oracle(with_depth, with_render):
    """Spawns from the network's outputs placed by P_s; with a depth map (holes:
    zero, negative, NaN) its values replace the predicted depth where valid;
    with a render the penalty of Eq. 2 enters P_s."""
    from paper_2506_05558_gb300 import synth
    from oracle import oracle as O
    rng = np.random.default_rng(6)
    W, H = 160, 96
    n_p = (W // 8) * (H // 8)
    out = np.stack([rng.normal(-2, 1.5, n_p), rng.uniform(-1, 15, n_p), rng.normal(-4, 0.5, n_p)], 1).astype(np.float32)
    image = rng.random((3, H, W)).astype(np.float32)
    render = None
    if with_render:
        render = np.clip(image + rng.normal(0, 0.05, image.shape), 0, 1).astype(np.float32)
        render[:, :, :40] = image[:, :, :40]  # a fully explained strip: P_s = 0 there
    depth = None
    if with_depth:
        depth = rng.uniform(1, 20, (H, W)).astype(np.float32)
        holes = rng.random((H, W))
        depth[holes < 0.2] = 0.0
        depth[(holes >= 0.2) & (holes < 0.25)] = -3.0
        depth[(holes >= 0.25) & (holes < 0.3)] = np.nan
    R, t = O.retract_pose(np.eye(3), np.zeros(3), [0.2, -0.1, 0.3, 0.1, 0.05, -0.2])
    cam = synth.camera(R.astype(np.float32), t.astype(np.float32), 120.0, W, H)
    sp = gs.Spawned.alloc(W * H)
    ws = gs.workspace(gs.gs_spawn_workspace_size(W, H))
    dev = lambda a: None if a is None else torch.from_numpy(a).cuda()
    gs.gs_spawn_learned(dev(image), dev(out), W, H, gs.cameras_tensor([cam]), 99, 7, sp, ws, depth=dev(depth),
                        render=dev(render))
    torch.cuda.synchronize()
    ref = OM.spawn_learned(image, out, cam, 99, 7, depth=depth, render=render)
    k = int(sp.count.item())
    assert k > 100
    pix = sp.pixel[:k].cpu().numpy()
    amb = set(np.nonzero(ref["amb"])[0].tolist())
    assert len(amb) <= 0.01 * W * H
    assert (set(pix.tolist()) ^ set(ref["pixel"].tolist())) <= amb
    common = np.array(sorted(set(pix.tolist()) & set(ref["pixel"].tolist())))
    gi, oi = np.searchsorted(pix, common), np.searchsorted(ref["pixel"], common)
    assert_close(sp.g.mean_opa[:k].cpu().numpy()[gi][:, :3], ref["mean"][oi], 1e-5, what="mean")
    assert_close(sp.g.scale[:k].cpu().numpy()[gi][:, :3], ref["log_scale"][oi], 1e-6, what="log scale")
    assert_close(sp.g.sh[:k].cpu().numpy()[gi][:, :3], ref["sh_dc"][oi], 1e-5, what="sh dc")
