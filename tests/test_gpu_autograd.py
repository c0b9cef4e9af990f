"""torch.autograd binding of the rasteriser (hand-written adjoint behind
torch.autograd.Function, pose on the SE(3) tangent, Sec. 4.3): the pose
composition and the tangent-gradient map against the FP64 oracle, the
Function's gradients against the raw C-ABI calls (identical kernels, so
bit-identical) and, through compare_views, against the oracle; config-1 loss
L1 + 0.2 (1 - SSIM) differentiated by PyTorch into dL/dC."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import oracle as O
from paper_2506_05558_gb300 import gs, synth
from paper_2506_05558_gb300.autograd import rasterize
from paper_2506_05558_gb300.raster import Rasterizer
from test_gpu_parity import compare_views

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2506_05558_gb300 import build
    build.build()


def params(sc):
    g = gs.Gaussians.from_scene(sc)
    return [t.clone().requires_grad_(True) for t in (g.mean_opa, g.scale, g.quat, g.sh)]


def test_pose_apply_and_tangent_grad_match_oracle():
    rng = np.random.default_rng(4)
    _, cams, _ = synth.multiview_scene(seed=5, n=10, n_views=6, sizes=[(64, 48)] * 6)
    xi = np.concatenate([rng.normal(0, 0.5, (6, 3)), rng.normal(0, 0.4, (6, 3))], 1)
    xi[0] = 0.0
    xi[1, 3:] = [2e-4, -1e-4, 3e-4]  # series branch
    xi[2, 3:] = 0.0                  # pure translation
    cams_t = gs.cameras_tensor(cams)
    xi_t = torch.tensor(xi, dtype=torch.float32, device="cuda")
    out = torch.empty_like(cams_t)
    gs.gs_pose_apply(cams_t, xi_t, 6, out)
    g = rng.standard_normal((6, 6))
    g_t = torch.tensor(g, dtype=torch.float32, device="cuda")
    d = torch.empty_like(g_t)
    gs.gs_pose_tangent_grad(xi_t, g_t, 6, d)
    got = gs.cameras_from_tensor(out)
    xi32 = xi.astype(np.float32).astype(np.float64)
    for i, c in enumerate(cams):
        R0 = np.asarray(c["R"], np.float32).astype(np.float64)
        t0 = np.asarray(c["t"], np.float32).astype(np.float64)
        R, t = O.retract_pose(R0, t0, xi32[i])
        np.testing.assert_allclose(got[i]["R"], R, atol=2e-7)
        np.testing.assert_allclose(got[i]["t"], t, atol=2e-6 * max(1.0, np.abs(t).max()))
        assert (got[i]["width"], got[i]["height"], got[i]["fx"]) == (c["width"], c["height"], np.float32(c["fx"]))
        ref = O.pose_tangent_grad(xi32[i], g.astype(np.float32)[i])
        np.testing.assert_allclose(d.cpu().numpy()[i], ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max())


def test_autograd_equals_raw_calls_and_oracle():
    """Config 0 scene, a nonzero pose tangent, loss sum(w * C)."""
    sc, cam, rng = synth.tiny_scene()
    xi = torch.tensor([[0.01, -0.02, 0.015, 0.01, 0.02, -0.01]], device="cuda")
    xi_p = xi.clone().requires_grad_(True)
    cams_ref = gs.cameras_tensor([cam])
    cfg = gs.config(sh_degree=0, bg=(0.2, 0.1, 0.0))
    mo, sca, qu, sh = params(sc)
    w = rng.standard_normal((3, 64, 64))
    w_t = torch.tensor(w.reshape(-1), dtype=torch.float32, device="cuda")
    color, t_final = rasterize(mo, sca, qu, sh, xi_p, cams_ref, [(64, 64)], cfg)
    (color * w_t).sum().backward()
    assert t_final.shape == (64 * 64,) and not t_final.requires_grad

    # raw C-ABI sequence on the same inputs
    cams = torch.empty_like(cams_ref)
    gs.gs_pose_apply(cams_ref, xi, 1, cams)
    g = gs.Gaussians.from_scene(sc)
    r = Rasterizer(sc.n, [(64, 64)], 1 << 16, cfg)
    r.fit_capacity(g, cams)
    r.forward(g, cams)
    assert torch.equal(r.img.color, color.detach())
    r.backward(g, cams, w_t)
    d_xi = torch.empty_like(r.dpose)
    gs.gs_pose_tangent_grad(xi, r.dpose, 1, d_xi)
    torch.cuda.synchronize()
    for got, want in ((mo.grad, r.grads.mean_opa), (sca.grad, r.grads.scale), (qu.grad, r.grads.quat),
                      (sh.grad, r.grads.sh), (xi_p.grad, d_xi)):
        assert torch.equal(got, want)

    # the same kernels against the oracle at the composed camera
    cam1 = gs.cameras_from_tensor(cams)[0]
    cam1 = dict(cam1, R=cam1["R"].astype(np.float64), t=cam1["t"].astype(np.float64))
    compare_views(sc, [cam1], 0, bg=(0.2, 0.1, 0.0), dLs=[w])


def ssim(img, ref, window=11, sigma=1.5):
    """Mean SSIM over a [3][H][W] image pair with an 11x11 Gaussian window
    (sigma 1.5), zero padding, C1 = 0.01^2, C2 = 0.03^2."""
    x = torch.arange(window, dtype=img.dtype, device=img.device) - window // 2
    k1 = torch.exp(-x * x / (2 * sigma * sigma))
    k1 = k1 / k1.sum()
    k = (k1[:, None] * k1[None, :]).expand(3, 1, window, window).contiguous()
    f = lambda t: F.conv2d(t[None], k, padding=window // 2, groups=3)[0]
    mu_x, mu_y = f(img), f(ref)
    sxx = f(img * img) - mu_x * mu_x
    syy = f(ref * ref) - mu_y * mu_y
    sxy = f(img * ref) - mu_x * mu_y
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    m = ((2 * mu_x * mu_y + c1) * (2 * sxy + c2)) / ((mu_x * mu_x + mu_y * mu_y + c1) * (sxx + syy + c2))
    return m.mean()


def test_config1_l1_dssim_loss_gradients():
    """1280x720, 200k Gaussians, SH3, L = L1 + 0.2 (1 - SSIM): PyTorch turns
    the loss into dL/dC, the Function's adjoint matches the oracle fed the
    same dL/dC, and a few torch.optim.Adam steps through the Function lower
    the loss."""
    sc, cam, rng = synth.view_720p_scene()
    W, H = 1280, 720
    cams_ref = gs.cameras_tensor([cam])
    cfg = gs.config(sh_degree=3)
    # target: render with means jittered by N(0, 0.01) plus N(0, 0.01) pixel noise
    jit = synth.Scene(sc.mean_opa.copy(), sc.scale, sc.quat, sc.sh, sc.sh_degree)
    jit.mean_opa[:, :3] += rng.normal(0, 0.01, (sc.n, 3))
    zero = torch.zeros((1, 6), device="cuda")
    with torch.no_grad():
        tgt, _ = rasterize(*params(jit), zero, cams_ref, [(W, H)], cfg)
    tgt = (tgt.view(3, H, W) + torch.tensor(rng.normal(0, 0.01, (3, H, W)), dtype=torch.float32,
                                             device="cuda")).contiguous()

    ps = params(sc)
    xi = zero.clone().requires_grad_(True)
    color, _ = rasterize(*ps, xi, cams_ref, [(W, H)], cfg)
    color.retain_grad()
    img = color.view(3, H, W)
    loss = (img - tgt).abs().mean() + 0.2 * (1.0 - ssim(img, tgt))
    loss.backward()
    dLdC = color.grad.detach().double().cpu().numpy().reshape(3, H, W)
    assert np.abs(dLdC).max() > 0
    r, _ = compare_views(sc, [cam], 3, dLs=[dLdC])
    for got, want in ((ps[0].grad, r.grads.mean_opa), (ps[1].grad, r.grads.scale), (ps[2].grad, r.grads.quat),
                      (ps[3].grad, r.grads.sh)):
        assert torch.equal(got, want)

    opt = torch.optim.Adam([{"params": [ps[0]], "lr": 1e-4}, {"params": [ps[1], ps[2]], "lr": 1e-3},
                            {"params": [ps[3]], "lr": 2.5e-3}, {"params": [xi], "lr": 1e-4}])
    losses = []
    for _ in range(8):
        opt.zero_grad()
        color, _ = rasterize(*ps, xi, cams_ref, [(W, H)], cfg)
        img = color.view(3, H, W)
        loss = (img - tgt).abs().mean() + 0.2 * (1.0 - ssim(img, tgt))
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    assert losses[-1] < losses[0], losses
