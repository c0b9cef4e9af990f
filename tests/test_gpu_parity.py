"""GPU path (libgs, sm_103a) against the FP64 oracle, element by element, on
the same seeded inputs. Image tolerance 1e-4, gradient tolerance 1e-3
(relative, per-tensor semantics of helpers.assert_close); tile lists, sort
orders and integer outputs bit-exact. Decisions the oracle flags as within
the FP32 margin are excluded and counted."""
import numpy as np
import pytest
import torch

from helpers import assert_close, assert_within, tile_pixel_mask, workload_gradients
from oracle import oracle as O
from paper_2506_05558_gb300 import gs, synth
from paper_2506_05558_gb300.raster import Rasterizer

pytestmark = pytest.mark.gpu

IMG_RTOL = 1e-4
GRAD_RTOL = 1e-3
MARGINS = dict(margin_alpha=1e-4, margin_T=1e-4, margin_rect_px=2e-3, margin_geo=1e-5)
# confidence factor on the root-sum-square FP32 rounding bound of the adjoint
FP32_LAMBDA = 1.0
# with the workload's loss gradient, the pose bound may use at most this share of |ref| + rms
POSE_SHARE = 1e-2


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2506_05558_gb300 import build
    from oracle import build as ob
    build.build()
    ob.build()
    assert torch.cuda.is_available()


def t32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def projected_from_items(items_per_view):
    """Concatenate per-view synthetic projected items into device buffers."""
    cat = lambda k: np.concatenate([it[k] for it in items_per_view], 0)
    p = gs.Projected(t32(cat("mean2d")), t32(cat("conic_opa")), t32(cat("rgb_depth")),
                     torch.from_numpy(cat("rect").astype(np.int16)).cuda(),
                     torch.from_numpy(cat("n_tiles").astype(np.int32)).cuda())
    return p


def oracle_proj(it):
    return dict(mean2d=it["mean2d"].astype(np.float64), conic=it["conic_opa"][:, :3].astype(np.float64),
                opacity=it["conic_opa"][:, 3].astype(np.float64), rgb=it["rgb_depth"][:, :3].astype(np.float64),
                depth_key=it["rgb_depth"][:, 3].astype(np.float32), rect=it["rect"],
                depth=it["rgb_depth"][:, 3].astype(np.float64))


def sort_items(items_per_view, sizes, n, capacity=None):
    f = gs.frame(sizes)
    p = projected_from_items(items_per_view)
    total = int(sum(int(it["n_tiles"].sum()) for it in items_per_view))
    cap = total if capacity is None else capacity
    pairs = gs.Pairs.alloc(n * len(sizes), int(f.tile_base[len(sizes)]), cap)
    ws = gs.workspace(gs.gs_sort_workspace_size(n, f, cap))
    gs.gs_sort(p, n, f, pairs, ws)
    torch.cuda.synchronize()
    return f, p, pairs, total


# ---------------------------------------------------------------------------
# Sort: bit-exact tile lists
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("depth_levels", [None, 3])
def test_sort_matches_oracle_lists(depth_levels):
    rng = np.random.default_rng(7)
    sizes = [(200, 120), (77, 50), (160, 160)]
    n = 3000
    items = [synth.projected_items(rng, n, (w + 15) // 16, (h + 15) // 16, 16, max_rect=5, depth_levels=depth_levels)
             for w, h in sizes]
    f, p, pairs, total = sort_items(items, sizes, n)
    assert int(pairs.count.item()) == total and int(pairs.status.item()) == gs.GS_OK
    src = pairs.src.cpu().numpy().view(np.uint32)[:total].astype(np.int64)
    emit = pairs.emit.cpu().numpy().view(np.uint32)[:total].astype(np.int64)
    rng_ = pairs.range.cpu().numpy().view(np.uint32).astype(np.int64)
    offset = pairs.offset.cpu().numpy().view(np.uint32).astype(np.int64)
    for v, ((w, h), it) in enumerate(zip(sizes, items)):
        tx, ty = (w + 15) // 16, (h + 15) // 16
        start, ids = O.tile_lists(it["rect"], it["rgb_depth"][:, 3], tx, ty)
        for t in range(tx * ty):
            gt = int(f.tile_base[v]) + t
            got = src[rng_[2 * gt]:rng_[2 * gt + 1]]
            want = ids[start[t]:start[t + 1]] + v * n
            assert np.array_equal(got, want), (v, t)
    # emission slots: a permutation of [0, total), each inside its item's block
    assert np.array_equal(np.sort(emit), np.arange(total))
    nt = np.concatenate([it["n_tiles"] for it in items])
    assert np.all(emit >= offset[src]) and np.all(emit < offset[src] + nt[src])


def test_sort_capacity_overflow_reports_status():
    rng = np.random.default_rng(8)
    sizes = [(128, 128)]
    n = 2000
    items = [synth.projected_items(rng, n, 8, 8, 16, max_rect=4)]
    total = int(items[0]["n_tiles"].sum())
    f, p, pairs, _ = sort_items(items, sizes, n, capacity=total // 3)
    assert int(pairs.count.item()) == total
    assert int(pairs.status.item()) == gs.GS_ERR_CAPACITY


def test_sort_empty_and_all_culled():
    sizes = [(64, 64)]
    for n in (0, 500):
        it = dict(mean2d=np.zeros((n, 2), np.float32), conic_opa=np.ones((n, 4), np.float32),
                  rgb_depth=np.ones((n, 4), np.float32), rect=np.zeros((n, 4), np.int32),
                  n_tiles=np.zeros(n, np.int32))
        f, p, pairs, total = sort_items([it], sizes, n, capacity=16)
        assert int(pairs.count.item()) == 0 and int(pairs.status.item()) == gs.GS_OK
        assert int(pairs.range.abs().sum().item()) == 0


# ---------------------------------------------------------------------------
# Compositing forward / adjoint on synthetic projected splats
# ---------------------------------------------------------------------------

def _render_items(sizes, n, seed, max_rect=4, bg=(0.0, 0.0, 0.0)):
    rng = np.random.default_rng(seed)
    items = [synth.projected_items(rng, n, (w + 15) // 16, (h + 15) // 16, 16, max_rect=max_rect) for w, h in sizes]
    f, p, pairs, total = sort_items(items, sizes, n)
    cfg = gs.config(bg=bg)
    img = gs.Image.alloc(int(f.pix_base[len(sizes)]))
    gs.gs_render_fwd(p, pairs, f, cfg, img)
    torch.cuda.synchronize()
    return rng, items, f, p, pairs, cfg, img


@pytest.mark.parametrize("bg", [(0.0, 0.0, 0.0), (0.3, 0.6, 0.1)])
def test_render_fwd_matches_oracle(bg):
    sizes = [(150, 100), (64, 48)]
    rng, items, f, p, pairs, cfg, img = _render_items(sizes, 4000, 11, bg=bg)
    ocfg = O.Config(bg=bg, **MARGINS)
    n_amb = 0
    for v, ((w, h), it) in enumerate(zip(sizes, items)):
        cam = synth.camera(np.eye(3), np.zeros(3), 100.0, w, h)
        start, ids = O.tile_lists(it["rect"], it["rgb_depth"][:, 3], (w + 15) // 16, (h + 15) // 16)
        ref = O.render_fwd(oracle_proj(it), start, ids, cam, ocfg)
        b = int(f.pix_base[v])
        color = img.color[3 * b:3 * (b + w * h)].view(3, h, w).cpu().numpy()
        T = img.t_final[b:b + w * h].view(h, w).cpu().numpy()
        nc = img.n_contrib[b:b + w * h].view(h, w).cpu().numpy()
        ok = ref["amb"] == 0
        n_amb += int((~ok).sum())
        assert_close(color, ref["color"], IMG_RTOL, np.broadcast_to(ok, color.shape), "color")
        assert_close(T, ref["t_final"], IMG_RTOL, ok, "t_final")
        assert np.array_equal(nc[ok], ref["n_contrib"][ok])
    assert n_amb <= 1e-3 * sum(w * h for w, h in sizes) + 2


def test_render_bwd_2d_adjoint_matches_oracle():
    """d_proj (dL/d(u, v, conic, opacity, rgb) per item) against the oracle's
    compositing adjoint on the same projected splats and lists."""
    sizes = [(120, 90)]
    n = 2500
    rng, items, f, p, pairs, cfg, img = _render_items(sizes, n, 12, bg=(0.1, 0.2, 0.3))
    w, h = sizes[0]
    dL = rng.standard_normal((3, h, w)).astype(np.float32)
    dummy = gs.Gaussians.zeros(n)
    dummy.quat[:, 0] = 1.0
    cams = gs.cameras_tensor([synth.camera(np.eye(3), np.zeros(3), 100.0, w, h)])
    grads = gs.Grads.alloc(n)
    dpose = torch.zeros((1, 6), device="cuda")
    ws = gs.workspace(gs.gs_backward_workspace_size(n, f, pairs.capacity))
    d_proj = torch.zeros((n, 9), device="cuda")
    gs.gs_render_bwd(dummy, cams, p, pairs, f, cfg, img, t32(dL.reshape(-1)), grads, dpose, ws, d_proj)
    torch.cuda.synchronize()
    it = items[0]
    ocfg = O.Config(bg=(0.1, 0.2, 0.3), **MARGINS)
    cam = synth.camera(np.eye(3), np.zeros(3), 100.0, w, h)
    start, ids = O.tile_lists(it["rect"], it["rgb_depth"][:, 3], (w + 15) // 16, (h + 15) // 16)
    oproj = oracle_proj(it)
    oproj.update(amb=np.zeros(n, np.uint8), depth=it["rgb_depth"][:, 3].astype(np.float64))
    ref = O.render_bwd(oproj, start, ids, cam, ocfg, dL.astype(np.float64))
    bb = O.render_bwd_bounds(oproj, start, ids, cam, ocfg, dL.astype(np.float64))
    got = d_proj.cpu().numpy()
    vis = it["n_tiles"] > 0
    for c, name in enumerate(["du", "dv", "da", "db", "dc", "dopa", "dr", "dg", "db_"]):
        assert_within(got[:, c], ref[:, c], GRAD_RTOL, bb["flip"][:, c] + FP32_LAMBDA * bb["fp32"][:, c], vis, name)


def test_render_bwd_deterministic():
    sizes = [(96, 96)]
    n = 2000
    rng, items, f, p, pairs, cfg, img = _render_items(sizes, n, 13)
    dL = t32(rng.standard_normal(3 * 96 * 96))
    dummy = gs.Gaussians.zeros(n)
    dummy.quat[:, 0] = 1.0
    cams = gs.cameras_tensor([synth.camera(np.eye(3), np.zeros(3), 100.0, 96, 96)])
    ws = gs.workspace(gs.gs_backward_workspace_size(n, f, pairs.capacity))
    outs = []
    for _ in range(2):
        grads = gs.Grads.alloc(n)
        d_proj = torch.zeros((n, 9), device="cuda")
        gs.gs_render_bwd(dummy, cams, p, pairs, f, cfg, img, dL, grads, torch.zeros((1, 6), device="cuda"), ws,
                         d_proj)
        torch.cuda.synchronize()
        outs.append(d_proj.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


# ---------------------------------------------------------------------------
# End to end: project -> sort -> render -> adjoint with pose gradients
# ---------------------------------------------------------------------------

def run_views(sc, cams, sh_degree, dLs=None, seed=0, pose_through_sh=0, bg=(0.0, 0.0, 0.0), filter3d=None,
              **launch):
    sizes = [(c["width"], c["height"]) for c in cams]
    cfg = gs.config(sh_degree=sh_degree, pose_grad_through_sh=pose_through_sh, bg=bg, **launch)
    g = gs.Gaussians.from_scene(sc)
    if filter3d is not None:
        g.filter3d = t32(filter3d)
    camt = gs.cameras_tensor(cams)
    r = Rasterizer(sc.n, sizes, capacity=1024, cfg=cfg)
    r.fit_capacity(g, camt)
    r.forward(g, camt)
    rng = np.random.default_rng(seed)
    if dLs is None:
        dLs = [rng.standard_normal((3, h, w)) for w, h in sizes]
    flat = t32(np.concatenate([d.reshape(-1) for d in dLs]))
    d_proj = torch.zeros((sc.n * len(cams), 9), device="cuda")
    r.backward(g, camt, flat, d_proj)
    torch.cuda.synchronize()
    assert r.status() == gs.GS_OK
    return r, dLs, d_proj.cpu().numpy()


def last_contributor_tied(view, w, h, tile):
    """Pixels whose last contributor (n_contrib) sits next to a list entry with
    an fp32 depth key within 2 ulps: the FP32 path may order that pair either
    way, which moves n_contrib by one without changing the image."""
    tx = (w + tile - 1) // tile
    ys, xs = np.mgrid[0:h, 0:w]
    t = (ys // tile) * tx + xs // tile
    start, ids = view["start"], view["ids"]
    keys = view["proj"]["depth_key"].view(np.uint32).astype(np.int64)
    nc = view["n_contrib"].astype(np.int64)
    k = start[t] + nc - 1  # list position of the last contributor
    has = nc > 0
    kk = np.where(has, k, 0)
    key = keys[ids[kk]] if ids.size else np.zeros_like(kk)
    tied = np.zeros((h, w), bool)
    for dk in (-1, 1):
        nb = kk + dk
        inside = has & (nb >= start[t]) & (nb < start[t + 1])
        nbk = keys[ids[np.clip(nb, 0, max(ids.size - 1, 0))]] if ids.size else np.zeros_like(kk)
        tied |= inside & (np.abs(nbk - key) <= 2)
    return tied


def compare_views(sc, cams, sh_degree, pose_through_sh=0, bg=(0.0, 0.0, 0.0), max_amb_frac=0.3, max_excl_frac=0.05,
                  dLs=None, grad="l1", mip=0, margins=None, lam=FP32_LAMBDA, max_pose_share=POSE_SHARE, filter3d=None,
                  alpha_rect=1, **launch):
    """GPU vs oracle on every view: projection, image, n_contrib, the 2D adjoint
    per item, every visible Gaussian's parameter gradients and the pose
    gradient of each view.

    The adjoint input dL/dC is the workload's L1 gradient (grad="l1": a render
    at the training pose against a target from a perturbed pose), standard
    normal noise (grad="random"), or dLs when given. Gradients are held to
    1e-3 * (|ref| + rms) plus the oracle's own bound on what an FP32 evaluation
    may legitimately change: every decision within its margin flipped on its
    own and every uncertain tile membership toggled, plus lam x the root sum of
    squares of the first-order FP32 error of each contribution, carried to
    the parameters and the pose through the projection adjoint. Only items
    with a flagged projection decision (near plane, determinant, guard band,
    colour clamp: the adjoint's own path may differ) are left out, and
    counted. With the workload gradient the pose bound must stay below
    max_pose_share of |ref| + rms, except in a view where a Gaussian lies
    within the FP32 uncertainty of the near plane (reported).

    filter3d (per-Gaussian variances): the GPU renders with the 3-D smoothing
    filter; the oracle renders the equivalent unfiltered scene
    (O.filtered_scene) and its log-scale and logit gradients, and their
    bounds, are carried back to the original parameters (O.filter3d_chain)."""
    sc_in = sc
    if filter3d is not None:
        sc = O.filtered_scene(sc_in, filter3d)
    dil = 0.1 if mip else 0.3
    tile = launch.get("tile", 16)
    ocfg = O.Config(sh_degree=sh_degree, pose_grad_through_sh=pose_through_sh, bg=bg, tile=tile, mip_filter=mip,
                    dilation=dil, alpha_rect=alpha_rect, **(margins or MARGINS))
    views = [O.render_view(sc, cam, ocfg) for cam in cams]
    workload = dLs is None and grad == "l1"
    if dLs is None:
        if grad == "l1":
            dLs = workload_gradients(O, sc, cams, ocfg, views, synth)
        else:
            rng = np.random.default_rng(0)
            dLs = [rng.standard_normal((3, c["height"], c["width"])) for c in cams]
    r, dLs, d_proj = run_views(sc_in, cams, sh_degree, dLs=dLs, pose_through_sh=pose_through_sh, bg=bg,
                               mip_filter=mip, dilation=dil, filter3d=filter3d, alpha_rect=alpha_rect, **launch)
    n = sc.n
    keys = ("mean", "logit", "log_scale", "quat", "sh")
    ref = {k: 0.0 for k in keys}
    bnd = {k: 0.0 for k in keys}
    excl = np.zeros(n, bool)
    vis_any = np.zeros(n, bool)
    n_amb_px = 0
    pose_gpu = r.dpose.cpu().numpy()
    report = []
    for v, cam in enumerate(cams):
        w, h = cam["width"], cam["height"]
        view = views[v]
        proj = view["proj"]
        # projection outputs
        vis = proj["n_tiles"] > 0
        vis_any |= vis
        pg = r.proj
        sl = slice(v * n, (v + 1) * n)
        nt = pg.n_tiles[sl].cpu().numpy()
        # exact counts and rects away from flagged decisions: bit 1 (near plane,
        # determinant, radius) and bits 4-32 (a rect edge within the margin of a
        # tile boundary, which FP32 may round either way)
        geo_ok = (proj["amb"] & (1 | 4 | 8 | 16 | 32 | 64)) == 0
        assert np.array_equal(nt[geo_ok], proj["n_tiles"][geo_ok]), "n_tiles"
        rect = pg.rect[sl].cpu().numpy().astype(np.int32) & 0xFFFF
        both = geo_ok & vis
        assert np.array_equal(rect[both], proj["rect"][both]), "rect"
        assert_close(pg.mean2d[sl].cpu().numpy()[both], proj["mean2d"][both], 1e-5, what="mean2d")
        co = pg.conic_opa[sl].cpu().numpy()[both]
        assert_close(co[:, :3], proj["conic"][both], 1e-4, what="conic")
        assert_close(co[:, 3], proj["opacity"][both], 1e-5, what="opacity")
        rd = pg.rgb_depth[sl].cpu().numpy()[both]
        assert_close(rd[:, :3], proj["rgb"][both], 1e-5, what="rgb")
        assert_close(rd[:, 3], proj["depth"][both], 1e-6, what="depth")
        # image: pixels with an ambiguous decision and tiles an ambiguous rect may touch
        bad = O.ambiguous_tiles(view, cam, ocfg)
        pm = ~tile_pixel_mask(bad, w, h, tile) & (view["amb"] == 0)
        n_amb_px += int((~pm).sum())
        color = r.view_color(v).cpu().numpy()
        assert_close(color, view["color"], IMG_RTOL, np.broadcast_to(pm, color.shape), f"color view {v}")
        # n_contrib is a list position: compare it where the tile lists are unique
        # (a Gaussian a flagged rect edge may add or drop shifts it, alpha or not)
        pl = ~tile_pixel_mask(O.ambiguous_tiles(view, cam, ocfg, any_alpha=True), w, h, tile) & pm
        # ...and where the last contributor's list neighbours are not depth near-ties (keys
        # within 2 fp32 ulps may be ordered either way; the colour does not depend on it)
        pl &= ~last_contributor_tied(view, w, h, tile)
        nc = r.view_pixels(r.img.n_contrib, v).cpu().numpy()
        assert np.array_equal(nc[pl], view["n_contrib"][pl]), (v, int((nc[pl] != view["n_contrib"][pl]).sum()))
        # the oracle's adjoint of this view and its bounds
        b = O.backward_view(sc, cam, ocfg, view, dLs[v])
        bb = O.adjoint_bounds(sc, view, cam, ocfg, dLs[v])
        b2d = bb["flip"] + lam * bb["fp32"]
        geo = (proj["amb"] & (1 | 2 | 64)) > 0
        excl |= geo
        ok = vis & ~geo
        worst2d = 0.0
        for c in range(9):
            wr, _ = assert_within(d_proj[sl][:, c], b["g2d"][:, c], GRAD_RTOL, b2d[:, c], ok, f"d_proj[{c}] view {v}")
            worst2d = max(worst2d, wr)
        ab = O.project_bwd_abs(sc, cam, ocfg, b2d)
        for k in keys:
            ref[k] = ref[k] + b[k]
            bnd[k] = bnd[k] + ab[k]
        # pose of this view: its sum runs over every item; the bound covers the flips and rounding
        pr = b["pose"]
        pb = bb["pose_flip"] + lam * bb["pose_fp32"]
        wp, _ = assert_within(pose_gpu[v], pr, GRAD_RTOL, pb, what=f"pose view {v}")
        share = float((pb / (np.abs(pr) + np.sqrt(np.mean(pr * pr)))).max())
        report.append(f"view {v}: 2D adjoint worst {worst2d:.3f}, pose worst {wp:.3f}, pose bound share {share:.2e} "
                      f"({bb['memberships']} uncertain memberships, {bb['near_plane']} near-plane items, "
                      f"{bb['masked_pixels']} masked pixels)")
        # a Gaussian within the FP32 uncertainty of the near plane may appear as a splat hundreds of pixels
        # wide in front of everything: the pose bound of such a view is that large, and is reported
        if workload and bb["near_plane"] == 0:
            assert share <= max_pose_share, (v, share)
    if filter3d is not None:
        ref = O.filter3d_chain(sc_in, filter3d, ref)
        bnd = O.filter3d_chain(sc_in, filter3d, bnd, absolute=True)
    keep = vis_any & ~excl
    gr = r.grads
    mo = gr.mean_opa.cpu().numpy()
    ncoef = 3 * (sh_degree + 1) ** 2
    got = dict(mean=mo[:, :3], logit=mo[:, 3], log_scale=gr.scale.cpu().numpy()[:, :3], quat=gr.quat.cpu().numpy(),
               sh=gr.sh.cpu().numpy()[:, :ncoef])
    shares = []
    for k in keys:
        rk, bk = ref[k], bnd[k]
        if k == "sh":
            rk, bk = rk[:, :ncoef], bk[:, :ncoef]
        wr, med = assert_within(got[k], rk, GRAD_RTOL, bk, keep, f"d {k}")
        shares.append(f"{k} worst {wr:.3f} median bound/tol {med:.2f}")
    assert np.array_equal(gr.visible.cpu().numpy().astype(bool)[keep], vis_any[keep])
    total_px = sum(c["width"] * c["height"] for c in cams)
    assert n_amb_px <= max_amb_frac * total_px + 256, n_amb_px
    n_excl = int(excl[vis_any].sum())
    assert n_excl <= max_excl_frac * vis_any.sum() + 10, (n_excl, int(vis_any.sum()))
    print(f"\n[{len(cams)} views, {int(vis_any.sum())} visible Gaussians, {n_excl} excluded "
          f"({n_excl / max(1, vis_any.sum()):.2e})]")
    for line in report + shares:
        print("  " + line)
    return r, n_excl


@pytest.mark.parametrize("n_views", [10, 18])
def test_many_views_end_to_end(n_views):
    """Many views in one call: up to 16 views the projection adjoint forms the
    SH-coefficient sums after the view loop from shared memory, above 16 it
    keeps them in registers view by view."""
    sizes = ([(64, 48), (72, 40), (48, 64)] * 6)[:n_views - 1] + [(80, 56)]
    sc, cams, _ = synth.multiview_scene(seed=12, n=4000, n_views=len(sizes), sizes=sizes)
    compare_views(sc, cams, 3)


def test_three_sigma_rects_end_to_end():
    """The same three-view SH3 workload with the opacity-aware tile rects off:
    every Gaussian listed on the whole 3-sigma square of tiles."""
    sc, cams, _ = synth.multiview_scene(seed=5, n=20000, n_views=3, sizes=[(200, 120), (131, 77), (96, 160)])
    compare_views(sc, cams, 3, alpha_rect=0)


def test_opacity_aware_rects_change_no_output():
    """The opacity-aware rects drop only list entries whose Gaussian reaches
    alpha_min at no pixel of the tile: such an entry is skipped by compositing
    and its partials are exact zeros, so the image, the transmittance and
    every gradient are bit-identical with and without them (n_contrib, a list
    position, may move), on fewer pairs; a Gaussian whose opacity lets alpha
    reach alpha_min nowhere leaves every list, so the visible set can only
    shrink."""
    sc, cams, _ = synth.multiview_scene(seed=5, n=20000, n_views=3, sizes=[(200, 120), (131, 77), (96, 160)])
    rng = np.random.default_rng(9)
    dLs = [rng.standard_normal((3, c["height"], c["width"])) for c in cams]
    out = {}
    for ar in (0, 1):
        r, _, d_proj = run_views(sc, cams, 3, dLs=dLs, alpha_rect=ar)
        out[ar] = dict(pairs=int(r.pairs.count.item()), color=r.img.color.cpu().numpy(),
                       t=r.img.t_final.cpu().numpy(), vis=r.grads.visible.cpu().numpy().astype(bool),
                       d_proj=d_proj, pose=r.dpose.cpu().numpy(),
                       **{k: getattr(r.grads, k).cpu().numpy() for k in ("mean_opa", "scale", "quat", "sh")})
    a, b = out[0], out[1]
    assert b["pairs"] < a["pairs"], (a["pairs"], b["pairs"])
    assert not (b["vis"] & ~a["vis"]).any()
    for k in ("color", "t", "d_proj", "pose", "mean_opa", "scale", "quat", "sh"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("mip", [0, 1])
def test_tiny_scene_sh0_end_to_end(mip):
    """64x64 view, 1,000 Gaussians, SH degree 0, pose gradient (seeded); with
    and without the integral-keeping 2-D filter."""
    sc, cam, _ = synth.tiny_scene()
    compare_views(sc, [cam], 0, bg=(0.2, 0.1, 0.0), mip=mip)


@pytest.mark.parametrize("through_sh", [0, 1])
@pytest.mark.parametrize("grad", ["l1", "random"])
def test_multiview_sh3_end_to_end(through_sh, grad):
    """Three views of different sizes (ragged edge tiles), SH degree 3, with
    and without the SH view-direction path in the pose gradient; adjoint input
    the workload's L1 gradient or standard normal noise."""
    sc, cams, _ = synth.multiview_scene(seed=5, n=20000, n_views=3, sizes=[(200, 120), (131, 77), (96, 160)])
    compare_views(sc, cams, 3, pose_through_sh=through_sh, grad=grad)


@pytest.mark.parametrize("mip", [0, 1])
def test_filter3d_end_to_end(mip):
    """The 3-D smoothing filter (with and without the 2-D filter): gs_filter3d's
    variances from the three cameras against the oracle's sampling-rate rule,
    then projection, images, adjoint and every gradient against the oracle's
    equivalent unfiltered scene, the log-scale and logit gradients carried back
    through the filter."""
    sc, cams, _ = synth.multiview_scene(seed=5, n=20000, n_views=3, sizes=[(200, 120), (131, 77), (96, 160)])
    g = gs.Gaussians.from_scene(sc)
    out = torch.zeros(sc.n, device="cuda")
    gs.gs_filter3d(g, gs.cameras_tensor(cams), len(cams), out, gs.workspace(256))
    torch.cuda.synchronize()
    v_ref, amb = O.filter3d_variance(sc, cams, margin=1e-5)
    v_gpu = out.cpu().numpy()
    ok = ~amb
    assert ok.mean() > 0.99
    np.testing.assert_allclose(v_gpu[ok], v_ref[ok], rtol=1e-5)
    # the scene's own scales are about e^-4 = 0.018 m; v makes the filter matter for the distant ones
    assert np.median(v_ref / np.exp(2 * sc.scale[:, :3].astype(np.float64)).min(1)) > 0.05
    compare_views(sc, cams, 3, mip=mip, filter3d=v_ref)


def test_multiview_sh3_mip_filter_end_to_end():
    """The same three views with the integral-keeping 2-D filter (dilation 0.1):
    small splats lose opacity, so the filter's gradient path is exercised."""
    sc, cams, _ = synth.multiview_scene(seed=5, n=20000, n_views=3, sizes=[(200, 120), (131, 77), (96, 160)])
    compare_views(sc, cams, 3, mip=1)


@pytest.mark.parametrize("tile,schedule,fb,bb", [(8, 0, 64, 256), (8, 1, 256, 64), (16, 1, 64, 32),
                                                 (16, 2, 256, 64), (32, 0, 128, 32), (32, 1, 256, 32)])
def test_tiles_batches_schedules_end_to_end(tile, schedule, fb, bb):
    """Every tile size (8, 16, 32), staging depth and both render schedules
    give the oracle's images and gradients (the oracle at the same tile size)."""
    sc, cams, _ = synth.multiview_scene(seed=6, n=8000, n_views=2, sizes=[(200, 120), (96, 160)])
    compare_views(sc, cams, 3, tile=tile, schedule=schedule, fwd_batch=fb, bwd_batch=bb)


def test_graph_replay_matches_eager_steps():
    """Four optimisation steps issued eagerly and one eager step + three replays
    of a captured CUDA graph (device-side step counter) give bit-identical
    parameters, poses and Adam state."""
    from paper_2506_05558_gb300.raster import JointOptimizer
    sc, cams, rng = synth.multiview_scene(seed=9, n=5000, n_views=3, sizes=[(128, 96), (160, 64), (64, 64)])
    sizes = [(c["width"], c["height"]) for c in cams]
    targets = t32(rng.random(sum(3 * w * h for w, h in sizes)))
    outs = []
    for mode in ("eager", "graph"):
        g = gs.Gaussians.from_scene(sc)
        camt = gs.cameras_tensor(cams)
        J = JointOptimizer(g, camt, sizes, targets, 1 << 16, gs.config(sh_degree=3, schedule=1))
        J.step()
        if mode == "eager":
            for _ in range(3):
                J.step()
        else:
            J.capture(per_stage=(len(outs) % 2 == 1))
            for _ in range(3):
                J.replay()
        torch.cuda.synchronize()
        assert J.r.status() == gs.GS_OK and int(J.step_dev.item()) == 5
        outs.append([t.cpu().numpy().copy() for t in (g.mean_opa, g.scale, g.quat, g.sh, J.m.sh, J.v.mean_opa, camt)])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_set_targets_switches_the_loss_buffer():
    """Steps alternating between two target buffers with set_targets() equal
    steps of optimisers built on each buffer (bit for bit), and a buffer of
    another shape is refused."""
    from paper_2506_05558_gb300.raster import JointOptimizer
    sc, cams, rng = synth.multiview_scene(seed=10, n=3000, n_views=2, sizes=[(96, 64), (64, 80)])
    sizes = [(c["width"], c["height"]) for c in cams]
    n = sum(3 * w * h for w, h in sizes)
    ta, tb = t32(rng.random(n)), t32(rng.random(n))
    runs = []
    for switch in (True, False):
        g = gs.Gaussians.from_scene(sc)
        J = JointOptimizer(g, gs.cameras_tensor(cams), sizes, ta.clone(), 1 << 16, gs.config(sh_degree=3))
        losses = []
        for k in range(4):
            t = ta if k % 2 == 0 else tb
            if switch:
                J.set_targets(t)
            else:
                J.targets.copy_(t)
            losses.append(float(J.step().item()))
        torch.cuda.synchronize()
        runs.append((losses, g.mean_opa.cpu().numpy().copy()))
    assert runs[0][0] == runs[1][0] and np.array_equal(runs[0][1], runs[1][1])
    with pytest.raises(ValueError):
        J.set_targets(ta[:-3])


def test_headline_1m_8x1080p_end_to_end():
    """The benchmark workload at full size - 1M Gaussians SH3, 8 views 1920x1080 on
    the camera path - in the benchmark's launch configuration (tile 16, staging
    depths 256 forward / 64 backward, one CTA per tile, all views in one launch):
    every view's projection, image, n_contrib and 2D adjoint, every visible
    Gaussian's gradients and the 8 pose gradients against the FP64 oracle, with
    the adjoint input the workload's L1 gradient."""
    sc, cams, _ = synth.multiview_scene()
    # rect edges flagged within 5e-4 px of a tile boundary (the FP32 screen position at 1080p is good to about
    # 5 ulp of 1400 px, 4e-4 px; the observed flips sat within 1e-4 px)
    m = dict(MARGINS, margin_rect_px=5e-4)
    compare_views(sc, cams, 3, tile=16, fwd_batch=256, bwd_batch=64, schedule=0, max_amb_frac=0.1, margins=m)


def test_720p_200k_random_adjoint_end_to_end():
    """1280x720, 200k Gaussians, SH3, with standard normal dL/dC: the pose is then
    a near-zero sum of large terms of both signs, the hardest case for its
    bound, which is reported (the per-item and parameter checks are as strict
    as with the workload gradient)."""
    sc, cam, _ = synth.view_720p_scene()
    compare_views(sc, [cam], 3, grad="random")


def test_720p_200k_end_to_end():
    """1280x720, 200k Gaussians, SH3, 16x16 tiles (full size)."""
    sc, cam, _ = synth.view_720p_scene()
    compare_views(sc, [cam], 3)


@pytest.mark.parametrize("schedule", [0, 1, 2])
def test_depth_channel_matches_oracle(schedule):
    """The optional depth-integral output of the forward pass against the
    oracle (three views of different sizes, SH3), with colour and transmittance
    unchanged by requesting it."""
    sc, cams, _ = synth.multiview_scene(seed=31, n=3000, n_views=3, sizes=[(96, 64), (80, 48), (72, 72)])
    sizes = [(c["width"], c["height"]) for c in cams]
    cfg = gs.config(sh_degree=3, schedule=schedule)
    g = gs.Gaussians.from_scene(sc)
    camt = gs.cameras_tensor(cams)
    r = Rasterizer(sc.n, sizes, capacity=1024, cfg=cfg)
    r.fit_capacity(g, camt)
    r.forward(g, camt)
    color0 = r.img.color.clone()
    r.img.depth = torch.zeros_like(r.img.t_final)
    r.forward(g, camt)
    torch.cuda.synchronize()
    assert torch.equal(color0, r.img.color)
    ocfg = O.Config(sh_degree=3, **MARGINS)
    for v, cam in enumerate(cams):
        w, h = cam["width"], cam["height"]
        view = O.render_view(sc, cam, ocfg)
        bad = O.ambiguous_tiles(view, cam, ocfg)
        pm = ~tile_pixel_mask(bad, w, h, 16) & (view["amb"] == 0)
        ref = O.render_depth(view["proj"], view["start"], view["ids"], cam, ocfg)
        got = r.view_pixels(r.img.depth, v).cpu().numpy()
        assert_close(got, ref, IMG_RTOL, pm, f"depth view {v}")
        assert (ref[pm] > 0).mean() > 0.3


def test_projection_batched_equals_per_view():
    """One projection launch over five views of unequal size equals five
    single-view launches, bit for bit (a ragged Gaussian count, so the last
    block of every view is partial)."""
    sizes = [(320, 180), (256, 144), (200, 120), (320, 180), (160, 90)]
    sc, cams, _ = synth.multiview_scene(seed=1311, n=1037, n_views=len(sizes), sizes=sizes)
    g = gs.Gaussians.from_scene(sc)
    cfg = gs.config(sh_degree=3)
    out = gs.Projected.alloc(len(sizes) * sc.n)
    gs.gs_project(g, gs.cameras_tensor(cams), gs.frame(sizes), cfg, out)
    for v, size in enumerate(sizes):
        one = gs.Projected.alloc(sc.n)
        gs.gs_project(g, gs.cameras_tensor([cams[v]]), gs.frame([size]), cfg, one)
        rows = slice(v * sc.n, (v + 1) * sc.n)
        for name in ("mean2d", "conic_opa", "rgb_depth", "rect", "n_tiles"):
            assert torch.equal(getattr(out, name)[rows], getattr(one, name)), (v, name)
        assert int((one.n_tiles > 0).sum()) > 0.1 * sc.n


def test_nonfinite_gaussians_are_culled():
    sc, cam, _ = synth.tiny_scene(n=200)
    sc.mean_opa[3, 0] = np.nan
    sc.scale[5, 1] = np.inf
    sc.quat[7, :] = 0.0
    sc.sh[9, 0] = np.nan
    r, _, _ = run_views(sc, [cam], 0)
    nt = r.proj.n_tiles.cpu().numpy()
    assert nt[3] == 0 and nt[5] == 0 and nt[7] == 0 and nt[9] == 0
    assert np.isfinite(r.img.color.cpu().numpy()).all()
    for t in (r.grads.mean_opa, r.grads.scale, r.grads.sh, r.dpose):
        assert np.isfinite(t.cpu().numpy()).all()


# ---------------------------------------------------------------------------
# Loss and optimiser
# ---------------------------------------------------------------------------

def test_l1_loss_matches_oracle():
    rng = np.random.default_rng(3)
    for n in (1, 1001, 3 * 64 * 64):
        c = rng.random(n).astype(np.float32)
        t = rng.random(n).astype(np.float32)
        t[: n // 7] = c[: n // 7]
        dL = torch.zeros(n, device="cuda")
        loss = torch.zeros(1, device="cuda")
        gs.gs_l1_loss(t32(c), t32(t), dL, loss, gs.workspace(4 * 4096))
        ref_l, ref_g = O.l1_loss_grad(c, t)
        assert abs(loss.item() - ref_l) <= 1e-6 * abs(ref_l) + 1e-7
        assert np.array_equal(dL.cpu().numpy(), ref_g.astype(np.float32))


@pytest.mark.parametrize("decay", [None, 0.97])
def test_adam_matches_oracle(decay):
    """Three sparse Adam steps; optionally with per-Gaussian rate multipliers
    that decay each time a Gaussian is processed."""
    rng = np.random.default_rng(4)
    n = 3000
    params = {k: rng.standard_normal((n, w)).astype(np.float32) for k, w in
              (("mean_opa", 4), ("scale", 4), ("quat", 4), ("sh", 48))}
    params["scale"][:, 3] = 0
    P = gs.Gaussians(*[t32(params[k]) for k in ("mean_opa", "scale", "quat", "sh")])
    M, V = gs.Gaussians.zeros(n), gs.Gaussians.zeros(n)
    vis = rng.random(n) < 0.7
    cfg = gs.adam_config(lr_mean=0.01, lr_opacity=0.05, lr_scale=0.005, lr_rot=0.001, lr_sh_dc=0.0025,
                         lr_sh_rest=0.000125, decay=decay or 1.0)
    ls = rng.uniform(0.5, 1.0, n) if decay else np.ones(n)
    ls_dev = t32(ls) if decay else None
    ref = {k: (params[k].astype(np.float64), np.zeros_like(params[k], np.float64),
               np.zeros_like(params[k], np.float64)) for k in params}
    lrs = {"mean_opa": [0.01] * 3 + [0.05], "scale": [0.005] * 3 + [0.0], "quat": [0.001] * 4,
           "sh": [0.0025] * 3 + [0.000125] * 45}
    for step in (1, 2, 3):
        grads = {k: rng.standard_normal(params[k].shape).astype(np.float32) for k in params}
        grads["scale"][:, 3] = 0
        G = gs.Grads(*[t32(grads[k]) for k in ("mean_opa", "scale", "quat", "sh")],
                     torch.from_numpy(vis.astype(np.uint8)).cuda())
        gs.gs_adam_step(P, G, M, V, cfg, step, lr_scale=ls_dev)
        for k in params:
            p, m, v = ref[k]
            lr = np.array(lrs[k])
            out = [O.adam_step(p[:, j], grads[k][:, j], m[:, j], v[:, j], step, lr[j] * ls, eps=1e-15, mask=vis)
                   for j in range(p.shape[1])]
            ref[k] = tuple(np.stack([o[i] for o in out], 1) for i in range(3))
        if decay:
            ls = O.lr_decay(ls, vis, decay)
    torch.cuda.synchronize()
    if decay:
        assert_close(ls_dev.cpu().numpy(), ls, 1e-6, what="rate multipliers")
    for k, t in (("mean_opa", P.mean_opa), ("scale", P.scale), ("quat", P.quat), ("sh", P.sh)):
        assert_close(t.cpu().numpy(), ref[k][0], 1e-5, what=k)


def test_pose_step_matches_oracle_retraction():
    rng = np.random.default_rng(5)
    cams = [synth.camera(*O.retract_pose(np.eye(3), rng.normal(0, 1, 3), rng.normal(0, 0.3, 6)), 500.0, 64, 64)
            for _ in range(3)]
    camt = gs.cameras_tensor(cams)
    grad = rng.standard_normal((3, 6)).astype(np.float32)
    m = torch.zeros((3, 6), device="cuda")
    v = torch.zeros((3, 6), device="cuda")
    gs.gs_pose_step(camt, 3, t32(grad), m, v, 0.01, 0.02, 1)
    out = gs.cameras_from_tensor(camt)
    for i in range(3):
        lr = np.array([0.01] * 3 + [0.02] * 3)
        step = -lr * np.sign(grad[i])  # Adam's first step
        R, t = O.retract_pose(cams[i]["R"], cams[i]["t"], step)
        assert np.abs(out[i]["R"] - R).max() < 2e-6
        assert np.abs(out[i]["t"] - t).max() < 2e-5 * max(1.0, np.abs(t).max())


def test_downsample_matches_oracle():
    rng = np.random.default_rng(9)
    for W, H, f in ((64, 48, 2), (67, 45, 4), (31, 17, 8), (16, 16, 1)):
        im = rng.random((3, H, W)).astype(np.float32)
        out = gs.gs_downsample(t32(im.reshape(-1)), W, H, f)
        torch.cuda.synchronize()
        ref = O.downsample(im, f)
        assert_close(out.cpu().numpy().reshape(ref.shape), ref, 1e-6, what=f"downsample {W}x{H}/{f}")


def test_counting_forward_gives_the_same_image_and_consistent_counts():
    """The measurement instantiation of the forward (gs_render_fwd_count) writes
    the same image, transmittance and n_contrib as gs_render_fwd, bit for bit,
    and its counts are ordered: composited <= live-lane evaluations <= 32 x warp
    hits, and composited equals the oracle's count of compositing evaluations
    away from flagged pixels within a small tolerance."""
    sc, cams, _ = synth.multiview_scene(seed=41, n=6000, n_views=2, sizes=[(160, 96), (96, 128)])
    sizes = [(c["width"], c["height"]) for c in cams]
    g = gs.Gaussians.from_scene(sc)
    camt = gs.cameras_tensor(cams)
    r = Rasterizer(sc.n, sizes, capacity=1024, cfg=gs.config(sh_degree=3))
    r.fit_capacity(g, camt)
    r.forward(g, camt)
    ref = [t.clone() for t in (r.img.color, r.img.t_final, r.img.n_contrib)]
    counts = torch.zeros(3, dtype=torch.int64, device="cuda")
    gs.gs_render_fwd_count(r.proj, r.pairs, r.f, r.cfg, r.img, counts, r.ws_render)
    torch.cuda.synchronize()
    for a, b in zip(ref, (r.img.color, r.img.t_final, r.img.n_contrib)):
        assert torch.equal(a, b)
    hits, lanes, comp = counts.cpu().tolist()
    assert 0 < comp <= lanes <= 32 * hits
    # the oracle's number of compositing evaluations (alpha >= alpha_min, before termination)
    ocfg = O.Config(sh_degree=3, **MARGINS)
    total = 0
    for cam in cams:
        view = O.render_view(sc, cam, ocfg)
        total += int(view["n_composited"].sum())
    assert abs(comp - total) <= 1e-3 * total, (comp, total)
