"""torch.autograd binding of the rasteriser: the forward is gs_pose_apply +
gs_project + gs_sort + gs_render_fwd, the backward the hand-written adjoint
gs_render_bwd followed by gs_pose_tangent_grad (Sec. 4.3: Gaussians and
camera poses optimised jointly; the pose gradient excludes the SH view
direction unless the config asks for it).

The camera pose of view i is exp(xi_i^) T_i with T_i the reference pose in
`cams_ref` and xi_i = (rho, phi) a tangent vector that requires grad, so a
PyTorch optimiser can step poses directly, or the caller can retract xi into
T and reset it to zero after each step.

Each call owns its rasteriser buffers (drawn from PyTorch's caching
allocator), so several renders may be alive before their backward passes. The
forward synchronises once, to grow the (tile, Gaussian) pair buffer when the
sort reports an overflow; the graph-captured training step in raster.py is the
synchronisation-free path.
"""
from __future__ import annotations

import torch

from . import gs
from .raster import Rasterizer


class _Rasterize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mean_opa, scale, quat, sh, xi, cams_ref, sizes, cfg, capacity_hint):
        n_views = len(sizes)
        cams = torch.empty_like(cams_ref)
        gs.gs_pose_apply(cams_ref, xi.detach().contiguous(), n_views, cams)
        g = gs.Gaussians(mean_opa.detach().contiguous(), scale.detach().contiguous(), quat.detach().contiguous(),
                         sh.detach().contiguous())
        r = Rasterizer(g.n, sizes, capacity_hint, cfg, mean_opa.device)
        r.fit_capacity(g, cams)
        r.forward(g, cams)
        ctx.r, ctx.g, ctx.cams = r, g, cams
        ctx.save_for_backward(xi)
        color, t_final = r.img.color.clone(), r.img.t_final.clone()
        ctx.mark_non_differentiable(t_final)
        return color, t_final

    @staticmethod
    def backward(ctx, d_color, d_t_final):
        (xi,) = ctx.saved_tensors
        r = ctx.r
        if d_color is None:
            d_color = torch.zeros_like(r.img.color)
        r.backward(ctx.g, ctx.cams, d_color.contiguous())
        gr = r.grads
        d_xi = None
        if ctx.needs_input_grad[4]:
            d_xi = torch.empty_like(r.dpose)
            gs.gs_pose_tangent_grad(xi.detach().contiguous(), r.dpose, r.n_views, d_xi)
        ctx.r = ctx.g = ctx.cams = None
        return gr.mean_opa, gr.scale, gr.quat, gr.sh, d_xi, None, None, None, None


def rasterize(mean_opa: torch.Tensor, scale: torch.Tensor, quat: torch.Tensor, sh: torch.Tensor, xi: torch.Tensor,
              cams_ref: torch.Tensor, sizes, cfg: gs.gs_config | None = None, capacity_hint: int = 1 << 20):
    """Differentiable render of n_views = len(sizes) views.

    mean_opa [N, 4] (mean xyz, opacity logit), scale [N, 4] (log-scales xyz,
    4th unused), quat [N, 4] (w, x, y, z; normalised inside), sh [N, 48] (16
    RGB coefficients per Gaussian, bands above cfg.sh_degree ignored): float32
    CUDA tensors. xi [n_views, 6] the pose tangents, cams_ref the reference
    cameras (gs.cameras_tensor). Returns (color, t_final): color float32
    [3 * sum(W * H)], view after view, each view planar [3][H][W];
    t_final [sum(W * H)] the final transmittance (not differentiable).
    Gradients flow to all five tensor inputs; the column after each 3-vector
    of mean_opa/scale receives its own gradient (opacity logit) or zero.
    """
    if cfg is None:
        cfg = gs.config()
    return _Rasterize.apply(mean_opa, scale, quat, sh, xi, cams_ref, list(sizes), cfg, capacity_hint)
