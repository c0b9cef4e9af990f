"""Thin Python binding of libgs (include/gs.h): argument marshalling only.

Every step of the hot path runs in the library's sm_103a kernels. PyTorch
supplies device memory and the current CUDA stream; the structures below mirror
the C structs byte for byte. If the compiled library is missing, `lib()`
raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libgs.so")

GS_OK = 0
GS_ERR_INVALID_ARG = -1
GS_ERR_CAPACITY = -2
GS_ERR_CUDA = -3
GS_ERR_TIMEOUT = -4
GS_MAX_VIEWS = 64

# Every entry point declared in include/gs.h.
EXPORTS = [
    "gs_config_default", "gs_frame_init", "gs_filter3d", "gs_project", "gs_sort_workspace_size", "gs_sort",
    "gs_render_workspace_size", "gs_render_fwd", "gs_render_fwd_count", "gs_probe_fma", "gs_probe_mufu",
    "gs_backward_workspace_size", "gs_render_bwd",
    "gs_adam_step", "gs_pose_step", "gs_l1_loss", "gs_composite_bwd", "gs_project_bwd", "gs_launch_count",
    "gs_spawn_workspace_size", "gs_spawn_propose", "gs_counter_add", "gs_spawn_propose_noalloc",
    "gs_anchor_check", "gs_anchor_offload", "gs_anchor_load",
    "gs_mlp_patches", "gs_mlp_param_count", "gs_mlp_workspace_size", "gs_mlp_forward", "gs_mlp_train_step",
    "gs_mlp_gemm_bf16", "gs_mlp_tc_error", "gs_mlp_targets_workspace_size", "gs_mlp_targets", "gs_spawn_learned",
    "gs_pose_apply", "gs_pose_tangent_grad", "gs_anchor_merge_workspace_size", "gs_anchor_merge",
    "gs_anchor_blend_weight", "gs_scale_opacity", "gs_cull_opacity_workspace_size", "gs_cull_opacity",
    "gs_downsample", "gs_ba_workspace_size", "gs_ba_lm", "gs_ba_project", "gs_guided_depth",
    "gs_ba_pose_workspace_size", "gs_ba_pose_lm",
]


class gs_camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class gs_config(C.Structure):
    _fields_ = [("tile", C.c_int32), ("sh_degree", C.c_int32), ("near_z", C.c_float), ("dilation", C.c_float),
                ("alpha_min", C.c_float), ("alpha_max", C.c_float), ("t_min", C.c_float), ("bg", C.c_float * 3),
                ("pose_grad_through_sh", C.c_int32), ("schedule", C.c_int32), ("accumulate", C.c_int32),
                ("fwd_batch", C.c_int32), ("bwd_batch", C.c_int32), ("mip_filter", C.c_int32),
                ("alpha_rect", C.c_int32)]


class gs_frame(C.Structure):
    _fields_ = [("n_views", C.c_int32), ("tile", C.c_int32), ("width", C.c_int32 * GS_MAX_VIEWS),
                ("height", C.c_int32 * GS_MAX_VIEWS), ("tiles_x", C.c_int32 * GS_MAX_VIEWS),
                ("tiles_y", C.c_int32 * GS_MAX_VIEWS), ("tile_base", C.c_int32 * (GS_MAX_VIEWS + 1)),
                ("pix_base", C.c_int64 * (GS_MAX_VIEWS + 1))]


class gs_gaussians(C.Structure):
    _fields_ = [("mean_opa", C.c_void_p), ("scale", C.c_void_p), ("quat", C.c_void_p), ("sh", C.c_void_p),
                ("n", C.c_int64), ("filter3d", C.c_void_p)]


class gs_projected(C.Structure):
    _fields_ = [("mean2d", C.c_void_p), ("conic_opa", C.c_void_p), ("rgb_depth", C.c_void_p), ("rect", C.c_void_p),
                ("n_tiles", C.c_void_p)]


class gs_pairs(C.Structure):
    _fields_ = [("src", C.c_void_p), ("emit", C.c_void_p), ("offset", C.c_void_p), ("range", C.c_void_p),
                ("capacity", C.c_int64), ("count", C.c_void_p), ("status", C.c_void_p), ("order", C.c_void_p)]


class gs_image(C.Structure):
    _fields_ = [("color", C.c_void_p), ("t_final", C.c_void_p), ("n_contrib", C.c_void_p), ("depth", C.c_void_p)]


class gs_grads(C.Structure):
    _fields_ = [("mean_opa", C.c_void_p), ("scale", C.c_void_p), ("quat", C.c_void_p), ("sh", C.c_void_p),
                ("visible", C.c_void_p)]


class gs_adam_config(C.Structure):
    _fields_ = [("lr_mean", C.c_float), ("lr_opacity", C.c_float), ("lr_scale", C.c_float), ("lr_rot", C.c_float),
                ("lr_sh_dc", C.c_float), ("lr_sh_rest", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("decay", C.c_float)]


class gs_spawn_config(C.Structure):
    _fields_ = [("sigma", C.c_float), ("frame", C.c_uint32), ("seed", C.c_uint64)]


class gs_spawn_out(C.Structure):
    _fields_ = [("mean_opa", C.c_void_p), ("scale", C.c_void_p), ("quat", C.c_void_p), ("sh", C.c_void_p),
                ("pixel", C.c_void_p), ("capacity", C.c_int64), ("count", C.c_void_p), ("status", C.c_void_p),
                ("p_l", C.c_void_p), ("p_pen", C.c_void_p), ("p_s", C.c_void_p)]


class gs_mlp_params(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("w1", "b1", "w2", "b2", "w3", "b3", "w4", "b4")]


class gs_mlp_config(C.Structure):
    _fields_ = [("tensor_path", C.c_int32), ("w_depth", C.c_float), ("w_scale", C.c_float), ("lr", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float)]


_lib = None


def lib():
    """Loads libgs.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgs.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        sig = {
            "gs_config_default": (None, [C.POINTER(gs_config)]),
            "gs_frame_init": (C.c_int, [C.POINTER(gs_frame), C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                        C.c_int32]),
            "gs_filter3d": (C.c_int, [C.POINTER(gs_gaussians), P, C.c_int32, C.c_float, C.c_float, P, P,
                                      C.c_size_t, P]),
            "gs_project": (C.c_int, [C.POINTER(gs_gaussians), P, C.POINTER(gs_frame), C.POINTER(gs_config),
                                     C.POINTER(gs_projected), P]),
            "gs_sort_workspace_size": (C.c_size_t, [C.c_int64, C.POINTER(gs_frame), C.c_int64]),
            "gs_sort": (C.c_int, [C.POINTER(gs_projected), C.c_int64, C.POINTER(gs_frame), C.POINTER(gs_pairs), P,
                                  C.c_size_t, P]),
            "gs_render_workspace_size": (C.c_size_t, [C.POINTER(gs_frame)]),
            "gs_render_fwd": (C.c_int, [C.POINTER(gs_projected), C.POINTER(gs_pairs), C.POINTER(gs_frame),
                                        C.POINTER(gs_config), C.POINTER(gs_image), P, C.c_size_t, P]),
            "gs_render_fwd_count": (C.c_int, [C.POINTER(gs_projected), C.POINTER(gs_pairs), C.POINTER(gs_frame),
                                              C.POINTER(gs_config), C.POINTER(gs_image), P, C.c_size_t, P, P]),
            "gs_probe_fma": (C.c_int, [P, C.c_int32, C.c_int32, P]),
            "gs_probe_mufu": (C.c_int, [P, C.c_int32, C.c_int32, P]),
            "gs_backward_workspace_size": (C.c_size_t, [C.c_int64, C.POINTER(gs_frame), C.c_int64]),
            "gs_render_bwd": (C.c_int, [C.POINTER(gs_gaussians), P, C.POINTER(gs_projected), C.POINTER(gs_pairs),
                                        C.POINTER(gs_frame), C.POINTER(gs_config), C.POINTER(gs_image), P,
                                        C.POINTER(gs_grads), P, P, P, C.c_size_t, P]),
            "gs_adam_step": (C.c_int, [C.POINTER(gs_gaussians), C.POINTER(gs_grads), C.POINTER(gs_gaussians),
                                       C.POINTER(gs_gaussians), C.POINTER(gs_adam_config), C.c_int32, P, P, P]),
            "gs_pose_step": (C.c_int, [P, C.c_int32, P, P, P, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float,
                                       C.c_int32, P, P]),
            "gs_counter_add": (C.c_int, [P, C.c_int32, P]),
            "gs_downsample": (C.c_int, [P, C.c_int32, C.c_int32, C.c_int32, P, P]),
            "gs_ba_workspace_size": (C.c_size_t, [C.c_int32, C.c_int64]),
            "gs_ba_project": (C.c_int, [P, P, P, C.c_int32, C.c_int64, C.c_float, C.c_float, P, P]),
            "gs_ba_lm": (C.c_int, [P, C.c_int32, C.c_int64, C.c_float, C.c_float, P, P, P, P, C.c_int32, C.c_float,
                                   C.c_float, P, P, P, C.c_size_t, P]),
            "gs_pose_apply": (C.c_int, [P, P, C.c_int32, P, P]),
            "gs_ba_pose_workspace_size": (C.c_size_t, [C.c_int64]),
            "gs_ba_pose_lm": (C.c_int, [P, P, C.c_int64, P, C.c_float, C.c_float, P, P, C.c_int32, C.c_float, C.c_float,
                                        P, P, P, C.c_size_t, P]),
            "gs_guided_depth": (C.c_int, [P, P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P, C.c_int32, C.c_float,
                                          P, P, P, P]),
            "gs_anchor_merge_workspace_size": (C.c_size_t, [C.c_int64, C.c_int32]),
            "gs_anchor_merge": (C.c_int, [C.POINTER(gs_gaussians)] * 3 + [P, P, C.c_float, C.c_int32, C.c_uint64] +
                                [C.POINTER(gs_gaussians)] * 3 + [P, P, P, C.c_size_t, P]),
            "gs_cull_opacity_workspace_size": (C.c_size_t, [C.c_int64]),
            "gs_cull_opacity": (C.c_int, [C.POINTER(gs_gaussians)] * 3 + [P, C.c_float] +
                                [C.POINTER(gs_gaussians)] * 3 + [P, P, P, C.c_size_t, P]),
            "gs_anchor_blend_weight": (C.c_float, [C.c_float, C.c_float, C.c_float]),
            "gs_scale_opacity": (C.c_int, [P, C.c_int64, C.c_float, P]),
            "gs_pose_tangent_grad": (C.c_int, [P, P, C.c_int32, P, P]),
            "gs_l1_loss": (C.c_int, [P, P, C.c_int64, P, P, P, C.c_size_t, P]),
            "gs_composite_bwd": (C.c_int, [C.POINTER(gs_projected), C.POINTER(gs_pairs), C.POINTER(gs_frame),
                                           C.POINTER(gs_config), C.POINTER(gs_image), P, C.c_int64, P, C.c_size_t,
                                           P]),
            "gs_project_bwd": (C.c_int, [C.POINTER(gs_gaussians), P, C.POINTER(gs_projected), C.POINTER(gs_pairs),
                                         C.POINTER(gs_frame), C.POINTER(gs_config), C.POINTER(gs_grads), P, P, P,
                                         C.c_size_t, P]),
            "gs_launch_count": (C.c_int64, []),
            "gs_anchor_check": (C.c_int, [C.POINTER(gs_gaussians), P, C.c_float, P, P, P]),
            "gs_mlp_patches": (C.c_int64, [C.c_int32, C.c_int32]),
            "gs_mlp_param_count": (C.c_int64, []),
            "gs_mlp_workspace_size": (C.c_size_t, [C.c_int64]),
            "gs_mlp_forward": (C.c_int, [C.POINTER(gs_mlp_params), P, C.c_int32, C.c_int32, P,
                                         C.POINTER(gs_mlp_config), P, C.c_size_t, P]),
            "gs_mlp_train_step": (C.c_int, [C.POINTER(gs_mlp_params), C.POINTER(gs_mlp_params),
                                            C.POINTER(gs_mlp_params), P, C.c_int32, C.c_int32, P,
                                            C.POINTER(gs_mlp_config), C.c_int32, P, P, P, P, P, C.c_size_t, P]),
            "gs_mlp_gemm_bf16": (C.c_int, [P, C.c_int64, P, C.c_int64, P, C.c_int64, C.c_int32, C.c_int32, C.c_int32,
                                           C.c_int32, P]),
            "gs_mlp_tc_error": (C.c_int, [C.POINTER(C.c_int32)]),
            "gs_mlp_targets_workspace_size": (C.c_size_t, [C.c_int32, C.c_int32]),
            "gs_mlp_targets": (C.c_int, [P, P, P, P, P, C.c_float, C.c_int64, C.c_int32, C.c_int32, P, P, C.c_size_t,
                                          P]),
            "gs_spawn_learned": (C.c_int, [P, P, P, P, C.c_int32, C.c_int32, P, C.POINTER(gs_spawn_config),
                                           C.POINTER(gs_spawn_out), P, C.c_size_t, P]),
            "gs_anchor_offload": (C.c_int, [C.POINTER(gs_gaussians)] * 6 + [P]),
            "gs_anchor_load": (C.c_int, [C.POINTER(gs_gaussians)] * 6 + [P]),
            "gs_spawn_workspace_size": (C.c_size_t, [C.c_int32, C.c_int32]),
            "gs_spawn_propose_noalloc": (C.c_int, [P, P, P, C.c_int32, C.c_int32, P, C.POINTER(gs_spawn_config),
                                                   C.POINTER(gs_spawn_out), P]),
            "gs_spawn_propose": (C.c_int, [P, P, P, C.c_int32, C.c_int32, P, C.POINTER(gs_spawn_config),
                                           C.POINTER(gs_spawn_out), P, C.c_size_t, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, name: str):
    if rc != GS_OK:
        raise RuntimeError(f"{name} returned {rc}")


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


# ---------------------------------------------------------------------------
# Host structures
# ---------------------------------------------------------------------------

def config(**kw) -> gs_config:
    c = gs_config()
    lib().gs_config_default(C.byref(c))
    for k, v in kw.items():
        if k == "bg":
            c.bg[:] = list(v)
        else:
            setattr(c, k, v)
    return c


def frame(sizes, tile: int = 16) -> gs_frame:
    """sizes: list of (width, height) per view."""
    f = gs_frame()
    n = len(sizes)
    w = (C.c_int32 * n)(*[int(s[0]) for s in sizes])
    h = (C.c_int32 * n)(*[int(s[1]) for s in sizes])
    _check(lib().gs_frame_init(C.byref(f), n, w, h, tile), "gs_frame_init")
    return f


def cameras_tensor(cams, device="cuda") -> torch.Tensor:
    """Packs camera dicts (R, t, fx, fy, cx, cy, width, height) into the device
    array of gs_camera structs (a uint8 tensor of n * 72 bytes)."""
    arr = (gs_camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i].R[:] = [float(x) for x in np.asarray(c["R"], np.float64).reshape(9)]
        arr[i].t[:] = [float(x) for x in np.asarray(c["t"], np.float64).reshape(3)]
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = c["fx"], c["fy"], c["cx"], c["cy"]
        arr[i].width, arr[i].height = c["width"], c["height"]
    raw = np.frombuffer(bytes(arr), np.uint8).copy()
    return torch.from_numpy(raw).to(device)


def cameras_from_tensor(t: torch.Tensor):
    raw = t.detach().cpu().numpy().tobytes()
    arr = (gs_camera * (len(raw) // C.sizeof(gs_camera))).from_buffer_copy(raw)
    return [dict(R=np.array(a.R[:], np.float32).reshape(3, 3), t=np.array(a.t[:], np.float32), fx=a.fx, fy=a.fy,
                 cx=a.cx, cy=a.cy, width=a.width, height=a.height) for a in arr]


# ---------------------------------------------------------------------------
# Device buffers (torch tensors) and their C views
# ---------------------------------------------------------------------------

@dataclass
class Gaussians:
    mean_opa: torch.Tensor  # [n, 4]
    scale: torch.Tensor     # [n, 4]
    quat: torch.Tensor      # [n, 4]
    sh: torch.Tensor        # [n, 48]
    filter3d: torch.Tensor | None = None  # [n] variance of the 3-D smoothing filter, or None (off)

    @property
    def n(self) -> int:
        return int(self.mean_opa.shape[0])

    @staticmethod
    def from_scene(sc, device="cuda") -> "Gaussians":
        f = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(device)
        return Gaussians(f(sc.mean_opa), f(sc.scale), f(sc.quat), f(sc.sh))

    @staticmethod
    def zeros(n, device="cuda") -> "Gaussians":
        z = lambda k: torch.zeros((n, k), dtype=torch.float32, device=device)
        return Gaussians(z(4), z(4), z(4), z(48))

    def c(self) -> gs_gaussians:
        return gs_gaussians(_ptr(self.mean_opa), _ptr(self.scale), _ptr(self.quat), _ptr(self.sh), self.n,
                            _ptr(self.filter3d))


@dataclass
class Projected:
    mean2d: torch.Tensor
    conic_opa: torch.Tensor
    rgb_depth: torch.Tensor
    rect: torch.Tensor
    n_tiles: torch.Tensor

    @staticmethod
    def alloc(items, device="cuda") -> "Projected":
        return Projected(torch.zeros((items, 2), dtype=torch.float32, device=device),
                         torch.zeros((items, 4), dtype=torch.float32, device=device),
                         torch.zeros((items, 4), dtype=torch.float32, device=device),
                         torch.zeros((items, 4), dtype=torch.int16, device=device),
                         torch.zeros((items,), dtype=torch.int32, device=device))

    def c(self) -> gs_projected:
        return gs_projected(_ptr(self.mean2d), _ptr(self.conic_opa), _ptr(self.rgb_depth), _ptr(self.rect),
                            _ptr(self.n_tiles))


@dataclass
class Pairs:
    src: torch.Tensor
    emit: torch.Tensor
    offset: torch.Tensor
    range: torch.Tensor
    count: torch.Tensor
    status: torch.Tensor
    order: torch.Tensor | None = None

    @property
    def capacity(self) -> int:
        return int(self.src.shape[0])

    @staticmethod
    def alloc(items, n_tiles_total, capacity, device="cuda", with_order=True) -> "Pairs":
        u32 = lambda k: torch.zeros((k,), dtype=torch.int32, device=device)
        return Pairs(u32(max(capacity, 1)), u32(max(capacity, 1)), u32(max(items, 1)), u32(2 * n_tiles_total),
                     torch.zeros((1,), dtype=torch.int64, device=device),
                     torch.zeros((1,), dtype=torch.int32, device=device),
                     u32(max(n_tiles_total, 1)) if with_order else None)

    def c(self) -> gs_pairs:
        return gs_pairs(_ptr(self.src), _ptr(self.emit), _ptr(self.offset), _ptr(self.range), self.capacity,
                        _ptr(self.count), _ptr(self.status), _ptr(self.order))


@dataclass
class Image:
    color: torch.Tensor
    t_final: torch.Tensor
    n_contrib: torch.Tensor
    depth: torch.Tensor | None = None  # depth integral, written only when present

    @staticmethod
    def alloc(n_pix, device="cuda", with_depth=False) -> "Image":
        return Image(torch.zeros((3 * n_pix,), dtype=torch.float32, device=device),
                     torch.zeros((n_pix,), dtype=torch.float32, device=device),
                     torch.zeros((n_pix,), dtype=torch.int32, device=device),
                     torch.zeros((n_pix,), dtype=torch.float32, device=device) if with_depth else None)

    def c(self) -> gs_image:
        return gs_image(_ptr(self.color), _ptr(self.t_final), _ptr(self.n_contrib), _ptr(self.depth))


@dataclass
class Grads:
    mean_opa: torch.Tensor
    scale: torch.Tensor
    quat: torch.Tensor
    sh: torch.Tensor
    visible: torch.Tensor

    @staticmethod
    def alloc(n, device="cuda") -> "Grads":
        z = lambda k: torch.zeros((n, k), dtype=torch.float32, device=device)
        return Grads(z(4), z(4), z(4), z(48), torch.zeros((n,), dtype=torch.uint8, device=device))

    def c(self) -> gs_grads:
        return gs_grads(_ptr(self.mean_opa), _ptr(self.scale), _ptr(self.quat), _ptr(self.sh), _ptr(self.visible))


def workspace(nbytes: int, device="cuda") -> torch.Tensor:
    """Caller-owned scratch; torch's allocator returns 512-byte aligned blocks."""
    return torch.empty((max(int(nbytes), 256),), dtype=torch.uint8, device=device)


# ---------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def gs_filter3d(g: Gaussians, cams: torch.Tensor, n_views: int, out: torch.Tensor, ws: torch.Tensor,
                near_z: float = 0.2, s2: float = 0.2, stream=None):
    gc = g.c()
    _check(lib().gs_filter3d(C.byref(gc), _ptr(cams), n_views, near_z, s2, _ptr(out), _ptr(ws), ws.numel(),
                             _stream(stream)), "gs_filter3d")


def gs_project(g: Gaussians, cams: torch.Tensor, f: gs_frame, cfg: gs_config, out: Projected, stream=None):
    gc, pc = g.c(), out.c()
    _check(lib().gs_project(C.byref(gc), _ptr(cams), C.byref(f), C.byref(cfg), C.byref(pc), _stream(stream)),
           "gs_project")


def gs_sort_workspace_size(n: int, f: gs_frame, capacity: int) -> int:
    return int(lib().gs_sort_workspace_size(n, C.byref(f), capacity))


def gs_sort(p: Projected, n: int, f: gs_frame, out: Pairs, ws: torch.Tensor, stream=None):
    pc, oc = p.c(), out.c()
    _check(lib().gs_sort(C.byref(pc), n, C.byref(f), C.byref(oc), _ptr(ws), ws.numel(), _stream(stream)), "gs_sort")


def gs_render_workspace_size(f: gs_frame) -> int:
    return int(lib().gs_render_workspace_size(C.byref(f)))


def gs_render_fwd(p: Projected, pairs: Pairs, f: gs_frame, cfg: gs_config, out: Image, ws=None, stream=None):
    pc, qc, oc = p.c(), pairs.c(), out.c()
    _check(lib().gs_render_fwd(C.byref(pc), C.byref(qc), C.byref(f), C.byref(cfg), C.byref(oc), _ptr(ws),
                               0 if ws is None else ws.numel(), _stream(stream)), "gs_render_fwd")


def gs_render_fwd_count(p: Projected, pairs: Pairs, f: gs_frame, cfg: gs_config, out: Image, counts: torch.Tensor,
                        ws=None, stream=None):
    """Measurement: the forward with its evaluations counted into counts
    (int64 [3] on the device): warp hits, lane evaluations of live pixels,
    compositing evaluations."""
    assert counts.dtype == torch.int64 and counts.numel() >= 3
    pc, qc, oc = p.c(), pairs.c(), out.c()
    _check(lib().gs_render_fwd_count(C.byref(pc), C.byref(qc), C.byref(f), C.byref(cfg), C.byref(oc), _ptr(ws),
                                     0 if ws is None else ws.numel(), _ptr(counts), _stream(stream)),
           "gs_render_fwd_count")


def gs_probe_fma(out: torch.Tensor, blocks: int, iters: int, stream=None):
    """Measurement: blocks x 256 threads x 128 iters FMAs; out float32 [blocks * 256]."""
    assert out.dtype == torch.float32 and out.numel() >= blocks * 256
    _check(lib().gs_probe_fma(_ptr(out), blocks, iters, _stream(stream)), "gs_probe_fma")


def gs_probe_mufu(out: torch.Tensor, blocks: int, iters: int, stream=None):
    """Measurement: blocks x 256 threads x 64 iters MUFU operations (2^x, 1/x)."""
    assert out.dtype == torch.float32 and out.numel() >= blocks * 256
    _check(lib().gs_probe_mufu(_ptr(out), blocks, iters, _stream(stream)), "gs_probe_mufu")


def gs_backward_workspace_size(n: int, f: gs_frame, capacity: int) -> int:
    return int(lib().gs_backward_workspace_size(n, C.byref(f), capacity))


def gs_render_bwd(g: Gaussians, cams: torch.Tensor, p: Projected, pairs: Pairs, f: gs_frame, cfg: gs_config,
                  fwd: Image, dL_dcolor: torch.Tensor, grads: Grads, dL_dpose: torch.Tensor, ws: torch.Tensor,
                  d_proj: torch.Tensor | None = None, stream=None):
    gc, pc, qc, ic, rc = g.c(), p.c(), pairs.c(), fwd.c(), grads.c()
    _check(lib().gs_render_bwd(C.byref(gc), _ptr(cams), C.byref(pc), C.byref(qc), C.byref(f), C.byref(cfg),
                               C.byref(ic), _ptr(dL_dcolor), C.byref(rc), _ptr(dL_dpose), _ptr(d_proj), _ptr(ws),
                               ws.numel(), _stream(stream)), "gs_render_bwd")


def gs_composite_bwd(p: Projected, pairs: Pairs, f: gs_frame, cfg: gs_config, fwd: Image, dL_dcolor: torch.Tensor,
                     n: int, ws: torch.Tensor, stream=None):
    pc, qc, ic = p.c(), pairs.c(), fwd.c()
    _check(lib().gs_composite_bwd(C.byref(pc), C.byref(qc), C.byref(f), C.byref(cfg), C.byref(ic), _ptr(dL_dcolor),
                                  n, _ptr(ws), ws.numel(), _stream(stream)), "gs_composite_bwd")


def gs_project_bwd(g: Gaussians, cams: torch.Tensor, p: Projected, pairs: Pairs, f: gs_frame, cfg: gs_config,
                   grads: Grads, dL_dpose: torch.Tensor, ws: torch.Tensor, d_proj=None, stream=None):
    gc, pc, qc, rc = g.c(), p.c(), pairs.c(), grads.c()
    _check(lib().gs_project_bwd(C.byref(gc), _ptr(cams), C.byref(pc), C.byref(qc), C.byref(f), C.byref(cfg),
                                C.byref(rc), _ptr(dL_dpose), _ptr(d_proj), _ptr(ws), ws.numel(), _stream(stream)),
           "gs_project_bwd")


def gs_launch_count() -> int:
    return int(lib().gs_launch_count())


@dataclass
class Spawned:
    """Spawned Gaussians (rows as in Gaussians) plus per-pixel maps."""
    g: Gaussians
    pixel: torch.Tensor
    count: torch.Tensor
    status: torch.Tensor
    p_l: torch.Tensor | None = None
    p_pen: torch.Tensor | None = None
    p_s: torch.Tensor | None = None

    @staticmethod
    def alloc(capacity, hw=None, device="cuda") -> "Spawned":
        maps = [torch.zeros((hw,), dtype=torch.float32, device=device) if hw else None for _ in range(3)]
        return Spawned(Gaussians.zeros(max(capacity, 1), device), torch.zeros((max(capacity, 1),), dtype=torch.int32,
                                                                                 device=device),
                       torch.zeros((1,), dtype=torch.int64, device=device),
                       torch.zeros((1,), dtype=torch.int32, device=device), *maps)

    def c(self, capacity) -> gs_spawn_out:
        return gs_spawn_out(_ptr(self.g.mean_opa), _ptr(self.g.scale), _ptr(self.g.quat), _ptr(self.g.sh),
                            _ptr(self.pixel), capacity, _ptr(self.count), _ptr(self.status), _ptr(self.p_l),
                            _ptr(self.p_pen), _ptr(self.p_s))


def gs_spawn_workspace_size(width: int, height: int) -> int:
    return int(lib().gs_spawn_workspace_size(width, height))


def gs_spawn_propose(image: torch.Tensor, render, depth: torch.Tensor, width: int, height: int, cam: torch.Tensor,
                     sigma: float, seed: int, frame: int, out: Spawned, ws: torch.Tensor, capacity=None, stream=None):
    sc = gs_spawn_config(sigma, frame, seed)
    oc = out.c(out.g.n if capacity is None else capacity)
    _check(lib().gs_spawn_propose(_ptr(image), _ptr(render), _ptr(depth), width, height, _ptr(cam), C.byref(sc),
                                  C.byref(oc), _ptr(ws), ws.numel(), _stream(stream)), "gs_spawn_propose")


def gs_spawn_propose_noalloc(image: torch.Tensor, render, depth: torch.Tensor, width: int, height: int,
                             cam: torch.Tensor, sigma: float, seed: int, frame: int, out: Spawned, capacity=None,
                             stream=None):
    """gs_spawn_propose without a workspace, for callers that cannot allocate
    device memory (the scratch is a fixed array inside the library; frames of
    at most 2,097,152 pixels). Returns the C status code instead of raising so
    callers can react to an oversized frame."""
    sc = gs_spawn_config(sigma, frame, seed)
    oc = out.c(out.g.n if capacity is None else capacity)
    return int(lib().gs_spawn_propose_noalloc(_ptr(image), _ptr(render), _ptr(depth), width, height, _ptr(cam),
                                              C.byref(sc), C.byref(oc), _stream(stream)))


def gs_anchor_check(g: Gaussians, cam: torch.Tensor, tau_px: float, too_fine: torch.Tensor, count: torch.Tensor,
                    stream=None):
    gc = g.c()
    _check(lib().gs_anchor_check(C.byref(gc), _ptr(cam), tau_px, _ptr(too_fine), _ptr(count), _stream(stream)),
           "gs_anchor_check")


def _opt_c(g):
    return None if g is None else C.byref(g.c())


def gs_anchor_offload(params: Gaussians, m, v, host_params: Gaussians, host_m, host_v, stream=None):
    """Device -> host copies of the active set (and its Adam state)."""
    _check(lib().gs_anchor_offload(C.byref(params.c()), _opt_c(m), _opt_c(v), C.byref(host_params.c()),
                                   _opt_c(host_m), _opt_c(host_v), _stream(stream)), "gs_anchor_offload")


def gs_anchor_load(host_params: Gaussians, host_m, host_v, params: Gaussians, m, v, stream=None):
    """Host -> device copies of an anchor's Gaussians (and Adam state)."""
    _check(lib().gs_anchor_load(C.byref(host_params.c()), _opt_c(host_m), _opt_c(host_v), C.byref(params.c()),
                                _opt_c(m), _opt_c(v), _stream(stream)), "gs_anchor_load")


def gs_anchor_merge_workspace_size(n: int, k: int = 3) -> int:
    return int(lib().gs_anchor_merge_workspace_size(n, k))


def gs_anchor_merge(g: Gaussians, too_fine: torch.Tensor, radius: float, seed: int, out: Gaussians,
                    n_out: torch.Tensor, ws: torch.Tensor, k: int = 3, m=None, v=None, m_out=None, v_out=None,
                    lr=None, lr_out=None, stream=None):
    """Merges a random 1/(k+1) of the too-fine Gaussians with their k nearest
    too-fine neighbours into out (n_out: device int64 row count)."""
    a, o = g.c(), out.c()
    cs = [None if t is None else C.byref(t.c()) for t in (m, v, m_out, v_out)]
    _check(lib().gs_anchor_merge(C.byref(a), cs[0], cs[1], _ptr(lr), _ptr(too_fine), radius, k, seed, C.byref(o),
                                 cs[2], cs[3], _ptr(lr_out), _ptr(n_out), _ptr(ws), ws.numel(), _stream(stream)),
           "gs_anchor_merge")


def gs_cull_opacity_workspace_size(n: int) -> int:
    return int(lib().gs_cull_opacity_workspace_size(n))


def gs_cull_opacity(g: Gaussians, min_opacity: float, out: Gaussians, n_out: torch.Tensor, ws: torch.Tensor, m=None,
                    v=None, m_out=None, v_out=None, lr=None, lr_out=None, stream=None):
    """Keeps the Gaussians with opacity >= min_opacity (compacted into out)."""
    a, o = g.c(), out.c()
    cs = [None if t is None else C.byref(t.c()) for t in (m, v, m_out, v_out)]
    _check(lib().gs_cull_opacity(C.byref(a), cs[0], cs[1], _ptr(lr), min_opacity, C.byref(o), cs[2], cs[3],
                                 _ptr(lr_out), _ptr(n_out), _ptr(ws), ws.numel(), _stream(stream)), "gs_cull_opacity")


def gs_anchor_blend_weight(d1: float, d2: float, overlap: float = 0.1) -> float:
    return float(lib().gs_anchor_blend_weight(d1, d2, overlap))


def gs_scale_opacity(mean_opa: torch.Tensor, w: float, stream=None):
    _check(lib().gs_scale_opacity(_ptr(mean_opa), mean_opa.shape[0], w, _stream(stream)), "gs_scale_opacity")


def pinned_gaussians(n: int) -> Gaussians:
    z = lambda k: torch.zeros((n, k), dtype=torch.float32).pin_memory()
    return Gaussians(z(4), z(4), z(4), z(48))


MLP_SHAPES = [("w1", (128, 194)), ("b1", (128,)), ("w2", (128, 128)), ("b2", (128,)), ("w3", (128, 128)),
              ("b3", (128,)), ("w4", (3, 128)), ("b4", (3,))]


@dataclass
class MlpParams:
    """FP32 master parameters of the learned spawn proposal (device tensors)."""
    t: dict

    @staticmethod
    def from_numpy(layers, device="cuda") -> "MlpParams":
        """layers: [(W1, b1), ..., (W4, b4)] in nn.Linear layout."""
        t = {}
        for l, (W, b) in enumerate(layers):
            t[f"w{l + 1}"] = torch.tensor(np.asarray(W, np.float32), device=device)
            t[f"b{l + 1}"] = torch.tensor(np.asarray(b, np.float32), device=device)
        return MlpParams(t)

    @staticmethod
    def zeros(device="cuda") -> "MlpParams":
        return MlpParams({k: torch.zeros(shape, dtype=torch.float32, device=device) for k, shape in MLP_SHAPES})

    def c(self) -> gs_mlp_params:
        return gs_mlp_params(*[_ptr(self.t[k]) for k, _ in MLP_SHAPES])

    def numpy(self):
        return [(self.t[f"w{l}"].cpu().numpy(), self.t[f"b{l}"].cpu().numpy()) for l in range(1, 5)]


def mlp_config(tensor_path=0, w_depth=1.0, w_scale=1.0, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8) -> gs_mlp_config:
    return gs_mlp_config(tensor_path, w_depth, w_scale, lr, beta1, beta2, eps)


def gs_mlp_patches(width: int, height: int) -> int:
    return int(lib().gs_mlp_patches(width, height))


def gs_mlp_param_count() -> int:
    return int(lib().gs_mlp_param_count())


def gs_mlp_workspace_size(n_patches: int) -> int:
    return int(lib().gs_mlp_workspace_size(n_patches))


def gs_mlp_forward(p: MlpParams, image: torch.Tensor, width: int, height: int, out: torch.Tensor,
                   cfg: gs_mlp_config, ws: torch.Tensor, stream=None):
    pc = p.c()
    _check(lib().gs_mlp_forward(C.byref(pc), _ptr(image), width, height, _ptr(out), C.byref(cfg), _ptr(ws),
                                ws.numel(), _stream(stream)), "gs_mlp_forward")


def gs_mlp_train_step(p: MlpParams, m, v, image: torch.Tensor, width: int, height: int, targets: torch.Tensor,
                      cfg: gs_mlp_config, step: int, loss: torch.Tensor, ws: torch.Tensor, out=None, grads=None,
                      step_dev=None, stream=None):
    pc = p.c()
    mc = None if m is None else C.byref(m.c())
    vc = None if v is None else C.byref(v.c())
    _check(lib().gs_mlp_train_step(C.byref(pc), mc, vc, _ptr(image), width, height, _ptr(targets), C.byref(cfg), step,
                                   _ptr(step_dev), _ptr(loss), _ptr(out), _ptr(grads), _ptr(ws), ws.numel(),
                                   _stream(stream)), "gs_mlp_train_step")


def gs_mlp_gemm_bf16(A: torch.Tensor, B: torch.Tensor, C_out: torch.Tensor, tensor_path: int, stream=None):
    """A [M][K], B [N][K] bfloat16 tensors; C_out [M][N] float32."""
    M, K = A.shape
    N = B.shape[0]
    _check(lib().gs_mlp_gemm_bf16(_ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(C_out), C_out.stride(0), M, N, K,
                                  tensor_path, _stream(stream)), "gs_mlp_gemm_bf16")


def gs_mlp_tc_error() -> int:
    v = C.c_int32(0)
    _check(lib().gs_mlp_tc_error(C.byref(v)), "gs_mlp_tc_error")
    return int(v.value)


def gs_mlp_targets(pixel, mean_opa, scale, scale0, cam: torch.Tensor, keep_threshold: float, n_spawn: int,
                   width: int, height: int, targets: torch.Tensor, ws: torch.Tensor, stream=None):
    _check(lib().gs_mlp_targets(_ptr(pixel), _ptr(mean_opa), _ptr(scale), _ptr(scale0), _ptr(cam), keep_threshold,
                                n_spawn, width, height, _ptr(targets), _ptr(ws), ws.numel(), _stream(stream)),
           "gs_mlp_targets")


def gs_mlp_targets_workspace_size(width: int, height: int) -> int:
    return int(lib().gs_mlp_targets_workspace_size(width, height))


def gs_spawn_learned(image: torch.Tensor, mlp_out: torch.Tensor, width: int, height: int, cam: torch.Tensor,
                     seed: int, frame: int, out: Spawned, ws: torch.Tensor, capacity=None, stream=None, depth=None,
                     render=None, sigma: float = 1.0):
    sc = gs_spawn_config(sigma, frame, seed)
    oc = out.c(out.g.n if capacity is None else capacity)
    _check(lib().gs_spawn_learned(_ptr(image), _ptr(mlp_out), _ptr(render), _ptr(depth), width, height, _ptr(cam),
                                  C.byref(sc), C.byref(oc), _ptr(ws), ws.numel(), _stream(stream)),
           "gs_spawn_learned")


def adam_config(lr_mean=1.6e-4, lr_opacity=0.05, lr_scale=5e-3, lr_rot=1e-3, lr_sh_dc=2.5e-3, lr_sh_rest=1.25e-4,
                beta1=0.9, beta2=0.999, eps=1e-15, decay=1.0) -> gs_adam_config:
    return gs_adam_config(lr_mean, lr_opacity, lr_scale, lr_rot, lr_sh_dc, lr_sh_rest, beta1, beta2, eps, decay)


def gs_adam_step(params: Gaussians, grads: Grads, m: Gaussians, v: Gaussians, cfg: gs_adam_config, step: int,
                 stream=None, step_dev: torch.Tensor | None = None, lr_scale: torch.Tensor | None = None):
    a, b, c, d = params.c(), grads.c(), m.c(), v.c()
    _check(lib().gs_adam_step(C.byref(a), C.byref(b), C.byref(c), C.byref(d), C.byref(cfg), step, _ptr(step_dev),
                              _ptr(lr_scale), _stream(stream)), "gs_adam_step")


def gs_pose_step(cams: torch.Tensor, n_views: int, dL_dpose: torch.Tensor, m: torch.Tensor, v: torch.Tensor,
                 lr_t: float, lr_r: float, step: int, beta1=0.9, beta2=0.999, eps=1e-15, stream=None,
                 step_dev: torch.Tensor | None = None):
    _check(lib().gs_pose_step(_ptr(cams), n_views, _ptr(dL_dpose), _ptr(m), _ptr(v), lr_t, lr_r, beta1, beta2, eps,
                              step, _ptr(step_dev), _stream(stream)), "gs_pose_step")


def gs_pose_apply(cams_ref: torch.Tensor, xi: torch.Tensor, n_views: int, cams_out: torch.Tensor, stream=None):
    _check(lib().gs_pose_apply(_ptr(cams_ref), _ptr(xi), n_views, _ptr(cams_out), _stream(stream)), "gs_pose_apply")


def gs_pose_tangent_grad(xi: torch.Tensor, dL_ddelta: torch.Tensor, n_views: int, dL_dxi: torch.Tensor, stream=None):
    _check(lib().gs_pose_tangent_grad(_ptr(xi), _ptr(dL_ddelta), n_views, _ptr(dL_dxi), _stream(stream)),
           "gs_pose_tangent_grad")


def gs_downsample(image: torch.Tensor, width: int, height: int, factor: int, out: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    """Block-mean downsampling of a planar [3][H][W] image by factor."""
    w, h = -(-width // factor), -(-height // factor)
    if out is None:
        out = torch.empty((3 * h * w,), dtype=torch.float32, device=image.device)
    _check(lib().gs_downsample(_ptr(image), width, height, factor, _ptr(out), _stream(stream)), "gs_downsample")
    return out


def downsample_cameras(cams: torch.Tensor, factor: int) -> torch.Tensor:
    """Cameras of factor-downsampled images (intrinsics / factor, sizes rounded up)."""
    cs = cameras_from_tensor(cams)
    for c in cs:
        for k in ("fx", "fy", "cx", "cy"):
            c[k] = c[k] / factor
        c["width"], c["height"] = -(-c["width"] // factor), -(-c["height"] // factor)
    return cameras_tensor(cs, cams.device)


def gs_ba_workspace_size(n_frames: int, n_points: int) -> int:
    return int(lib().gs_ba_workspace_size(n_frames, n_points))


def gs_ba_lm(obs: torch.Tensor, cx: float, cy: float, fl: torch.Tensor, poses: torch.Tensor, points: torch.Tensor,
             lam: torch.Tensor, iterations: int, ws: torch.Tensor, failed: torch.Tensor, huber_delta: float = 2.0,
             nu: float = 2.0, history: torch.Tensor | None = None, stream=None):
    """Levenberg-Marquardt iterations of the mini bundle adjustment (obs
    [P][F][2], poses [F][12], points [P][4], fl and lam [1], all device)."""
    P, F = obs.shape[0], obs.shape[1]
    _check(lib().gs_ba_lm(_ptr(obs), F, P, cx, cy, _ptr(fl), _ptr(poses), _ptr(points), _ptr(lam), iterations,
                          huber_delta, nu, _ptr(history), _ptr(failed), _ptr(ws), ws.numel(), _stream(stream)),
           "gs_ba_lm")


def gs_ba_pose_workspace_size(n_obs: int) -> int:
    return int(lib().gs_ba_pose_workspace_size(n_obs))


def gs_ba_pose_lm(points: torch.Tensor, obs: torch.Tensor, fl: torch.Tensor, cx: float, cy: float,
                  pose: torch.Tensor, lam: torch.Tensor, iterations: int, ws: torch.Tensor, failed: torch.Tensor,
                  huber_delta: float = 2.0, nu: float = 2.0, history: torch.Tensor | None = None, stream=None):
    """Levenberg-Marquardt refinement of one pose [12] from points [M][4] and
    their observations obs [M][2] (all device; points and fl fixed)."""
    _check(lib().gs_ba_pose_lm(_ptr(points), _ptr(obs), obs.shape[0], _ptr(fl), cx, cy, _ptr(pose), _ptr(lam),
                               iterations, huber_delta, nu, _ptr(history), _ptr(failed), _ptr(ws), ws.numel(),
                               _stream(stream)), "gs_ba_pose_lm")


def gs_ba_project(fl: torch.Tensor, poses: torch.Tensor, points: torch.Tensor, cx: float, cy: float,
                  obs: torch.Tensor, stream=None):
    """obs [P][F][2] = pixels of points [P][4] in the F cameras poses [F][12]."""
    _check(lib().gs_ba_project(_ptr(fl), _ptr(poses), _ptr(points), poses.shape[0], points.shape[0], cx, cy,
                               _ptr(obs), _stream(stream)), "gs_ba_project")


def gs_guided_depth(feats: torch.Tensor, cams: torch.Tensor, z_mono: torch.Tensor, n_cand: int = 32,
                    window: float = 0.1, depth: torch.Tensor | None = None, nb: torch.Tensor | None = None,
                    corr: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Refined depth [H][W] of the reference frame from feats [1 + n_nb][H][W][C]
    (bfloat16 bit patterns as int16/uint16, or a bfloat16 tensor), cams (device
    gs_camera array, reference first) and z_mono [H][W]."""
    J1, H, W, Ch = feats.shape
    if depth is None:
        depth = torch.empty((H, W), dtype=torch.float32, device=feats.device)
    _check(lib().gs_guided_depth(_ptr(feats), _ptr(cams), J1 - 1, W, H, Ch, _ptr(z_mono), n_cand, window,
                                 _ptr(depth), _ptr(nb), _ptr(corr), _stream(stream)), "gs_guided_depth")
    return depth


def gs_counter_add(counter: torch.Tensor, delta: int = 1, stream=None):
    _check(lib().gs_counter_add(_ptr(counter), delta, _stream(stream)), "gs_counter_add")


def gs_l1_loss(color: torch.Tensor, target: torch.Tensor, dL_dcolor: torch.Tensor, loss: torch.Tensor,
               ws: torch.Tensor, stream=None):
    _check(lib().gs_l1_loss(_ptr(color), _ptr(target), color.numel(), _ptr(dL_dcolor), _ptr(loss), _ptr(ws),
                            ws.numel(), _stream(stream)), "gs_l1_loss")
