"""The C-ABI library builds, loads and exports every symbol include/gs.h
declares; the Python structs match the C layout (CPU only, no kernel calls)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:int|void|size_t|int64_t|float)\s+\**\s*(gs_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def built():
    from paper_2506_05558_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("gs_project", "gs_sort", "gs_render_fwd", "gs_render_bwd", "gs_adam_step"):
        assert n in names


def test_library_exports_every_declared_symbol(built):
    lib = C.CDLL(built)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol(built):
    from paper_2506_05558_gb300 import gs
    assert sorted(gs.EXPORTS) == declared_functions()


def test_struct_layouts_and_host_helpers(built):
    from paper_2506_05558_gb300 import gs
    assert C.sizeof(gs.gs_camera) == 72
    c = gs.config()
    assert c.tile == 16 and abs(c.alpha_min - 1 / 255) < 1e-9 and c.sh_degree == 3
    f = gs.frame([(64, 48), (33, 17)])
    assert f.n_views == 2 and f.tiles_x[0] == 4 and f.tiles_y[0] == 3 and f.tiles_x[1] == 3 and f.tiles_y[1] == 2
    assert f.tile_base[1] == 12 and f.tile_base[2] == 18 and f.pix_base[1] == 64 * 48 and f.pix_base[2] == 64 * 48 + 33 * 17
    with pytest.raises(RuntimeError):
        gs.frame([(0, 10)])
    with pytest.raises(RuntimeError):
        gs.frame([(10, 10)] * 65)


def test_invalid_arguments_rejected_on_host(built):
    """Host-side argument checks return GS_ERR_INVALID_ARG without touching the GPU."""
    from paper_2506_05558_gb300 import gs
    L = gs.lib()
    f = gs.frame([(64, 64)])
    cfg = gs.config()
    g = gs.gs_gaussians(None, None, None, None, 10)
    p = gs.gs_projected(None, None, None, None, None)
    assert L.gs_project(C.byref(g), None, C.byref(f), C.byref(cfg), C.byref(p), None) == gs.GS_ERR_INVALID_ARG
    cfg.sh_degree = 4
    assert L.gs_project(C.byref(g), 1, C.byref(f), C.byref(cfg), C.byref(p), None) == gs.GS_ERR_INVALID_ARG
    pairs = gs.gs_pairs(None, None, None, None, 100, None, None)
    assert L.gs_sort(C.byref(p), 10, C.byref(f), C.byref(pairs), None, 0, None) == gs.GS_ERR_INVALID_ARG
    assert L.gs_l1_loss(None, None, 0, None, None, None, 0, None) == gs.GS_ERR_INVALID_ARG
    assert gs.gs_sort_workspace_size(1000, f, 5000) > 0
    assert gs.gs_backward_workspace_size(1000, f, 5000) > 5000 * 36
