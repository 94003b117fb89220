"""The C-ABI library: it builds, loads, exports every symbol include/*.h declares, and
rejects invalid arguments on the host (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def vg():
    from paper_2402_17427_gb300 import _build, binding
    _build.build()
    return binding


def declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b(vg_[a-z0-9_]+)\s*\(", txt, flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("vg_rasterize_forward", "vg_rasterize_backward", "vg_render_batch", "vg_render_batch_backward",
                 "vg_loss_l1_dssim", "vg_workspace_bytes", "vg_read_render_state", "vg_airspace_boxes",
                 "vg_camera_visibility", "vg_merge_cells"):
        assert must in names


def test_library_exports_every_declared_symbol(vg):
    L = ctypes.CDLL(vg.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert set(vg.EXPORTED) <= set(declared_functions())


def test_default_options_are_the_method_constants(vg):
    o = vg.vg_default_opts()
    assert o.tile_size == 16 and o.stop_rule == 0
    assert abs(o.dilation - 0.3) < 1e-7 and abs(o.alpha_max - 0.99) < 1e-7
    assert abs(o.alpha_min - 1 / 255) < 1e-9 and abs(o.t_min - 1e-4) < 1e-11
    assert list(o.bg) == [0.0, 0.0, 0.0]


def test_workspace_sizes(vg):
    o = vg.vg_default_opts()
    a = vg.vg_workspace_bytes(1000, 128, 128, 4096, o)
    b = vg.vg_workspace_bytes(2000, 128, 128, 4096, o)
    c = vg.vg_workspace_bytes(1000, 128, 128, 8192, o)
    assert 0 < a < b and a < c
    assert vg.vg_workspace_bytes(-1, 128, 128, 4096, o) == 0
    assert vg.vg_workspace_bytes(10, 0, 128, 4096, o) == 0
    assert vg.vg_workspace_bytes(10, 128, 128, 0, o) == 0
    o.tile_size = 12
    assert vg.vg_workspace_bytes(10, 128, 128, 4096, o) == 0
    assert vg.vg_loss_workspace_bytes(100, 50) > 9 * 100 * 50 * 4 - 1
    assert vg.vg_loss_workspace_bytes(0, 50) == 0


def test_invalid_arguments_rejected_before_any_launch(vg):
    o = vg.vg_default_opts()
    cam = vg.vg_camera()
    cam.width, cam.height, cam.fx, cam.fy, cam.near_plane = 64, 64, 50.0, 50.0, 0.2
    g = vg.vg_gaussians()
    g.n, g.sh_degree = 0, 0
    L = vg.lib()
    # null workspace / outputs
    st = L.vg_rasterize_forward(ctypes.byref(g), ctypes.byref(cam), ctypes.byref(o), None, 0, 16, None, None, None,
                                None, None)
    assert st == vg.VG_ERR_INVALID
    # bad degree
    g.sh_degree = 4
    st = L.vg_rasterize_forward(ctypes.byref(g), ctypes.byref(cam), ctypes.byref(o), 256, 1 << 20, 16, 256, 256,
                                256, 256, None)
    assert st == vg.VG_ERR_INVALID
    g.sh_degree = 0
    # non-positive focal length
    cam.fx = 0.0
    st = L.vg_rasterize_forward(ctypes.byref(g), ctypes.byref(cam), ctypes.byref(o), 256, 1 << 20, 16, 256, 256,
                                256, 256, None)
    assert st == vg.VG_ERR_INVALID
    cam.fx = 50.0
    # workspace too small
    st = L.vg_rasterize_forward(ctypes.byref(g), ctypes.byref(cam), ctypes.byref(o), 256, 16, 16, 256, 256, 256,
                                256, None)
    assert st == vg.VG_ERR_CAPACITY
    # misaligned quaternion array
    g.n, g.means, g.log_scales, g.quats, g.opacity_logits, g.sh = 4, 256, 256, 260, 256, 256
    st = L.vg_rasterize_forward(ctypes.byref(g), ctypes.byref(cam), ctypes.byref(o), 256, 1 << 20, 16, 256, 256,
                                256, 256, None)
    assert st == vg.VG_ERR_INVALID
    assert L.vg_loss_l1_dssim(None, None, 10, 10, 0.2, None, 0, None, None, None) == vg.VG_ERR_INVALID
    assert L.vg_approx_probe(2, 256, 256, 4, None) == vg.VG_ERR_INVALID
    assert L.vg_approx_probe(0, None, None, 4, None) == vg.VG_ERR_INVALID
    assert L.vg_approx_probe(0, None, None, 0, None) == vg.VG_OK
    assert vg.status_string(vg.VG_ERR_CAPACITY) == "workspace too small"


def test_product_path_has_no_oracle_dependency():
    pkg = os.path.join(ROOT, "paper_2402_17427_gb300")
    for root, _dirs, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(root, f)).read()
                assert "import oracle" not in src and "from oracle" not in src and "vg_oracle" not in src, f
