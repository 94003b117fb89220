"""ctypes binding of libvgrast.so: the C ABI of ``include/vgrast.h`` with the same names.

Argument marshalling only.  Every entry point takes raw device pointers (Python ints) and a
CUDA stream handle; all computation happens in the library's CUDA kernels.  There is no CPU
fallback: if the library cannot be loaded, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libvgrast.so")

VG_OK, VG_ERR_INVALID, VG_ERR_CAPACITY, VG_ERR_CUDA, VG_ERR_TIMEOUT, VG_ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5
VG_STATUS_PAIR_OVERFLOW = 1
VG_STATUS_WAIT_TIMEOUT = 2
(VG_CNT_PAIRS, VG_CNT_VISIBLE, VG_CNT_STATUS, VG_CNT_DEPTH_BITS, VG_CNT_EVALS, VG_CNT_BLENDS, VG_CNT_EVALS_RUN,
 VG_CNT_EVALS_RUN_BWD) = range(8)
VG_CNT_LEN = 8
VG_FLAG_ACCUMULATE_GRADS = 1
VG_FLAG_COUNT_BLENDS = 2
VG_FLAG_TEST_STALL_LOOKBACK = 4

EXPORTED = ("vg_default_opts", "vg_status_string", "vg_kernel_launches", "vg_workspace_bytes", "vg_rasterize_forward",
            "vg_rasterize_backward", "vg_read_render_state", "vg_loss_workspace_bytes", "vg_loss_l1_dssim",
            "vg_batch_workspace_bytes", "vg_render_batch", "vg_render_batch_backward",
            "vg_views_workspace_bytes", "vg_render_views", "vg_loss_l1_dssim_noalloc", "vg_read_batch_state",
            "vg_loss_l1_dssim_grad", "vg_read_counters", "vg_alu_probe", "vg_approx_probe",
            "vg_airspace_boxes", "vg_visibility_workspace_bytes", "vg_camera_visibility", "vg_merge_workspace_bytes",
            "vg_merge_cells", "vg_eval_workspace_bytes", "vg_eval_color_corrected", "vg_adam_step",
            "vg_densify_accumulate", "vg_densify_workspace_bytes", "vg_densify", "vg_appearance_param_count",
            "vg_appearance_workspace_bytes", "vg_appearance_loss")
VG_LOSS_NOALLOC_MAX_PIXELS = 1024 * 1024


class vg_param_ptrs(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacity_logits", ctypes.c_void_p), ("sh", ctypes.c_void_p)]


class vg_adam_opts(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float * 6), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("step", ctypes.c_int32)]


class vg_densify_opts(ctypes.Structure):
    _fields_ = [("grad_threshold", ctypes.c_float), ("percent_dense", ctypes.c_float),
                ("scene_extent", ctypes.c_float), ("min_opacity", ctypes.c_float), ("max_world_scale", ctypes.c_float)]


class vg_camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("world_to_cam", ctypes.c_float * 12), ("cam_pos", ctypes.c_float * 3),
                ("near_plane", ctypes.c_float)]


class vg_gaussians(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacity_logits", ctypes.c_void_p), ("sh", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32), ("reserved", ctypes.c_int32)]


VG_STAGE_PROJECT, VG_STAGE_SORT, VG_STAGE_BLEND, VG_STAGE_BLEND_BACKWARD, VG_STAGE_PROJECT_BACKWARD = range(5)
VG_STAGE_COUNT = 5


class vg_stage_events(ctypes.Structure):
    _fields_ = [("begin", ctypes.c_void_p * VG_STAGE_COUNT), ("end", ctypes.c_void_p * VG_STAGE_COUNT)]


class vg_raster_opts(ctypes.Structure):
    _fields_ = [("tile_size", ctypes.c_int32), ("chunk", ctypes.c_int32), ("bg", ctypes.c_float * 3),
                ("dilation", ctypes.c_float), ("alpha_max", ctypes.c_float), ("alpha_min", ctypes.c_float),
                ("t_min", ctypes.c_float), ("guard", ctypes.c_float), ("stop_rule", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("events", ctypes.POINTER(vg_stage_events)),
                ("key_inputs", ctypes.c_void_p)]


class VGError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


_lib = None
_P = ctypes.c_void_p
_PP = ctypes.POINTER(ctypes.c_void_p)


def lib():
    """Loads libvgrast.so (built by ``paper_2402_17427_gb300._build``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2402_17427_gb300._build.build()")
    L = ctypes.CDLL(LIB_PATH)
    L.vg_default_opts.argtypes = [ctypes.POINTER(vg_raster_opts)]
    L.vg_default_opts.restype = None
    L.vg_status_string.argtypes = [ctypes.c_int]
    L.vg_status_string.restype = ctypes.c_char_p
    L.vg_kernel_launches.argtypes = []
    L.vg_kernel_launches.restype = ctypes.c_uint64
    L.vg_workspace_bytes.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                     ctypes.POINTER(vg_raster_opts)]
    L.vg_workspace_bytes.restype = ctypes.c_size_t
    L.vg_rasterize_forward.argtypes = [ctypes.POINTER(vg_gaussians), ctypes.POINTER(vg_camera),
                                       ctypes.POINTER(vg_raster_opts), _P, ctypes.c_size_t, ctypes.c_int64,
                                       _P, _P, _P, _P, _P]
    L.vg_rasterize_forward.restype = ctypes.c_int
    L.vg_rasterize_backward.argtypes = [ctypes.POINTER(vg_gaussians), ctypes.POINTER(vg_camera),
                                        ctypes.POINTER(vg_raster_opts), _P, ctypes.c_size_t, ctypes.c_int64,
                                        _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]
    L.vg_rasterize_backward.restype = ctypes.c_int
    L.vg_read_render_state.argtypes = [_P, ctypes.c_size_t, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int64, ctypes.POINTER(vg_raster_opts), _P, _P, _P, _P, _P]
    L.vg_read_render_state.restype = ctypes.c_int
    L.vg_loss_workspace_bytes.argtypes = [ctypes.c_int32, ctypes.c_int32]
    L.vg_loss_workspace_bytes.restype = ctypes.c_size_t
    L.vg_loss_l1_dssim.argtypes = [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, _P, ctypes.c_size_t,
                                   _P, _P, _P]
    L.vg_loss_l1_dssim.restype = ctypes.c_int
    L.vg_loss_l1_dssim_grad.argtypes = [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, _P, ctypes.c_size_t,
                                        _P, _P, _P]
    L.vg_loss_l1_dssim_grad.restype = ctypes.c_int
    L.vg_read_counters.argtypes = [_P, ctypes.c_size_t, _P, _P]
    L.vg_read_counters.restype = ctypes.c_int
    L.vg_alu_probe.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P]
    L.vg_alu_probe.restype = ctypes.c_int
    L.vg_approx_probe.argtypes = [ctypes.c_int32, _P, _P, ctypes.c_int32, _P]
    L.vg_approx_probe.restype = ctypes.c_int
    if hasattr(L, "vg_render_batch"):
        L.vg_batch_workspace_bytes.argtypes = [ctypes.POINTER(vg_gaussians), ctypes.c_int32,
                                               ctypes.POINTER(vg_camera), ctypes.POINTER(vg_raster_opts),
                                               ctypes.c_int64]
        L.vg_batch_workspace_bytes.restype = ctypes.c_size_t
        L.vg_render_batch.argtypes = [ctypes.POINTER(vg_gaussians), ctypes.c_int32, ctypes.POINTER(vg_camera),
                                      ctypes.POINTER(vg_raster_opts), _P, ctypes.c_size_t, ctypes.c_int64,
                                      _PP, _PP, _PP, _P, _P]
        L.vg_render_batch.restype = ctypes.c_int
        L.vg_read_batch_state.argtypes = [_P, ctypes.c_size_t, ctypes.POINTER(vg_gaussians), ctypes.c_int32,
                                          ctypes.POINTER(vg_camera), ctypes.POINTER(vg_raster_opts), ctypes.c_int64,
                                          _P, _P, _P, _P, _P]
        L.vg_read_batch_state.restype = ctypes.c_int
        L.vg_render_batch_backward.argtypes = [ctypes.POINTER(vg_gaussians), ctypes.c_int32,
                                               ctypes.POINTER(vg_camera), ctypes.POINTER(vg_raster_opts), _P,
                                               ctypes.c_size_t, ctypes.c_int64, _PP, _PP, _PP, _PP, _PP, _PP,
                                               _PP, _PP, _P]
        L.vg_render_batch_backward.restype = ctypes.c_int
    L.vg_loss_l1_dssim_noalloc.argtypes = [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, _P, _P, _P]
    L.vg_loss_l1_dssim_noalloc.restype = ctypes.c_int
    L.vg_views_workspace_bytes.argtypes = [ctypes.POINTER(vg_gaussians), ctypes.c_int32, _P,
                                           ctypes.POINTER(vg_camera), ctypes.POINTER(vg_raster_opts), ctypes.c_int32,
                                           ctypes.c_int64]
    L.vg_views_workspace_bytes.restype = ctypes.c_size_t
    L.vg_render_views.argtypes = [ctypes.POINTER(vg_gaussians), ctypes.c_int32, _P, ctypes.POINTER(vg_camera),
                                  ctypes.POINTER(vg_raster_opts), ctypes.c_int32, _P, ctypes.c_size_t,
                                  ctypes.c_int64, _PP, _PP, _PP, _P, _P, _P]
    L.vg_render_views.restype = ctypes.c_int
    L.vg_airspace_boxes.argtypes = [_P, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32, ctypes.c_float, _P, _P]
    L.vg_airspace_boxes.restype = ctypes.c_int
    L.vg_visibility_workspace_bytes.argtypes = [ctypes.c_int32]
    L.vg_visibility_workspace_bytes.restype = ctypes.c_size_t
    L.vg_camera_visibility.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(vg_camera), ctypes.c_int32, ctypes.c_float,
                                       _P, ctypes.c_size_t, _P, _P, _P]
    L.vg_camera_visibility.restype = ctypes.c_int
    L.vg_merge_workspace_bytes.argtypes = [ctypes.POINTER(vg_gaussians), ctypes.c_int32]
    L.vg_merge_workspace_bytes.restype = ctypes.c_size_t
    L.vg_merge_cells.argtypes = [ctypes.POINTER(vg_gaussians), ctypes.POINTER(ctypes.c_float), ctypes.c_int32, _P,
                                 ctypes.c_size_t, _P, _P, _P, _P, _P, _P, _P]
    L.vg_merge_cells.restype = ctypes.c_int
    L.vg_eval_workspace_bytes.argtypes = [ctypes.c_int32, ctypes.c_int32]
    L.vg_eval_workspace_bytes.restype = ctypes.c_size_t
    L.vg_eval_color_corrected.argtypes = [_P, _P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_size_t, _P, _P]
    L.vg_eval_color_corrected.restype = ctypes.c_int
    L.vg_adam_step.argtypes = [vg_param_ptrs, ctypes.POINTER(vg_gaussians), vg_param_ptrs, vg_param_ptrs,
                               ctypes.POINTER(vg_adam_opts), _P]
    L.vg_adam_step.restype = ctypes.c_int
    L.vg_densify_accumulate.argtypes = [_P, ctypes.c_size_t, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int64, ctypes.POINTER(vg_raster_opts), _P, _P, _P]
    L.vg_densify_accumulate.restype = ctypes.c_int
    L.vg_densify_workspace_bytes.argtypes = [ctypes.c_int64]
    L.vg_densify_workspace_bytes.restype = ctypes.c_size_t
    L.vg_densify.argtypes = [ctypes.POINTER(vg_gaussians), ctypes.POINTER(vg_gaussians), ctypes.POINTER(vg_gaussians),
                             _P, _P, _P, ctypes.POINTER(vg_densify_opts), _P, ctypes.c_size_t, vg_param_ptrs,
                             vg_param_ptrs, vg_param_ptrs, _P, _P]
    L.vg_densify.restype = ctypes.c_int
    L.vg_appearance_param_count.argtypes = []
    L.vg_appearance_param_count.restype = ctypes.c_int64
    L.vg_appearance_workspace_bytes.argtypes = [ctypes.c_int32, ctypes.c_int32]
    L.vg_appearance_workspace_bytes.restype = ctypes.c_size_t
    L.vg_appearance_loss.argtypes = [_P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P, ctypes.c_float, _P,
                                     ctypes.c_size_t, _P, _P, _P, _P, _P, _P]
    L.vg_appearance_loss.restype = ctypes.c_int
    _lib = L
    return L


def status_string(status: int) -> str:
    try:
        return lib().vg_status_string(int(status)).decode()
    except Exception:  # the library itself may be what is missing
        return "status"


def _check(status: int, where: str):
    if status != VG_OK:
        raise VGError(status, where)


def vg_kernel_launches() -> int:
    return int(lib().vg_kernel_launches())


def vg_default_opts() -> vg_raster_opts:
    o = vg_raster_opts()
    lib().vg_default_opts(ctypes.byref(o))
    return o


def vg_workspace_bytes(n: int, width: int, height: int, pair_capacity: int, opts: vg_raster_opts) -> int:
    return int(lib().vg_workspace_bytes(n, width, height, pair_capacity, ctypes.byref(opts)))


def vg_rasterize_forward(g: vg_gaussians, cam: vg_camera, opts: vg_raster_opts, workspace: int, workspace_bytes: int,
                         pair_capacity: int, out_rgb: int, out_final_T: int, out_last: int, counters: int,
                         stream: int) -> None:
    _check(lib().vg_rasterize_forward(ctypes.byref(g), ctypes.byref(cam), ctypes.byref(opts), workspace,
                                      workspace_bytes, pair_capacity, out_rgb, out_final_T, out_last, counters,
                                      stream), "vg_rasterize_forward")


def vg_rasterize_backward(g: vg_gaussians, cam: vg_camera, opts: vg_raster_opts, workspace: int,
                          workspace_bytes: int, pair_capacity: int, out_final_T: int, out_last: int, dL_drgb: int,
                          g_means: int, g_log_scales: int, g_quats: int, g_opacity_logits: int, g_sh: int,
                          g_means2d_abs: int | None, stream: int) -> None:
    _check(lib().vg_rasterize_backward(ctypes.byref(g), ctypes.byref(cam), ctypes.byref(opts), workspace,
                                       workspace_bytes, pair_capacity, out_final_T, out_last, dL_drgb, g_means,
                                       g_log_scales, g_quats, g_opacity_logits, g_sh, g_means2d_abs, stream),
           "vg_rasterize_backward")


def vg_read_render_state(workspace: int, workspace_bytes: int, n: int, width: int, height: int, pair_capacity: int,
                         opts: vg_raster_opts, ranges: int | None, ids: int | None, projected: int | None,
                         touched: int | None, stream: int) -> None:
    _check(lib().vg_read_render_state(workspace, workspace_bytes, n, width, height, pair_capacity, ctypes.byref(opts),
                                      ranges, ids, projected, touched, stream), "vg_read_render_state")


def vg_loss_workspace_bytes(width: int, height: int) -> int:
    return int(lib().vg_loss_workspace_bytes(width, height))


def vg_loss_l1_dssim(img: int, target: int, width: int, height: int, lam: float, workspace: int,
                     workspace_bytes: int, out_loss: int, out_grad: int | None, stream: int) -> None:
    _check(lib().vg_loss_l1_dssim(img, target, width, height, lam, workspace, workspace_bytes, out_loss, out_grad,
                                  stream), "vg_loss_l1_dssim")


def vg_read_counters(workspace: int, workspace_bytes: int, counters: int, stream: int) -> None:
    _check(lib().vg_read_counters(workspace, workspace_bytes, counters, stream), "vg_read_counters")


def vg_alu_probe(kind: int, blocks: int, iters: int, scratch: int, stream: int) -> None:
    _check(lib().vg_alu_probe(kind, blocks, iters, scratch, stream), "vg_alu_probe")


def vg_approx_probe(kind: int, inp: int, out: int, n: int, stream: int) -> None:
    _check(lib().vg_approx_probe(kind, inp, out, n, stream), "vg_approx_probe")


def vg_loss_l1_dssim_grad(img: int, target: int, width: int, height: int, lam: float, workspace: int,
                          workspace_bytes: int, scale: int | None, out_grad: int, stream: int) -> None:
    _check(lib().vg_loss_l1_dssim_grad(img, target, width, height, lam, workspace, workspace_bytes, scale, out_grad,
                                       stream), "vg_loss_l1_dssim_grad")


def _ptr_array(ptrs):
    arr = (ctypes.c_void_p * len(ptrs))(*[p or None for p in ptrs])
    return ctypes.cast(arr, _PP), arr


def vg_batch_workspace_bytes(cells, cams, opts, pair_capacity: int) -> int:
    n = len(cells)
    G = (vg_gaussians * n)(*cells)
    C = (vg_camera * n)(*cams)
    O = (vg_raster_opts * n)(*opts)
    return int(lib().vg_batch_workspace_bytes(G, n, C, O, pair_capacity))


def vg_render_batch(cells, cams, opts, workspace: int, workspace_bytes: int, pair_capacity: int, out_rgb, out_final_T,
                    out_last, counters: int, stream: int) -> None:
    n = len(cells)
    G = (vg_gaussians * n)(*cells)
    C = (vg_camera * n)(*cams)
    O = (vg_raster_opts * n)(*opts)
    a, _ka = _ptr_array(out_rgb)
    b, _kb = _ptr_array(out_final_T)
    c, _kc = _ptr_array(out_last)
    _check(lib().vg_render_batch(G, n, C, O, workspace, workspace_bytes, pair_capacity, a, b, c, counters, stream),
           "vg_render_batch")


def vg_read_batch_state(workspace: int, workspace_bytes: int, cells, cams, opts, pair_capacity: int,
                        ranges: int | None, ids: int | None, projected: int | None, touched: int | None,
                        stream: int) -> None:
    n = len(cells)
    G = (vg_gaussians * n)(*cells)
    C = (vg_camera * n)(*cams)
    O = (vg_raster_opts * n)(*opts)
    _check(lib().vg_read_batch_state(workspace, workspace_bytes, G, n, C, O, pair_capacity, ranges, ids, projected,
                                     touched, stream), "vg_read_batch_state")


def vg_render_batch_backward(cells, cams, opts, workspace: int, workspace_bytes: int, pair_capacity: int,
                             out_final_T, out_last, dL_drgb, g_means, g_log_scales, g_quats, g_opacity_logits, g_sh,
                             stream: int) -> None:
    n = len(cells)
    G = (vg_gaussians * n)(*cells)
    C = (vg_camera * n)(*cams)
    O = (vg_raster_opts * n)(*opts)
    keep = []
    arrs = []
    for lst in (out_final_T, out_last, dL_drgb, g_means, g_log_scales, g_quats, g_opacity_logits, g_sh):
        p, k = _ptr_array(lst)
        arrs.append(p)
        keep.append(k)
    _check(lib().vg_render_batch_backward(G, n, C, O, workspace, workspace_bytes, pair_capacity, *arrs, stream),
           "vg_render_batch_backward")


def vg_views_workspace_bytes(cells, aabbs, cams, opts, pair_capacity: int) -> int:
    """aabbs: None or a C float array / numpy float32 [n_cells, 6] kept alive by the caller."""
    n, nv = len(cells), len(cams)
    G = (vg_gaussians * n)(*cells)
    C = (vg_camera * nv)(*cams)
    O = (vg_raster_opts * nv)(*opts)
    ab = None if aabbs is None else aabbs.ctypes.data
    return int(lib().vg_views_workspace_bytes(G, n, ab, C, O, nv, pair_capacity))


def vg_render_views(cells, aabbs, cams, opts, workspace: int, workspace_bytes: int, pair_capacity: int, out_rgb,
                    out_final_T, out_last, counters: int, stream: int):
    """Returns the number of cells rendered in each view."""
    n, nv = len(cells), len(cams)
    G = (vg_gaussians * n)(*cells)
    C = (vg_camera * nv)(*cams)
    O = (vg_raster_opts * nv)(*opts)
    ab = None if aabbs is None else aabbs.ctypes.data
    kept = (ctypes.c_int32 * nv)()
    a, _ka = _ptr_array(out_rgb)
    b, _kb = _ptr_array(out_final_T)
    c, _kc = _ptr_array(out_last)
    _check(lib().vg_render_views(G, n, ab, C, O, nv, workspace, workspace_bytes, pair_capacity, a, b, c, kept,
                                 counters, stream), "vg_render_views")
    return list(kept)


def vg_loss_l1_dssim_noalloc(img: int, target: int, width: int, height: int, lam: float, out_loss: int,
                             out_grad: int | None, stream: int) -> None:
    """Eq. 1 loss without a caller workspace (scratch compiled into the library; see vgrast.h)."""
    _check(lib().vg_loss_l1_dssim_noalloc(img, target, width, height, lam, out_loss, out_grad, stream),
           "vg_loss_l1_dssim_noalloc")


# ------------------------------------------------------------------ scene partition (vgpartition.h)

def vg_airspace_boxes(points: int, cell_offsets, ground_y: float, out_boxes: int, stream: int) -> None:
    """Airspace box of each cell; cell_offsets is a host sequence of n_cells + 1 int64."""
    n = len(cell_offsets) - 1
    off = (ctypes.c_int64 * (n + 1))(*[int(v) for v in cell_offsets])
    _check(lib().vg_airspace_boxes(points, off, n, ground_y, out_boxes, stream), "vg_airspace_boxes")


def vg_visibility_workspace_bytes(n_cams: int) -> int:
    return int(lib().vg_visibility_workspace_bytes(n_cams))


def vg_camera_visibility(boxes: int, n_cells: int, cams, threshold: float, workspace: int, workspace_bytes: int,
                         out_visibility: int | None, out_selected: int | None, stream: int) -> None:
    n = len(cams)
    C = cams if isinstance(cams, ctypes.Array) else (vg_camera * n)(*cams)
    _check(lib().vg_camera_visibility(boxes, n_cells, C, n, threshold, workspace, workspace_bytes, out_visibility,
                                      out_selected, stream), "vg_camera_visibility")


def vg_merge_workspace_bytes(cells) -> int:
    n = len(cells)
    G = (vg_gaussians * n)(*cells)
    return int(lib().vg_merge_workspace_bytes(G, n))


def vg_merge_cells(cells, regions, workspace: int, workspace_bytes: int, out_means: int, out_log_scales: int,
                   out_quats: int, out_logits: int, out_sh: int, out_n: int, stream: int) -> None:
    n = len(cells)
    G = (vg_gaussians * n)(*cells)
    R = (ctypes.c_float * (4 * n))(*[float(v) for r in regions for v in r])
    _check(lib().vg_merge_cells(G, R, n, workspace, workspace_bytes, out_means, out_log_scales, out_quats, out_logits,
                                out_sh, out_n, stream), "vg_merge_cells")


# ------------------------------------------------------------------ evaluation (Sec. 5.1 metrics)

def vg_eval_workspace_bytes(width: int, height: int) -> int:
    return int(lib().vg_eval_workspace_bytes(width, height))


def vg_eval_color_corrected(img: int, target: int, width: int, height: int, workspace: int, workspace_bytes: int,
                            out: int, stream: int) -> None:
    _check(lib().vg_eval_color_corrected(img, target, width, height, workspace, workspace_bytes, out, stream),
           "vg_eval_color_corrected")


# ------------------------------------------------------------------ optimiser step (vgoptim.h)

def vg_adam_step(params: vg_param_ptrs, grads: vg_gaussians, m: vg_param_ptrs, v: vg_param_ptrs,
                 opts: vg_adam_opts, stream: int) -> None:
    _check(lib().vg_adam_step(params, ctypes.byref(grads), m, v, ctypes.byref(opts), stream), "vg_adam_step")


def vg_densify_accumulate(workspace: int, workspace_bytes: int, n: int, width: int, height: int, pair_capacity: int,
                          opts: vg_raster_opts, accum: int, count: int, stream: int) -> None:
    _check(lib().vg_densify_accumulate(workspace, workspace_bytes, n, width, height, pair_capacity, ctypes.byref(opts),
                                       accum, count, stream), "vg_densify_accumulate")


def vg_densify_workspace_bytes(n: int) -> int:
    return int(lib().vg_densify_workspace_bytes(n))


def vg_densify(inp: vg_gaussians, m_in: vg_gaussians, v_in: vg_gaussians, accum: int, count: int, normals: int,
               opts: vg_densify_opts, workspace: int, workspace_bytes: int, out: vg_param_ptrs, m_out: vg_param_ptrs,
               v_out: vg_param_ptrs, out_n: int, stream: int) -> None:
    _check(lib().vg_densify(ctypes.byref(inp), ctypes.byref(m_in), ctypes.byref(v_in), accum, count, normals,
                            ctypes.byref(opts), workspace, workspace_bytes, out, m_out, v_out, out_n, stream),
           "vg_densify")


# ------------------------------------------------------------------ appearance model (vgappearance.h)

def vg_appearance_param_count() -> int:
    return int(lib().vg_appearance_param_count())


def vg_appearance_workspace_bytes(width: int, height: int) -> int:
    return int(lib().vg_appearance_workspace_bytes(width, height))


def vg_appearance_loss(img: int, target: int, width: int, height: int, embedding: int, params: int, lam: float,
                       workspace: int, workspace_bytes: int, out_loss: int, out_map: int, grad_img: int,
                       grad_embedding: int, grad_params: int, stream: int) -> None:
    _check(lib().vg_appearance_loss(img, target, width, height, embedding, params, lam, workspace, workspace_bytes,
                                    out_loss, out_map, grad_img, grad_embedding, grad_params, stream),
           "vg_appearance_loss")
