"""Scene partition on the GPU: airspace-aware camera selection (Sec. 4.1) and seamless merging
(Sec. 4.3), through the C ABI of include/vgpartition.h.

* ``airspace_boxes``: each cell's box, x and z over its points, y from the ground plane to the
  highest point.
* ``camera_visibility``: visibility of every cell box in every camera (projected area inside the
  image / image area) and the selection, visibility > threshold (25% in Sec. 5.1).
* ``merge_cells``: each cell keeps the Gaussians inside its original ground rectangle and the
  kept Gaussians of all cells are concatenated into one model, in one pass on the device.
"""
from __future__ import annotations

import ctypes

import torch

from . import binding as B
from .rasterize import _stream, camera_c, gaussians_c

VISIBILITY_THRESHOLD = 0.25


def airspace_boxes(points: torch.Tensor, cell_offsets, ground_y: float) -> torch.Tensor:
    """points: CUDA float32 [N,3], the cells one after another; cell_offsets: host ints [n_cells + 1]."""
    if not (points.is_cuda and points.dtype == torch.float32 and points.is_contiguous()):
        raise ValueError("points must be a contiguous float32 CUDA tensor")
    out = torch.empty((len(cell_offsets) - 1, 6), dtype=torch.float32, device=points.device)
    B.vg_airspace_boxes(points.data_ptr(), cell_offsets, ground_y, out.data_ptr(), _stream())
    return out


def camera_table(cameras):
    """The cameras marshalled once for repeated visibility calls."""
    cams = [camera_c(c) for c in cameras]
    return (B.vg_camera * len(cams))(*cams)


def camera_visibility(boxes: torch.Tensor, cameras, threshold: float = VISIBILITY_THRESHOLD):
    """boxes: CUDA float32 [n_cells, 6]; cameras: scenes.Camera list or a camera_table.  Returns
    (visibility float32 [n_cams, n_cells], selected bool [n_cams, n_cells])."""
    boxes = boxes.contiguous()
    n_cells = int(boxes.shape[0])
    cams = cameras if isinstance(cameras, ctypes.Array) else camera_table(cameras)
    need = B.vg_visibility_workspace_bytes(len(cams))
    ws = torch.empty(need, dtype=torch.uint8, device=boxes.device)
    vis = torch.empty((len(cams), n_cells), dtype=torch.float32, device=boxes.device)
    sel = torch.empty((len(cams), n_cells), dtype=torch.uint8, device=boxes.device)
    B.vg_camera_visibility(boxes.data_ptr(), n_cells, cams, threshold, ws.data_ptr(), need, vis.data_ptr(),
                           sel.data_ptr(), _stream())
    return vis, sel.bool()


def merge_cells(cells, regions, degree: int):
    """cells: list of (means, log_scales, quats, logits, sh) CUDA tensors; regions: list of
    (x0, x1, z0, z1).  Returns the merged parameter tensors (trimmed to the merged count)."""
    gs = [gaussians_c(*c, degree) for c in cells]
    dev = cells[0][0].device
    total = sum(int(c[0].shape[0]) for c in cells)
    need = B.vg_merge_workspace_bytes(gs)
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    k3 = int(cells[0][4].shape[1])
    out = (torch.empty((total, 3), device=dev), torch.empty((total, 3), device=dev),
           torch.empty((total, 4), device=dev), torch.empty((total,), device=dev),
           torch.empty((total, k3, 3), device=dev))
    n = torch.empty((), dtype=torch.int64, device=dev)
    B.vg_merge_cells(gs, regions, ws.data_ptr(), need, *[t.data_ptr() for t in out], n.data_ptr(), _stream())
    m = int(n)
    if m < 0:
        raise RuntimeError("vg_merge_cells: a bounded device wait gave up")
    return tuple(t[:m] for t in out)
