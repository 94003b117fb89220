"""Oracle for the scene-partition kernels (paper Sec. 4.1 and Sec. 4.3), plain NumPy in FP64.

TEST INFRASTRUCTURE ONLY: imported by the tests and by the benchmark's CPU baseline, never by the
product path.  Shares no code with the CUDA kernels.

* ``airspace_box``: the axis-aligned box of a cell's points whose height spans from the ground
  plane to the highest point (Sec. 4.1, airspace-aware visibility).  World frame: +y is up and
  the ground plane is y = ground_y (Sec. 5.1 aligns the y-axis with the ground normal).
* ``visibility``: projected area of a box inside image i divided by the image area (Sec. 4.1,
  visibility-based camera selection): the box is clipped to the half-space in front of the near
  plane, its vertices are projected with the pinhole model, their convex hull is clipped to the
  image rectangle [-1/2, W - 1/2] x [-1/2, H - 1/2] (pixel (i, j) is sampled at (i, j)), and the
  polygon's area is divided by W H.  A camera is selected for a cell when the visibility is
  greater than the threshold (25% in Sec. 5.1).
* ``merge_keep``: a Gaussian survives the merge when its mean lies inside the cell's original,
  unexpanded ground rectangle (Sec. 4.3), read as x0 <= x < x1 and z0 <= z < z1 so that the
  cells of a partition never both keep a Gaussian on their shared edge.

Pins (tests/test_oracle_partition.py): the visibility is checked against ray casting on a fine
grid of image points (the fraction of rays that meet the box in front of the near plane), the
nadir view of a box against its closed form, and the merge filter against the definition.
"""
from __future__ import annotations

import numpy as np

_EDGES = [(0, 1), (2, 3), (4, 5), (6, 7), (0, 2), (1, 3), (4, 6), (5, 7), (0, 4), (1, 5), (2, 6), (3, 7)]


def airspace_box(points: np.ndarray, ground_y: float) -> np.ndarray:
    """[xmin, ymin, zmin, xmax, ymax, zmax] of points [n,3], with ymin = ground_y."""
    p = np.asarray(points, dtype=np.float64)
    lo, hi = p.min(axis=0), p.max(axis=0)
    return np.array([lo[0], ground_y, lo[2], hi[0], hi[1], hi[2]], dtype=np.float64)


def box_corners(box) -> np.ndarray:
    """The 8 corners, corner k = (x[k & 1], y[(k >> 1) & 1], z[(k >> 2) & 1])."""
    b = np.asarray(box, dtype=np.float64)
    xs, ys, zs = (b[0], b[3]), (b[1], b[4]), (b[2], b[5])
    return np.array([[xs[k & 1], ys[(k >> 1) & 1], zs[(k >> 2) & 1]] for k in range(8)])


def _hull(pts: np.ndarray) -> np.ndarray:
    """Convex hull (counter-clockwise) by the monotone chain."""
    P = sorted(map(tuple, pts))
    if len(P) <= 2:
        return np.array(P)

    def cross(o, a, b):
        return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])

    lower, upper = [], []
    for p in P:
        while len(lower) >= 2 and cross(lower[-2], lower[-1], p) <= 0:
            lower.pop()
        lower.append(p)
    for p in reversed(P):
        while len(upper) >= 2 and cross(upper[-2], upper[-1], p) <= 0:
            upper.pop()
        upper.append(p)
    return np.array(lower[:-1] + upper[:-1])


def _clip(poly: np.ndarray, axis: int, bound: float, keep_greater: bool) -> np.ndarray:
    """Sutherland-Hodgman clip of a polygon by one axis-aligned half-plane."""
    out = []
    n = len(poly)
    for k in range(n):
        a, b = poly[k], poly[(k + 1) % n]
        ina = a[axis] >= bound if keep_greater else a[axis] <= bound
        inb = b[axis] >= bound if keep_greater else b[axis] <= bound
        if ina:
            out.append(a)
        if ina != inb:
            t = (bound - a[axis]) / (b[axis] - a[axis])
            out.append(a + t * (b - a))
    return np.array(out)


def _area(poly: np.ndarray) -> float:
    if len(poly) < 3:
        return 0.0
    x, y = poly[:, 0], poly[:, 1]
    return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))


def visibility(box, cam) -> float:
    """Visibility of the box in camera ``cam`` (a scenes.Camera)."""
    Rt = np.asarray(cam.world_to_cam, dtype=np.float64).reshape(3, 4)
    c = box_corners(box) @ Rt[:, :3].T + Rt[:, 3]
    near = float(cam.near)
    front = [p for p in c if p[2] >= near]
    for i, j in _EDGES:
        a, b = c[i], c[j]
        if (a[2] - near) * (b[2] - near) < 0:
            t = (near - a[2]) / (b[2] - a[2])
            front.append(a + t * (b - a))
    if not front:
        return 0.0
    f = np.array(front)
    uv = np.stack([cam.fx * f[:, 0] / f[:, 2] + cam.cx, cam.fy * f[:, 1] / f[:, 2] + cam.cy], axis=1)
    poly = _hull(uv)
    if len(poly) < 3:
        return 0.0
    for axis, bound, keep in ((0, -0.5, True), (0, cam.width - 0.5, False), (1, -0.5, True), (1, cam.height - 0.5, False)):
        poly = _clip(poly, axis, bound, keep)
        if len(poly) < 3:
            return 0.0
    return _area(poly) / (cam.width * cam.height)


def visibility_matrix(boxes, cams) -> np.ndarray:
    """[n_cams, n_cells] visibilities."""
    return np.array([[visibility(b, c) for b in boxes] for c in cams])


def select(vis: np.ndarray, threshold: float = 0.25) -> np.ndarray:
    """Cameras selected for each cell: visibility greater than the threshold."""
    return vis > threshold


def merge_keep(means: np.ndarray, region) -> np.ndarray:
    """Boolean mask of the Gaussians kept by a cell with ground rectangle (x0, x1, z0, z1)."""
    m = np.asarray(means, dtype=np.float64)
    x0, x1, z0, z1 = (float(v) for v in region)
    return (m[:, 0] >= x0) & (m[:, 0] < x1) & (m[:, 2] >= z0) & (m[:, 2] < z1)


def merge(cells, regions):
    """Concatenation, in cell order, of the kept Gaussians of every cell (index order inside a
    cell): returns the list of (cell, index) pairs."""
    out = []
    for k, (g, r) in enumerate(zip(cells, regions)):
        idx = np.nonzero(merge_keep(g, r))[0]
        out.extend((k, int(i)) for i in idx)
    return out
