"""Pins of the partition oracle (paper Sec. 4.1 visibility-based camera selection, Sec. 4.3 merging).

The visibility (projected box area inside the image / image area) is checked against an
independent ray caster: the fraction of a fine grid of image points whose viewing ray meets the
box at a depth >= the near plane.  A nadir view of a box is checked against its closed form, and
the merge filter against its definition on points placed on the cell edges.
"""
import math

import numpy as np
import pytest

from oracle import partition as OP
from paper_2402_17427_gb300 import scenes


def ray_cast_visibility(box, cam, step=0.25):
    """Fraction of image points (grid of spacing `step` px over [-1/2, W-1/2] x [-1/2, H-1/2]) whose
    ray hits the box in front of the near plane (slab test in world coordinates)."""
    Rt = np.asarray(cam.world_to_cam, np.float64).reshape(3, 4)
    R, t = Rt[:, :3], Rt[:, 3]
    centre = -R.T @ t
    xs = np.arange(-0.5 + step / 2, cam.width - 0.5, step)
    ys = np.arange(-0.5 + step / 2, cam.height - 0.5, step)
    X, Y = np.meshgrid(xs, ys)
    d_cam = np.stack([(X - cam.cx) / cam.fx, (Y - cam.cy) / cam.fy, np.ones_like(X)], -1).reshape(-1, 3)
    d = d_cam @ R            # world direction; the ray parameter s equals the camera-space depth
    lo, hi = np.asarray(box[:3], np.float64), np.asarray(box[3:], np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = (lo - centre) / d
        t2 = (hi - centre) / d
    tmin = np.where(np.isnan(t1), -np.inf, np.minimum(t1, t2))
    tmax = np.where(np.isnan(t1), np.inf, np.maximum(t1, t2))
    # a zero direction component: the ray is inside that slab for all s or for none
    zero = d == 0
    inside = (centre >= lo) & (centre <= hi)
    tmin = np.where(zero, np.where(inside, -np.inf, np.inf), tmin)
    tmax = np.where(zero, np.where(inside, np.inf, -np.inf), tmax)
    enter = np.max(tmin, axis=1)
    leave = np.min(tmax, axis=1)
    hit = np.maximum(enter, cam.near) <= leave
    return float(hit.mean())


def _cams(seed, n=12, W=64, H=48):
    rng = np.random.default_rng(seed)
    cams = []
    for _ in range(n):
        eye = rng.uniform([-30, 5, -30], [30, 60, 30])
        yaw, pitch = rng.uniform(0, 2 * math.pi), math.radians(rng.uniform(-89, -10))
        cams.append(scenes.camera_from_forward(eye, scenes.yaw_pitch_forward(yaw, pitch), W, H))
    return cams


def test_visibility_matches_ray_casting():
    rng = np.random.default_rng(0)
    cams = _cams(1)
    boxes = []
    for _ in range(6):
        c = rng.uniform([-20, 0, -20], [20, 0, 20])
        ext = rng.uniform([2, 5, 2], [25, 40, 25])
        boxes.append(np.array([c[0] - ext[0], 0.0, c[2] - ext[2], c[0] + ext[0], ext[1], c[2] + ext[2]]))
    checked = 0
    for cam in cams:
        for b in boxes:
            v = OP.visibility(b, cam)
            r = ray_cast_visibility(b, cam)
            # grid quantisation: the boundary crosses at most ~2 (W + H) / step sample cells
            assert abs(v - r) <= 0.02, (v, r)
            checked += v > 0
    assert checked >= 10      # the case mix includes partly and fully visible boxes


def test_visibility_box_straddling_the_near_plane():
    # camera inside the box's airspace: the box surrounds the camera, so every ray meets it
    cam = scenes.camera_from_forward((0.0, 10.0, 0.0), (0.3, -0.5, 1.0), 64, 48)
    box = np.array([-50.0, 0.0, -50.0, 50.0, 30.0, 50.0])
    assert OP.visibility(box, cam) == pytest.approx(1.0, abs=1e-12)
    assert ray_cast_visibility(box, cam) == pytest.approx(1.0)
    # a box entirely behind the camera
    behind = np.array([-5.0, 0.0, -40.0, 5.0, 8.0, -20.0])
    cam2 = scenes.camera_from_forward((0.0, 10.0, 0.0), (0.0, 0.0, 1.0), 64, 48)
    assert OP.visibility(behind, cam2) == 0.0
    assert ray_cast_visibility(behind, cam2) == 0.0
    # a box cut by the near plane: the clipped part still matches ray casting
    cut = np.array([1.0, 8.0, -3.0, 3.0, 12.0, 6.0])   # beside the camera, partly behind it
    v, r = OP.visibility(cut, cam2), ray_cast_visibility(cut, cam2)
    assert 0.05 < v < 1.0 and abs(v - r) <= 0.02


def test_visibility_nadir_closed_form():
    # camera 100 m above the centre of a 40 x 30 m box of height 20 m: the projection is the top
    # face (depth 80 m), fx Lx / d by fy Lz / d pixels
    W, H = 640, 480
    cam = scenes.camera_from_forward((10.0, 100.0, -5.0), (0.0, -1.0, 0.0), W, H)
    box = np.array([-10.0, 0.0, -20.0, 30.0, 20.0, 10.0])
    d = 100.0 - 20.0
    expect = (cam.fx * 40.0 / d) * (cam.fy * 30.0 / d) / (W * H)
    assert OP.visibility(box, cam) == pytest.approx(expect, rel=1e-6)
    assert OP.select(np.array([expect]), 0.25)[0] == (expect > 0.25)


def test_airspace_box_spans_ground_to_highest_point():
    rng = np.random.default_rng(3)
    p = rng.uniform([0, 2, 5], [10, 7, 9], (100, 3))
    b = OP.airspace_box(p, ground_y=-1.0)
    assert b[1] == -1.0 and b[4] == p[:, 1].max()
    assert b[0] == p[:, 0].min() and b[3] == p[:, 0].max() and b[2] == p[:, 2].min() and b[5] == p[:, 2].max()


def test_merge_filter_half_open_rectangles():
    # points on a 2 x 2 partition's shared edges are kept by exactly one cell
    xs = np.array([-1.0, 0.0, 0.5, 1.0, 2.0])
    pts = np.array([[x, 3.0, z] for x in xs for z in xs])
    regions = [(-1.0, 1.0, -1.0, 1.0), (1.0, 3.0, -1.0, 1.0), (-1.0, 1.0, 1.0, 3.0), (1.0, 3.0, 1.0, 3.0)]
    masks = np.stack([OP.merge_keep(pts, r) for r in regions])
    assert np.all(masks.sum(axis=0) == 1)
    # the whole partition keeps everything once; the merged list is cell-major, index order
    merged = OP.merge([pts] * 4, regions)
    assert len(merged) == len(pts)
    assert merged == sorted(merged)
