"""GPU parity of the scene-partition kernels (Sec. 4.1 airspace-aware visibility, Sec. 4.3 merging)
against the FP64 partition oracle, through the C ABI."""
import math

import numpy as np
import pytest
import torch

from oracle import partition as OP
from paper_2402_17427_gb300 import binding as B
from paper_2402_17427_gb300 import partition as PT
from paper_2402_17427_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2402_17427_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()


def _cells_points(seed, n_cells=5, empty=2):
    rng = np.random.default_rng(seed)
    pts, offs = [], [0]
    for k in range(n_cells):
        n = 0 if k == empty else int(rng.integers(1, 200_000))
        c = rng.uniform([-300, 0, -300], [300, 0, 300])
        p = c + rng.uniform([-60, 0, -60], [60, 80, 60], (n, 3))
        pts.append(p.astype(np.float32))
        offs.append(offs[-1] + n)
    return np.concatenate(pts), offs


def test_airspace_boxes_are_exact():
    pts, offs = _cells_points(0)
    out = PT.airspace_boxes(torch.from_numpy(pts).cuda(), offs, ground_y=-2.5).cpu().numpy()
    for k in range(len(offs) - 1):
        p = pts[offs[k]:offs[k + 1]]
        if len(p) == 0:
            assert np.isinf(out[k, 0]) and out[k, 0] > 0 and np.isinf(out[k, 3]) and out[k, 3] < 0
            continue
        ref = OP.airspace_box(p, -2.5).astype(np.float32)
        assert np.array_equal(out[k], ref), (k, out[k], ref)


def _cameras(seed, n, sizes=((64, 48), (1920, 1080), (1152, 864))):
    rng = np.random.default_rng(seed)
    cams = []
    for i in range(n):
        W, H = sizes[i % len(sizes)]
        eye = rng.uniform([-400, 10, -400], [400, 200, 400])
        yaw, pitch = rng.uniform(0, 2 * math.pi), math.radians(rng.uniform(-90, -5))
        cams.append(scenes.camera_from_forward(eye, scenes.yaw_pitch_forward(yaw, pitch), W, H))
    return cams


def test_visibility_and_selection_match_oracle():
    pts, offs = _cells_points(1, n_cells=8, empty=-1)
    boxes_t = PT.airspace_boxes(torch.from_numpy(pts).cuda(), offs, ground_y=0.0)
    boxes = boxes_t.cpu().numpy().astype(np.float64)
    cams = _cameras(2, 60)
    # a camera inside a box's airspace, one right above a box and one looking away
    cams.append(scenes.camera_from_forward(boxes[0, [0, 1, 2]] + (boxes[0, 3:] - boxes[0, :3]) / 2, (0.2, -0.5, 1.0), 640, 480))
    c = (boxes[3, :3] + boxes[3, 3:]) / 2
    cams.append(scenes.camera_from_forward((c[0], boxes[3, 4] + 150.0, c[2]), (0.0, -1.0, 0.0), 640, 480))
    cams.append(scenes.camera_from_forward((c[0], 50.0, c[2] - 1000.0), (0.0, 0.0, -1.0), 640, 480))
    vis, sel = PT.camera_visibility(boxes_t, cams, 0.25)
    vis, sel = vis.cpu().numpy(), sel.cpu().numpy()
    ref = OP.visibility_matrix(boxes, cams)
    assert np.abs(vis - ref).max() <= 1e-6
    settled = np.abs(ref - 0.25) > 1e-9
    assert np.array_equal(sel[settled], OP.select(ref, 0.25)[settled])
    assert (ref > 0).sum() > 20 and (ref > 0.25).sum() > 3 and (ref == 0).sum() > 20   # a mix of cases
    assert ref[-3, 0] == pytest.approx(1.0) and ref[-1, 3] == 0.0


def _expanded_cells(seed, grid=2, n=40_000, cell=100.0, degree=3):
    """Cells of a grid x grid partition whose Gaussians cover the 20%-expanded rectangle (Sec. 4.1),
    plus points on the original edges; regions are the original rectangles."""
    rng = np.random.default_rng(seed)
    cells, regions = [], []
    for gz in range(grid):
        for gx in range(grid):
            x0, z0 = gx * cell, gz * cell
            m = rng.uniform([x0 - 0.1 * cell, 0, z0 - 0.1 * cell], [x0 + 1.1 * cell, 30, z0 + 1.1 * cell], (n, 3))
            m[:50, 0] = x0            # on the left edge (kept) and the right edge (not kept)
            m[50:100, 0] = x0 + cell
            m[100:150, 2] = z0 + cell
            g = scenes.Gaussians(m.astype(np.float32),
                                 rng.normal(-2, 0.3, (n, 3)).astype(np.float32),
                                 rng.standard_normal((n, 4)).astype(np.float32),
                                 rng.standard_normal(n).astype(np.float32),
                                 rng.standard_normal((n, (degree + 1) ** 2, 3)).astype(np.float32), degree)
            cells.append(g)
            regions.append((x0, x0 + cell, z0, z0 + cell))
    return cells, regions


@pytest.mark.parametrize("degree", [0, 3])
def test_merge_matches_oracle(degree):
    cells, regions = _expanded_cells(3, degree=degree)
    cells[1] = cells[1].subset(np.arange(0))     # an empty cell
    dev = [tuple(torch.from_numpy(a).cuda() for a in (g.means, g.log_scales, g.quats, g.opacity_logits, g.sh))
           for g in cells]
    merged = PT.merge_cells(dev, regions, degree)
    keep = OP.merge([g.means for g in cells], regions)
    assert int(merged[0].shape[0]) == len(keep)
    for name, t in zip(["means", "log_scales", "quats", "opacity_logits", "sh"], merged):
        ref = np.concatenate([getattr(cells[k], name)[[i]] for k, i in keep]) if keep else None
        assert np.array_equal(t.cpu().numpy(), ref), name


def test_merge_keeps_nothing_and_everything():
    cells, _ = _expanded_cells(4, grid=1, n=1000, degree=1)
    dev = [tuple(torch.from_numpy(a).cuda() for a in (g.means, g.log_scales, g.quats, g.opacity_logits, g.sh))
           for g in cells]
    none = PT.merge_cells(dev, [(1e6, 1e6 + 1, 0, 1)], 1)
    assert int(none[0].shape[0]) == 0
    allm = PT.merge_cells(dev, [(-1e9, 1e9, -1e9, 1e9)], 1)
    assert np.array_equal(allm[4].cpu().numpy(), cells[0].sh)


def test_partition_rejects_bad_arguments():
    with pytest.raises(B.VGError):
        B.vg_camera_visibility(0, 1, [], 0.25, 0, 0, 0, 0, 0)
    assert B.vg_visibility_workspace_bytes(0) == 0
