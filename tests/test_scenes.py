"""The seeded synthetic inputs: each generator is deterministic for its seed and follows the
recipe its docstring states (the shapes, boxes, distributions and cameras of the paper's
workloads that these inputs stand in for)."""
import math

import numpy as np
import pytest

from paper_2402_17427_gb300 import scenes


def _check_camera(cam, width, height, hfov_deg=60.0):
    assert (cam.width, cam.height) == (width, height)
    R = cam.R.astype(np.float64)
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-5)            # a rotation
    assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-5)
    # camera = R world + t, so the centre maps to the origin
    assert np.allclose(R @ cam.cam_pos + cam.t, 0.0, atol=1e-3)
    assert cam.fx == pytest.approx(0.5 * width / math.tan(math.radians(hfov_deg) / 2), rel=1e-5)
    assert cam.world_to_cam.shape == (3, 4)


def _forward(cam):
    """World-space viewing direction (the camera's +z axis)."""
    return cam.R.astype(np.float64)[2]


def test_blob_cell_is_deterministic_and_follows_its_recipe():
    a = scenes.blob_cell_1080p(seed=7, n=50_000)
    b = scenes.blob_cell_1080p(seed=7, n=50_000)
    for x, y in zip(a[0].arrays(), b[0].arrays()):
        assert np.array_equal(x, y)
    assert np.array_equal(a[2], b[2])
    g, cam, target = a
    assert g.n == 50_000 and g.sh_degree == 3 and g.sh.shape == (50_000, 16, 3)
    m = g.means
    assert m.min(axis=0).min() >= 0.0 and np.all(m.max(axis=0) <= np.array([100.0, 20.0, 100.0]) + 1e-4)
    assert float(g.log_scales.mean()) == pytest.approx(math.log(0.08), abs=0.02)
    assert float(g.log_scales.std()) == pytest.approx(0.5, abs=0.02)
    q = g.quats.astype(np.float64)
    assert np.allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-5)
    _check_camera(cam, 1920, 1080)
    assert cam.cam_pos[1] == pytest.approx(30.0, abs=1e-4)      # 30 m altitude
    r = math.hypot(cam.cam_pos[0] - 50.0, cam.cam_pos[2] - 50.0)
    assert r == pytest.approx(30.0, abs=1e-3)                    # on the 30 m orbit
    assert _forward(cam)[1] == pytest.approx(-math.sin(math.pi / 4), abs=1e-5)   # pitched down 45 deg
    assert target.shape == (3, 1080, 1920) and target.min() >= 0.0 and target.max() <= 1.0
    c = scenes.blob_cell_1080p(seed=8, n=50_000)
    assert not np.array_equal(a[0].means, c[0].means)            # the seed matters


def test_small_cell_recipe():
    g, cam, target = scenes.small_cell(3)
    assert g.n == 10_000 and g.sh_degree == 0
    assert g.means.min() >= -2.0 and g.means.max() <= 2.0
    assert float(g.log_scales.mean()) == pytest.approx(-3.0, abs=0.03)
    assert (cam.width, cam.height) == (128, 128) and cam.fx == pytest.approx(128.0)
    assert np.allclose(cam.cam_pos, [0.0, 0.0, -6.0], atol=1e-5)
    assert target.shape == (3, 128, 128)


def test_request_stream_mix_rate_and_cameras():
    reqs = scenes.request_stream(seed=11, rate_hz=200.0, duration_s=20.0)
    n = len(reqs)
    assert n == pytest.approx(4000, rel=0.06)                   # Poisson, 200 per second
    t = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(t) > 0) and t[-1] < 20.0
    sizes = [(r.camera.width, r.camera.height) for r in reqs]
    frac = [sizes.count(s) / n for s in [(1280, 720), (1920, 1080), (3840, 2160)]]
    assert frac == pytest.approx([0.50, 0.35, 0.15], abs=0.03)
    alt = np.array([r.camera.cam_pos[1] for r in reqs])
    assert alt.min() >= 20.0 - 1e-3 and alt.max() <= 150.0 + 1e-3
    pitch = np.degrees(np.arcsin(np.clip([-_forward(r.camera)[1] for r in reqs], -1, 1)))
    assert pitch.min() >= 30.0 - 1e-2 and pitch.max() <= 90.0 + 1e-2
    assert [r.rid for r in reqs] == list(range(n))
    again = scenes.request_stream(seed=11, rate_hz=200.0, duration_s=20.0)
    assert [r.arrival_s for r in again] == list(t)


def test_aerial_cells_grid_cameras_and_scales():
    sizes = (3000, 5000, 8000, 12000, 15000, 20000, 25000, 30000)
    cells = scenes.aerial_cells(step=5, sizes=sizes)
    assert [c.gaussians.n for c in cells] == list(sizes)
    for k, c in enumerate(cells):
        x0, z0 = 250.0 * (k % 4), 500.0 * (k // 4)          # 4 x 2 grid of 250 x 500 m cells
        m = c.gaussians.means
        # ground points stay inside the cell; facade points at most half a footprint outside it
        assert np.median(m[:, 0]) == pytest.approx(x0 + 125.0, abs=60.0)
        assert np.median(m[:, 2]) == pytest.approx(z0 + 250.0, abs=120.0)
        assert np.allclose(c.aabb, np.concatenate([m.min(0), m.max(0)]))
        mu = math.log(0.5 * math.sqrt(250.0 * 500.0 / sizes[k]))
        assert float(c.gaussians.log_scales.mean()) == pytest.approx(mu, abs=0.05)
        cam = c.camera
        _check_camera(cam, 1152, 864)
        assert np.allclose(_forward(cam), [0.0, -1.0, 0.0], atol=1e-5)      # nadir
        ground = float(scenes._heightfield(cam.cam_pos[0], cam.cam_pos[2]))
        assert cam.cam_pos[1] - ground == pytest.approx(100.0, abs=1e-3)   # 100 m above ground
        assert x0 < cam.cam_pos[0] < x0 + 250.0 and z0 < cam.cam_pos[2] < z0 + 500.0


def test_merged_city_sizes_and_grid():
    cells = scenes.merged_city(total_scale=0.01)
    sizes = [c.gaussians.n for c in cells]
    assert sizes == [int(round(500_000 * (1 + k / 5) * 0.01)) for k in range(16)]
    slots = set()
    for c in cells:
        cx, cz = np.median(c.gaussians.means[:, 0]), np.median(c.gaussians.means[:, 2])
        slots.add((int(cx // 250.0), int(cz // 250.0)))
        assert c.camera is None
    assert slots == {(i, j) for i in range(4) for j in range(4)}  # every grid slot holds one cell
