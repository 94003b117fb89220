"""Serving the merged scene at full scale (pattern 5): 16 cells, 20,000,000 Gaussians (SH degree 3)
resident on the device.  Novel views at 3840x2160 and 1920x1080 match the oracle (rendering all
cells) on sampled tiles; every view is the same alone and in a batch; a request stream with its
4K requests kept at 4K is served with every result equal to the same view rendered alone; memory
admission serves an oversized request alone and never holds more in flight than the budget.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2402_17427_gb300 import scenes, serving

from _gpu import conservative_tile_rects, subset_reaching

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def city():
    from paper_2402_17427_gb300 import _build
    _build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    cells = scenes.merged_city()
    srv = serving.SceneServer(cells, slots=3, max_batch=8)
    merged = scenes.Gaussians.concat([c.gaussians for c in cells])
    yield cells, srv, merged
    del srv
    torch.cuda.empty_cache()


def _view(seed, W, H):
    rng = np.random.default_rng(seed)
    yaw = rng.uniform(0, 2 * np.pi)
    pitch = np.radians(rng.uniform(-75, -40))
    eye = (rng.uniform(300, 700), rng.uniform(60, 110), rng.uniform(300, 700))
    return scenes.camera_from_forward(eye, scenes.yaw_pitch_forward(yaw, pitch), W, H)


@pytest.mark.parametrize("W,H,seed", [(3840, 2160, 21), (1920, 1080, 22)])
def test_full_city_view_matches_oracle_on_sampled_tiles(city, W, H, seed):
    cells, srv, merged = city
    cam = _view(seed, W, H)
    outs, counters, kept = srv.render([cam])
    assert counters[2] == 0 and 0 < kept[0] <= 16
    T = 16
    tx, ty = (W + T - 1) // T, (H + T - 1) // T
    rng = np.random.default_rng(seed)
    tiles = sorted(set(rng.choice(tx * ty, 16, replace=False).tolist()) | {(ty // 2) * tx + tx // 2})
    m = np.zeros(tx * ty, np.uint8)
    m[tiles] = 1
    sub = subset_reaching(conservative_tile_rects(merged, cam, T), m, tx, ty)
    orc = oracle.render(merged.subset(sub), cam, oracle.Options(), tile_mask=m)
    pm = np.repeat(np.repeat(m.reshape(ty, tx).astype(bool), T, 0), T, 1)[:H, :W]
    ok = pm & ~orc.amb.astype(bool)
    img = outs[0][0].cpu().numpy()
    assert ok.sum() > 0.9 * pm.sum()
    assert np.abs(img - orc.image)[:, ok].max() <= 1e-4
    assert np.abs(outs[0][1].cpu().numpy() - orc.T)[ok].max() <= 1e-4


def test_full_city_views_same_alone_and_in_the_mix(city):
    _, srv, _ = city
    cams = [_view(30 + i, *wh) for i, wh in enumerate([(3840, 2160), (1280, 720), (1920, 1080), (1280, 720)])]
    mix, _, _ = srv.render(cams)
    for i, cam in enumerate(cams):
        alone, _, _ = srv.render([cam])
        for a, b in zip(alone[0], mix[i]):
            assert torch.equal(a, b), i


def test_full_city_request_stream_with_4k_requests(city):
    _, srv, _ = city
    reqs = scenes.request_stream(seed=12, rate_hz=200.0, duration_s=1.0)
    assert any(r.camera.width == 3840 for r in reqs)
    stats, outs = srv.serve(reqs, keep_outputs=True)
    assert stats.requests == len(reqs) and stats.p99_ms >= stats.p50_ms > 0
    for r in reqs[:: max(1, len(reqs) // 8)]:
        alone, _, _ = srv.render([r.camera])
        assert torch.equal(alone[0][0], outs[r.rid][0]), r.rid


def test_memory_admission_with_a_budget_below_one_4k_request(city):
    cells, srv, _ = city
    pool = scenes.request_stream(seed=13, rate_hz=200.0, duration_s=2.0)
    big = [r for r in pool if r.camera.width == 3840][:4]
    small = [r for r in pool if r.camera.width != 3840][:8]
    reqs = sorted(big + small, key=lambda r: r.rid)
    for k, r in enumerate(reqs):          # all arrive within the first 50 ms
        r.arrival_s = 0.005 * k
    assert len(big) == 4
    one_4k = srv._bytes(big[0].camera)
    tight = serving.SceneServer.__new__(serving.SceneServer)
    tight.__dict__.update(srv.__dict__)
    tight.budget = one_4k // 2                 # smaller than one 4K request
    stats, outs = tight.serve(reqs, keep_outputs=True)
    assert stats.requests == len(reqs)         # every request served, one batch at a time
    assert stats.max_inflight == 1 and stats.mean_batch == 1.0
    roomy = serving.SceneServer.__new__(serving.SceneServer)
    roomy.__dict__.update(srv.__dict__)
    roomy.budget = int(2.5 * one_4k)
    stats2, outs2 = roomy.serve(reqs, keep_outputs=True)
    assert stats2.requests == len(reqs)
    # nothing beyond the budget is in flight unless a single request alone exceeds it
    assert stats2.max_inflight_bytes <= roomy.budget
    for r in reqs:
        assert torch.equal(outs[r.rid][0], outs2[r.rid][0])
