"""Stage-isolated parity of the key path, and the bounded-wait error path, through the C ABI.

Strict protocol: the forward pass records, per Gaussian, the FP32 values it decided the tile
rectangle and the sort key from, (u, v, r, depth).  Fed those values, the oracle's own key
generation, stable sort and range code (``oracle.pairs_from_fp32``) must reproduce the kernel's
pair count, every tile range and every tile list exactly: no Gaussian is excluded, so this
isolates the integer stages (rectangles, keys, the two-level radix sort, ranges) from the
floating-point ones.  Separately, u, v and depth — computed on both sides in FP32 with one stated
operation order — must equal the oracle's bit for bit, and r must agree to FP32 accuracy (it goes
through exp and sqrt, which may differ in the last bits).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2402_17427_gb300 import batch as BT
from paper_2402_17427_gb300 import binding as B
from paper_2402_17427_gb300 import rasterize as R
from paper_2402_17427_gb300 import scenes

from _gpu import oracle_opts, read_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2402_17427_gb300 import _build
    _build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _render_recording(g, cam, settings):
    r = R.Rasterizer(settings)
    params = R.to_device(g)
    ki = torch.zeros((max(g.n, 1), 4), dtype=torch.float32, device="cuda")
    r.forward(*params, g.sh_degree, cam, key_inputs=ki)
    torch.cuda.synchronize()
    return r, ki.cpu().numpy()[:g.n], r.counters.cpu().numpy()


def _assert_lists_identical(gpu_ranges, gpu_ids, P, uvrd, W, H, tile, tile_base=0, id_base=0):
    keys, ids, ranges = oracle.pairs_from_fp32(uvrd, W, H, tile)
    tiles = ranges.shape[0]
    got_r = gpu_ranges[tile_base:tile_base + tiles]
    # the GPU numbers pairs globally: shift this view's ranges to start at 0 (empty stays (0, 0))
    nonempty = got_r[:, 1] > got_r[:, 0]
    first = int(got_r[nonempty, 0].min()) if nonempty.any() else 0
    got_r = np.where(nonempty[:, None], got_r - first, 0)
    assert np.array_equal(got_r, ranges.astype(np.int64)), "tile ranges differ"
    got_ids = gpu_ids[first:first + len(ids)].astype(np.int64) - id_base
    assert np.array_equal(got_ids, ids.astype(np.int64)), "tile lists differ"
    return len(ids)


def _check_key_path(uvrd, orc):
    """u, v, depth bit-exact against the oracle's FP32 key path; r to FP32 accuracy."""
    both = orc.rec["valid"] & (uvrd[:, 2] >= 0)
    assert np.array_equal(orc.rec["valid"], uvrd[:, 2] >= 0) or \
        (orc.rec["valid"] != (uvrd[:, 2] >= 0)).sum() <= 1e-5 * len(uvrd) + 1
    for k, name in enumerate(["u32", "v32"]):
        assert np.array_equal(uvrd[both, k].view(np.uint32), orc.rec[name][both].view(np.uint32)), name
    assert np.array_equal(uvrd[both, 3].view(np.uint32), orc.rec["depth32"][both].view(np.uint32))
    r_gpu, r_orc = uvrd[both, 2].astype(np.float64), orc.rec["radius"][both]
    rel = np.abs(r_gpu - r_orc) / r_orc
    # FP32 through exp, the covariance products and two square roots: a few units in 1e-6, up to
    # about 1.2e-5 for Gaussians thousands of pixels wide (the oracle's rectangle band covers it)
    assert rel.max() <= 2e-5, (rel.max(), np.percentile(rel, 99))
    return int(both.sum())


@pytest.mark.parametrize("case", ["small", "tiny8", "tiny32", "ragged"])
def test_strict_lists_small_scenes(case):
    if case == "small":
        g, cam, _ = scenes.small_cell(0)
        s = R.RasterSettings()
    elif case == "tiny8":
        g, cam, _ = scenes.tiny_scene(n=300, width=100, height=61, degree=3, seed=6)
        s = R.RasterSettings(tile_size=8)
    elif case == "tiny32":
        g, cam, _ = scenes.tiny_scene(n=150, width=64, height=32, degree=3, seed=5)
        s = R.RasterSettings(tile_size=32)
    else:
        g, cam, _ = scenes.tiny_scene(n=80, width=33, height=35, degree=0, seed=4)
        s = R.RasterSettings()
    r, uvrd, cnt = _render_recording(g, cam, s)
    assert cnt[B.VG_CNT_STATUS] == 0
    st = read_state(r, g, cam)
    P = _assert_lists_identical(st["ranges"], st["ids"], int(cnt[B.VG_CNT_PAIRS]), uvrd, cam.width, cam.height,
                                s.tile_size)
    assert P == int(cnt[B.VG_CNT_PAIRS])
    orc = oracle.render(g, cam, oracle_opts(s))
    _check_key_path(uvrd, orc)


def test_strict_lists_blob_cell_1080p_full_frame():
    """1M Gaussians, SH3, 1920x1080 (the benchmark's render): all 2M pairs, every tile."""
    g, cam, _ = scenes.blob_cell_1080p()
    s = R.RasterSettings()
    r, uvrd, cnt = _render_recording(g, cam, s)
    assert cnt[B.VG_CNT_STATUS] == 0
    st = read_state(r, g, cam)
    P = _assert_lists_identical(st["ranges"], st["ids"], int(cnt[B.VG_CNT_PAIRS]), uvrd, cam.width, cam.height, 16)
    assert P == int(cnt[B.VG_CNT_PAIRS]) > 1_000_000
    # the FP32 key path of every Gaussian (projection only: no tile is rendered)
    tiles = ((cam.width + 15) // 16) * ((cam.height + 15) // 16)
    orc = oracle.render(g, cam, oracle.Options(), tile_mask=np.zeros(tiles, np.uint8))
    assert _check_key_path(uvrd, orc) > 100_000


@pytest.mark.parametrize("n,longest", [(1600, 1249), (12000, 9361)])
def test_strict_lists_dense_clusters_with_long_lists(n, longest):
    """Dense clusters whose longest tile list holds over a thousand and over nine thousand entries
    (the oracle's count): every list equals the oracle's from the kernel's own FP32 inputs."""
    g, cam, _ = scenes.tiny_scene(n=n, width=96, height=64, degree=1, seed=8, box=0.25, log_scale=(-3.0, 0.3))
    s = R.RasterSettings()
    r, uvrd, cnt = _render_recording(g, cam, s)
    assert cnt[B.VG_CNT_STATUS] == 0
    st = read_state(r, g, cam)
    lens = st["ranges"][:, 1] - st["ranges"][:, 0]
    assert abs(int(lens.max()) - longest) <= 2, lens.max()
    P = _assert_lists_identical(st["ranges"], st["ids"], int(cnt[B.VG_CNT_PAIRS]), uvrd, cam.width, cam.height, 16)
    assert P == int(cnt[B.VG_CNT_PAIRS])


@pytest.mark.slow
def test_strict_lists_aerial_cells_batched_mixed_tiles():
    """Eight uneven aerial cells (0.3M..3.0M, 1152x864) in one batched call with tile sizes 8, 16
    and 32 mixed across cells: every cell's lists equal the oracle's from its own FP32 inputs."""
    cells = scenes.aerial_cells(step=3)
    tiles = [8, 16, 32, 16, 8, 32, 16, 8]
    settings = [R.RasterSettings(tile_size=t) for t in tiles]
    br = BT.BatchRasterizer(settings)
    params = [R.to_device(c.gaussians) for c in cells]
    cams = [c.camera for c in cells]
    total = sum(c.gaussians.n for c in cells)
    ki = torch.zeros((total, 4), dtype=torch.float32, device="cuda")
    br.forward(params, 3, cams, key_inputs=ki)
    torch.cuda.synchronize()
    cnt = br.counters.cpu().numpy()
    assert cnt[B.VG_CNT_STATUS] == 0
    ranges, ids = br.read_state(params, 3, cams)
    uvrd = ki.cpu().numpy()
    off, tbase, P = 0, 0, 0
    for c, s in zip(cells, settings):
        cam, n = c.camera, c.gaussians.n
        nt = ((cam.width + s.tile_size - 1) // s.tile_size) * ((cam.height + s.tile_size - 1) // s.tile_size)
        P += _assert_lists_identical(ranges, ids, 0, uvrd[off:off + n], cam.width, cam.height, s.tile_size,
                                     tile_base=tbase, id_base=off)
        off += n
        tbase += nt
    assert P == int(cnt[B.VG_CNT_PAIRS])


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """A look-back predecessor that never publishes (test-only flag): the wait gives up after its
    limit, the status word reports it, the wrapper raises VGError(VG_ERR_TIMEOUT), the outputs
    are the empty-list render, and the next render on the same workspace is correct."""
    g, cam, _ = scenes.small_cell(0)
    params = R.to_device(g)
    r = R.Rasterizer(R.RasterSettings(test_stall=True, bg=(0.25, 0.5, 0.75)))
    with pytest.raises(B.VGError) as e:
        r.forward(*params, g.sh_degree, cam)
    assert e.value.status == B.VG_ERR_TIMEOUT
    c = r.counters if r.counters is not None else None
    # the deferred form reports the same status without raising at the call
    r.check = "defer"
    rgb, T, last = r.forward(*params, g.sh_degree, cam)
    torch.cuda.synchronize()
    cnt = r.counters.cpu().numpy()
    assert cnt[B.VG_CNT_STATUS] & B.VG_STATUS_WAIT_TIMEOUT
    assert cnt[B.VG_CNT_PAIRS] == 0
    assert torch.all(T == 1) and torch.all(last == 0)
    bg = torch.tensor([0.25, 0.5, 0.75], device="cuda")[:, None, None]
    assert torch.all(rgb == bg.expand_as(rgb))
    with pytest.raises(B.VGError):
        r.verify()
    # a backward on the timed-out workspace writes no gradient of a visible Gaussian and faults nothing
    dL = torch.ones_like(rgb)
    r.backward(*params, g.sh_degree, cam, T, last, dL)
    torch.cuda.synchronize()
    del c
    # the same rasteriser and workspace, stall off: a normal, correct render
    r.settings.test_stall = False
    r.check = "sync"
    rgb, T, last = r.forward(*params, g.sh_degree, cam)
    torch.cuda.synchronize()
    assert r.counters.cpu().numpy()[B.VG_CNT_STATUS] == 0
    orc = oracle.render(g, cam, oracle_opts(r.settings))
    ok = ~orc.amb.astype(bool)
    assert np.abs(rgb.cpu().numpy() - orc.image)[:, ok].max() <= 1e-4
