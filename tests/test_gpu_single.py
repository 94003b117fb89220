"""GPU parity of the single-view path (forward, tile lists, backward, loss) against the oracle.

Calls go through the C ABI (libvgrast.so via ctypes).  Tolerances: tile lists and sort order
bit-exact; images max-abs 1e-4 outside the pixels the oracle marks as sitting inside a decision
band; gradients relative L2 error <= 2e-3 per parameter group (FP32 GPU vs FP64 oracle).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2402_17427_gb300 import binding as B
from paper_2402_17427_gb300 import rasterize as R
from paper_2402_17427_gb300 import scenes

from _gpu import (group_errors, oracle_opts, reachable_subset, read_state, run_backward, run_forward,
                  tile_lists_equal)

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4
GRAD_TOL = 2e-3


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2402_17427_gb300 import _build
    _build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def check_image(orc, out, tol=IMG_TOL, mask=None):
    amb = orc.amb.astype(bool)
    ok = ~amb if mask is None else (~amb & mask)
    diff = np.abs(out["image"] - orc.image)[:, ok]
    assert diff.size == 0 or diff.max() <= tol, diff.max()
    dT = np.abs(out["T"] - orc.T)[ok]
    assert dT.size == 0 or dT.max() <= tol, dT.max()
    return int(amb.sum())


def check_grads(gpu, ref, keep, tol=GRAD_TOL):
    errs = group_errors(gpu, ref, keep)
    for k, (rel, _elem, norm) in errs.items():
        if norm > 0:
            assert rel <= tol, (k, errs)
    return errs


def render_both(g, cam, settings=None, **kw):
    settings = settings or R.RasterSettings()
    r, params, out = run_forward(g, cam, settings, **kw)
    orc = oracle.render(g, cam, oracle_opts(settings))
    return r, params, out, orc


# ------------------------------------------------------------------ small cell (10k Gaussians)

def test_small_cell_forward_and_tile_lists():
    g, cam, _ = scenes.small_cell(0)
    r, params, out, orc = render_both(g, cam)
    assert out["counters"][B.VG_CNT_STATUS] == 0
    namb = int(orc.rec["rect_amb"].sum())
    assert abs(int(out["counters"][B.VG_CNT_VISIBLE]) - orc.n_visible) <= namb
    st = read_state(r, g, cam)
    amb_ids = np.nonzero(orc.rec["rect_amb"])[0]
    bad = tile_lists_equal(orc, st, range(orc.ranges.shape[0]), amb_ids)
    assert not bad, bad
    if namb == 0:
        assert int(out["counters"][B.VG_CNT_PAIRS]) == orc.num_pairs
        assert np.array_equal(st["ranges"], orc.ranges)
    check_image(orc, out)
    # projected records: the blending position (FP32 + remainder) to 1e-6 px, the rest to FP32
    # accuracy (the FP32 key path itself is checked through the bit-exact tile lists above)
    vis = orc.rec["visible"] & (st["touched"] > 0)
    u = st["proj"][vis, 0].astype(np.float64) + st["proj"][vis, 10]
    v = st["proj"][vis, 1].astype(np.float64) + st["proj"][vis, 11]
    assert np.abs(u - orc.rec["u"][vis]).max() < 1e-6 and np.abs(v - orc.rec["v"][vis]).max() < 1e-6
    conic = orc.rec["conic"][vis]
    scale = np.abs(conic).max(1, keepdims=True)
    assert (np.abs(st["proj"][vis, 2:5] - conic) / scale).max() < 2e-5
    assert np.abs(st["proj"][vis, 5] - orc.rec["opacity"][vis]).max() < 1e-6
    assert np.abs(st["proj"][vis, 6:9] - orc.rec["rgb"][vis]).max() < 1e-5
    # last contributor: equal wherever the pixel is unambiguous and its tile list matches in full
    full_ok = np.zeros(orc.ranges.shape[0], bool)
    full_ok[[t for t in range(len(full_ok)) if t not in set(tile_lists_equal(orc, st, range(len(full_ok))))]] = True
    tmask = np.repeat(np.repeat(full_ok.reshape(orc.tiles_y, orc.tiles_x), 16, 0), 16, 1)[:cam.height, :cam.width]
    sel = tmask & ~orc.amb.astype(bool)
    assert np.array_equal(out["last"][sel], orc.last[sel])


def test_small_cell_gradients_l1():
    g, cam, target = scenes.small_cell(0)
    r, params, out, orc = render_both(g, cam)
    # dL/dI of the L1 loss at the oracle's image, zero at ambiguous pixels
    dL = np.sign(orc.image - target) / orc.image.size
    dL[:, orc.amb.astype(bool)] = 0.0
    dL = dL.astype(np.float32)
    gpu = run_backward(r, params, g, cam, out, dL)
    ref = orc.backward(dL.astype(np.float64))
    keep = ~(orc.rec["grad_amb"] | orc.rec["rect_amb"])
    check_grads(gpu, ref, keep)


@pytest.mark.parametrize("n,W,H,tile,deg,seed,bg,stop", [
    (60, 32, 32, 16, 3, 1, (0, 0, 0), 0),
    (200, 48, 40, 16, 2, 2, (1.0, 0.5, 0.25), 0),
    (120, 40, 24, 8, 1, 3, (0, 0, 0), 1),
    (80, 33, 35, 16, 0, 4, (0, 0, 0), 0),
    (150, 64, 32, 32, 3, 5, (0.2, 0.2, 0.2), 1),
    (300, 100, 61, 8, 3, 6, (0, 0, 0), 0),
])
def test_tiny_scenes_forward_backward(n, W, H, tile, deg, seed, bg, stop):
    g, cam, _ = scenes.tiny_scene(n=n, width=W, height=H, degree=deg, seed=seed)
    s = R.RasterSettings(tile_size=tile, bg=bg, stop_rule=stop)
    r, params, out, orc = render_both(g, cam, s)
    check_image(orc, out)
    st = read_state(r, g, cam)
    assert not tile_lists_equal(orc, st, range(orc.ranges.shape[0]), np.nonzero(orc.rec["rect_amb"])[0])
    w = np.random.default_rng(seed).standard_normal((3, H, W)).astype(np.float32)
    w[:, orc.amb.astype(bool)] = 0
    gpu = run_backward(r, params, g, cam, out, w)
    ref = orc.backward(w.astype(np.float64))
    check_grads(gpu, ref, ~(orc.rec["grad_amb"] | orc.rec["rect_amb"]))


def test_means2d_abs_statistic_matches_oracle():
    """The adjoint variant that also accumulates the densification statistic (per Gaussian, the sum
    over pixels of |dL/du| + |dL/dv| of each pixel's contribution, added to the caller's buffer):
    the statistic and every gradient group against the FP64 oracle."""
    g, cam, _ = scenes.tiny_scene(n=200, width=48, height=40, degree=2, seed=2)
    r, params, out, orc = render_both(g, cam)
    w = np.random.default_rng(2).standard_normal((3, cam.height, cam.width)).astype(np.float32)
    w[:, orc.amb.astype(bool)] = 0
    acc = torch.zeros(g.n, dtype=torch.float32, device="cuda")
    gpu = run_backward(r, params, g, cam, out, w, means2d_abs=acc)
    ref = orc.backward(w.astype(np.float64))
    keep = ~(orc.rec["grad_amb"] | orc.rec["rect_amb"])
    check_grads(gpu, ref, keep)
    got, want = acc.cpu().numpy().astype(np.float64)[keep], ref["g2d_abs"][keep]
    assert np.linalg.norm(want) > 0
    assert np.linalg.norm(got - want) <= GRAD_TOL * np.linalg.norm(want), np.linalg.norm(got - want) / np.linalg.norm(want)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_opaque_splats_clamped_at_alpha_max(tile):
    """Splats whose opacity is nearly 1 reach alpha_max near their centres: there alpha is clamped
    and does not depend on the Gaussian's power, so the adjoint drops that pixel's power gradient.
    Random opacities (logits ~ N(0, 1)) almost never get there; this scene makes half the splats
    nearly opaque and large (~11 px on screen), checks that clamped steps are blended, and compares
    the image and every gradient with the FP64 adjoint."""
    g, cam, _ = scenes.tiny_scene(n=60, width=64, height=48, degree=2, seed=11, log_scale=(-0.5, 0.3))
    rng = np.random.default_rng(11)
    opaque = rng.random(g.n) < 0.5
    g.opacity_logits = np.where(opaque, rng.uniform(5.0, 10.0, g.n), g.opacity_logits).astype(np.float32)
    s = R.RasterSettings(tile_size=tile)
    r, params, out, orc = render_both(g, cam, s)
    check_image(orc, out)
    # blended steps at alpha_max, from the oracle's per-pixel traces
    a, b, c = (orc.rec["conic"][:, k] for k in range(3))
    clamped = 0
    for y in range(cam.height):
        for x in range(cam.width):
            _, ids = orc.pixel_trace(x, y)
            if ids.size:
                dx, dy = x - orc.rec["u"][ids], y - orc.rec["v"][ids]
                power = -0.5 * (a[ids] * dx * dx + c[ids] * dy * dy) - b[ids] * dx * dy
                clamped += int((orc.rec["opacity"][ids] * np.exp(power) >= s.alpha_max).sum())
    assert clamped >= 20, clamped
    w = np.random.default_rng(tile).standard_normal((3, cam.height, cam.width)).astype(np.float32)
    w[:, orc.amb.astype(bool)] = 0
    gpu = run_backward(r, params, g, cam, out, w)
    ref = orc.backward(w.astype(np.float64))
    check_grads(gpu, ref, ~(orc.rec["grad_amb"] | orc.rec["rect_amb"]))


# ------------------------------------------------------------------ edge cases

def test_empty_and_fully_culled_inputs():
    g, cam, _ = scenes.tiny_scene(n=20, width=40, height=24, degree=1, seed=9)
    s = R.RasterSettings(bg=(0.3, 0.6, 0.9))
    empty = g.subset(np.arange(0))
    _, _, out = run_forward(empty, cam, s)
    assert np.allclose(out["image"], np.array(s.bg, np.float32)[:, None, None]) and (out["T"] == 1).all()
    assert (out["last"] == 0).all() and out["counters"][B.VG_CNT_PAIRS] == 0
    behind = g.subset(np.arange(g.n))
    behind.means = (np.asarray(cam.cam_pos)[None, :] - 5.0 * np.asarray(cam.R)[2][None, :] +
                    0.01 * np.random.default_rng(0).standard_normal((g.n, 3))).astype(np.float32)
    r, params, out = run_forward(behind, cam, s)
    assert out["counters"][B.VG_CNT_VISIBLE] == 0 and (out["T"] == 1).all()
    gr = run_backward(r, params, behind, cam, out, np.ones((3, 24, 40), np.float32))
    assert all(np.all(v == 0) for v in gr.values())


def test_pair_overflow_is_reported_and_recovered():
    g, cam, _ = scenes.tiny_scene(n=200, width=48, height=40, degree=2, seed=2)
    r0, _, out = run_forward(g, cam, capacity=8, check="defer")
    assert out["counters"][B.VG_CNT_STATUS] & B.VG_STATUS_PAIR_OVERFLOW
    assert out["counters"][B.VG_CNT_PAIRS] > 8
    assert not read_state(r0, g, cam)["ranges"].any()     # nothing sorted: every tile list is empty
    r, _, out2 = run_forward(g, cam, capacity=8, check="sync")
    assert out2["counters"][B.VG_CNT_STATUS] == 0 and r.ws.capacity >= out2["counters"][B.VG_CNT_PAIRS]
    orc = oracle.render(g, cam)
    check_image(orc, out2)


def test_forward_is_deterministic_and_permutation_invariant():
    g, cam, _ = scenes.small_cell(0)
    _, _, a = run_forward(g, cam)
    _, _, b = run_forward(g, cam)
    assert np.array_equal(a["image"], b["image"]) and np.array_equal(a["last"], b["last"])
    perm = np.random.default_rng(1).permutation(g.n)
    r, _, c = run_forward(g.subset(perm), cam)
    # tiles without FP32 depth ties hold the same Gaussians in the same order: bitwise equal
    orc = oracle.render(g, cam)
    tied = np.array([np.any(orc.keys[s + 1:e] == orc.keys[s:e - 1]) for s, e in orc.ranges])
    m = np.repeat(np.repeat((~tied).reshape(8, 8), 16, 0), 16, 1)
    assert np.array_equal(a["image"][:, m], c["image"][:, m])


def test_blend_counts_match_oracle():
    g, cam, _ = scenes.small_cell(0)
    s = R.RasterSettings(count_blends=True)
    _, _, out = run_forward(g, cam, s)
    orc = oracle.render(g, cam)
    ev, bl = int(out["counters"][B.VG_CNT_EVALS]), int(out["counters"][B.VG_CNT_BLENDS])
    # an ambiguous pixel may stop at a different list position: bound by its tile's list length
    lens = (orc.ranges[:, 1] - orc.ranges[:, 0]).reshape(orc.tiles_y, orc.tiles_x)
    per_pix = np.repeat(np.repeat(lens, 16, 0), 16, 1)[:128, :128]
    slack = int(per_pix[orc.amb.astype(bool)].sum())
    assert abs(ev - orc.n_eval) <= slack and abs(bl - orc.n_blend) <= slack


# ------------------------------------------------------------------ loss (Eq. 1)

@pytest.mark.parametrize("H,W", [(75, 100), (37, 33), (1080, 1920)])
def test_loss_l1_dssim_matches_oracle(H, W):
    rng = np.random.default_rng(H)
    x = rng.random((3, H, W)).astype(np.float32)
    y = np.clip(x + 0.2 * rng.standard_normal((3, H, W)), 0, 1).astype(np.float32)
    lossobj = R.LossL1DSSIM(0.2)
    L, G = lossobj(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    torch.cuda.synchronize()
    Lr, Gr = oracle.loss_l1_dssim(x.astype(np.float64), y.astype(np.float64), 0.2)
    assert abs(float(L) - Lr) <= 1e-5 * abs(Lr) + 1e-6
    G = G.cpu().numpy()
    assert np.abs(G - Gr).max() <= 1e-3 * np.abs(Gr).max()
    assert np.linalg.norm(G - Gr) <= 2e-4 * np.linalg.norm(Gr)


def test_loss_autograd_backward_scales_on_the_device():
    # through torch.autograd: the forward takes the loss only, the backward runs the gradient pass
    # scaled by the incoming gradient; it equals the one-call gradient times that scale
    rng = np.random.default_rng(17)
    H, W = 200, 330
    x = torch.from_numpy(rng.random((3, H, W)).astype(np.float32)).cuda().requires_grad_(True)
    y = torch.from_numpy(rng.random((3, H, W)).astype(np.float32)).cuda()
    L = R.l1_dssim_loss(x, y, 0.2)
    (2.5 * L).backward()
    _, G = R.LossL1DSSIM(0.2)(x.detach(), y)
    torch.cuda.synchronize()
    assert torch.allclose(x.grad, 2.5 * G, rtol=1e-6, atol=0.0)
    lossobj = R.LossL1DSSIM(0.2)
    L1 = R.l1_dssim_loss(x, y, 0.2, lossobj)
    R.l1_dssim_loss(x.detach(), y, 0.2, lossobj)       # overwrites the workspace L1 needs
    with pytest.raises(RuntimeError):
        L1.backward()


# ------------------------------------------------------------------ full-size single cell

def _sampled_tiles(tiles_x, tiles_y, k, seed):
    rng = np.random.default_rng(seed)
    t = set(rng.choice(tiles_x * tiles_y, k, replace=False).tolist())
    t |= {0, tiles_x - 1, (tiles_y - 1) * tiles_x, tiles_x * tiles_y - 1, (tiles_y // 2) * tiles_x + tiles_x // 2}
    return sorted(t)


def _full_size_case(g, cam, seed, k_tiles):
    s = R.RasterSettings()
    r, params, out = run_forward(g, cam, s)
    assert out["counters"][B.VG_CNT_STATUS] == 0
    st = read_state(r, g, cam)
    tiles_x, tiles_y = (cam.width + 15) // 16, (cam.height + 15) // 16
    tiles = _sampled_tiles(tiles_x, tiles_y, k_tiles, seed)
    sub = reachable_subset(g, cam, tiles, 16)
    mask = np.zeros(tiles_x * tiles_y, np.uint8)
    mask[tiles] = 1
    orc = oracle.render(g.subset(sub), cam, oracle_opts(s), tile_mask=mask)
    pmask = np.repeat(np.repeat(mask.reshape(tiles_y, tiles_x).astype(bool), 16, 0), 16, 1)[:cam.height, :cam.width]
    check_image(orc, out, mask=pmask)
    # tile lists of the sampled tiles, oracle ids mapped back to the full set
    amb = set(sub[np.nonzero(orc.rec["rect_amb"])[0]].tolist())
    bad = []
    for t in tiles:
        s0, e0 = orc.ranges[t]
        want = [int(sub[i]) for i in orc.vals[s0:e0] if int(sub[i]) not in amb]
        gs, ge = st["ranges"][t]
        got = [int(i) for i in st["ids"][gs:ge] if int(i) not in amb]
        if want != got:
            bad.append(t)
    assert not bad, bad
    # gradients of a random loss restricted to the sampled, unambiguous pixels
    w = np.random.default_rng(seed).standard_normal((3, cam.height, cam.width)).astype(np.float32)
    w[:, ~pmask] = 0
    w[:, orc.amb.astype(bool)] = 0
    gpu = run_backward(r, params, g, cam, out, w)
    ref_sub = orc.backward(w.astype(np.float64))
    outside = np.ones(g.n, bool)
    outside[sub] = False
    for k, v in gpu.items():
        assert np.all(v[outside] == 0), k
    gpu_sub = {k: v[sub] for k, v in gpu.items()}
    keep = ~(orc.rec["grad_amb"] | orc.rec["rect_amb"])
    errs = check_grads(gpu_sub, ref_sub, keep)
    return out, orc, errs


def test_blob_cell_1080p_sampled_parity():
    """1M Gaussians, SH degree 3, 1920x1080 — the benchmark's workload and launch configuration."""
    g, cam, _ = scenes.blob_cell_1080p()
    _full_size_case(g, cam, seed=7, k_tiles=40)
