"""Pins of the CPU oracle against things other than itself (closed forms, an independent
brute-force renderer, library routines, quadrature, finite differences, invariants).

Paper reference: Sec. 3 (projection to 2D Gaussians, tile assignment, depth sort,
front-to-back alpha blending; differentiable rasteriser) and Eq. 1 (L1 + D-SSIM loss).
"""
import math

import numpy as np
import pytest

from paper_2402_17427_gb300 import scenes
from paper_2402_17427_gb300.scenes import Camera, Gaussians


def _cam_identity(W=64, H=64, f=80.0, cx=None, cy=None):
    """Camera at the world origin looking along +z (R = I)."""
    return Camera(W, H, f, f, W / 2 if cx is None else cx, H / 2 if cy is None else cy,
                  np.eye(3, dtype=np.float32), np.zeros(3, np.float32), np.zeros(3, np.float32), 0.2)


def _gauss(means, log_scales, quats, logits, dc_colour, degree=0):
    n = len(means)
    K = (degree + 1) ** 2
    sh = np.zeros((n, K, 3), np.float32)
    Y00 = 0.5 / math.sqrt(math.pi)
    sh[:, 0, :] = (np.asarray(dc_colour, np.float64) - 0.5) / Y00
    return Gaussians(np.asarray(means, np.float32), np.asarray(log_scales, np.float32),
                     np.asarray(quats, np.float32), np.asarray(logits, np.float32), sh, degree)


# ------------------------------------------------------------------ spherical harmonics

def test_sh_orthonormal_by_quadrature(oracle_lib):
    """Gauss-Legendre in cos(theta) x uniform phi integrates degree <= 6 products exactly."""
    zs, wz = np.polynomial.legendre.leggauss(12)
    phis = np.arange(16) * 2 * np.pi / 16
    G = np.zeros((16, 16))
    for z, w in zip(zs, wz):
        s = math.sqrt(1 - z * z)
        for ph in phis:
            Y, _ = oracle_lib.sh_basis(3, [s * math.cos(ph), s * math.sin(ph), z])
            G += np.outer(Y, Y) * w * (2 * np.pi / 16)
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_sh_matches_scipy(oracle_lib):
    from oracle import brute
    rng = np.random.default_rng(3)
    d = rng.standard_normal((50, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    ref = brute.real_sh(3, d)
    got = np.stack([oracle_lib.sh_basis(3, x)[0] for x in d])
    assert np.abs(got - ref).max() < 1e-12
    # degree 0 and the l = 1 band in closed form: Y00 = 1/(2 sqrt pi), (y, z, x) bands with -,+,- signs
    c1 = math.sqrt(3 / (4 * math.pi))
    assert np.allclose(got[:, 0], 0.5 / math.sqrt(math.pi), atol=1e-15)
    assert np.allclose(got[:, 1:4], np.stack([-c1 * d[:, 1], c1 * d[:, 2], -c1 * d[:, 0]], 1), atol=1e-14)


def test_sh_tangential_gradient(oracle_lib):
    rng = np.random.default_rng(4)
    for _ in range(10):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        Y, dY = oracle_lib.sh_basis(3, d)
        tang = dY - np.outer(dY @ d, d)
        h = 1e-6
        for k in range(3):
            e = np.zeros(3); e[k] = h
            yp = oracle_lib.sh_basis(3, (d + e) / np.linalg.norm(d + e))[0]
            ym = oracle_lib.sh_basis(3, (d - e) / np.linalg.norm(d - e))[0]
            assert np.allclose((yp - ym) / (2 * h), tang[:, k], atol=1e-8)


# ------------------------------------------------------------------ closed forms

def test_single_isotropic_gaussian_closed_form(oracle_lib):
    """Head-on isotropic Gaussian: pixel = o c exp(-rho^2 / (2 sigma^2)), sigma^2 = (f s / Z)^2 + 0.3."""
    f, Z, s, o_logit, c = 80.0, 5.0, 0.06, 1.2, (0.9, 0.4, 0.2)
    cam = _cam_identity(64, 64, f)
    g = _gauss([[0, 0, Z]], [[math.log(s)] * 3], [[1, 0, 0, 0]], [o_logit], [c])
    r = oracle_lib.render(g, cam)
    o = 1 / (1 + math.exp(-float(np.float32(o_logit))))      # parameters are stored as float32
    sig2 = (f * math.exp(float(np.float32(math.log(s)))) / Z) ** 2 + 0.3
    rad = 3 * math.sqrt(sig2)
    ys, xs = np.mgrid[0:64, 0:64]
    rho2 = (xs - 32.0) ** 2 + (ys - 32.0) ** 2
    alpha = o * np.exp(-rho2 / (2 * sig2))
    tile_lo, tile_hi = int(math.ceil(32 - rad)) // 16, int(math.floor(32 + rad)) // 16
    in_rect = (xs // 16 >= tile_lo) & (xs // 16 <= tile_hi) & (ys // 16 >= tile_lo) & (ys // 16 <= tile_hi)
    alpha = np.where(in_rect & (alpha >= 1 / 255), np.minimum(alpha, 0.99), 0.0)
    for ch in range(3):
        assert np.abs(r.image[ch] - c[ch] * alpha).max() < 1e-6   # colour c carries float32 rounding
    assert np.abs(r.T - (1 - alpha)).max() < 1e-12
    assert r.n_amb == 0


def test_stacked_gaussians_closed_form(oracle_lib):
    """Three head-on Gaussians: C = c1 a1 + c2 a2 (1 - a1) + c3 a3 (1 - a1)(1 - a2) at the centre."""
    cam = _cam_identity(32, 32, 60.0)
    logits = [0.3, -0.5, 1.0]
    cols = [(1.0, 0.0, 0.25), (0.0, 1.0, 0.5), (0.5, 0.5, 1.0)]
    # listed back to front on purpose: the sort must put depth 3 first
    g = _gauss([[0, 0, 5.0], [0, 0, 4.0], [0, 0, 3.0]], [[-2.0] * 3] * 3, [[1, 0, 0, 0]] * 3,
               logits[::-1], cols[::-1])
    r = oracle_lib.render(g, cam)
    a = [1 / (1 + math.exp(-float(np.float32(l)))) for l in logits]
    Y00 = 0.5 / math.sqrt(math.pi)
    cols32 = [np.maximum(0.0, np.float32((np.array(c) - 0.5) / Y00).astype(np.float64) * Y00 + 0.5)
              for c in cols]
    expect = cols32[0] * a[0] + cols32[1] * a[1] * (1 - a[0]) + cols32[2] * a[2] * (1 - a[0]) * (1 - a[1])
    assert np.abs(r.image[:, 16, 16] - expect).max() < 1e-12
    assert abs(r.T[16, 16] - (1 - a[0]) * (1 - a[1]) * (1 - a[2])) < 1e-14
    Ts, ids = r.pixel_trace(16, 16)
    assert list(ids) == [2, 1, 0]


def test_stop_rules(oracle_lib):
    """Layers of alpha ~0.95: T = 0.05, 2.5e-3, 1.25e-4, then 6.25e-6 < 1e-4 on the fourth.

    Rule 0 leaves the fourth unblended (3 blended); rule 1 blends it and then stops (4).
    """
    cam = _cam_identity(16, 16, 40.0)
    lg = math.log(0.95 / 0.05)
    g = _gauss([[0, 0, 3.0 + k] for k in range(5)], [[-1.0] * 3] * 5, [[1, 0, 0, 0]] * 5, [lg] * 5,
               [(1, 1, 1)] * 5)
    a = 1 / (1 + math.exp(-float(np.float32(lg))))
    r0 = oracle_lib.render(g, cam, oracle_lib.Options(stop_rule=0))
    r1 = oracle_lib.render(g, cam, oracle_lib.Options(stop_rule=1))
    assert r0.last[8, 8] == 3 and abs(r0.T[8, 8] - (1 - a) ** 3) < 1e-15
    assert r1.last[8, 8] == 4 and abs(r1.T[8, 8] - (1 - a) ** 4) < 1e-15


def test_anisotropic_covariance_closed_form(oracle_lib):
    """Rotation about the optical axis by theta: Sigma2 = (f/Z)^2 R2 diag(sx^2, sy^2) R2^T + 0.3 I."""
    f, Z, th = 100.0, 6.0, 0.7
    cam = _cam_identity(64, 64, f)
    ls = np.array([math.log(0.05), math.log(0.12), math.log(0.3)], np.float32)
    q = [math.cos(th / 2), 0, 0, math.sin(th / 2)]
    g = _gauss([[0, 0, Z]], [ls], [q], [0.0], [(0.5, 0.5, 0.5)])
    r = oracle_lib.render(g, cam)
    qf = np.array(q, np.float32).astype(np.float64)
    qf /= np.linalg.norm(qf)
    thf = 2 * math.atan2(qf[3], qf[0])
    R2 = np.array([[math.cos(thf), -math.sin(thf)], [math.sin(thf), math.cos(thf)]])
    s = np.exp(ls.astype(np.float64))
    S2 = (f / Z) ** 2 * R2 @ np.diag(s[:2] ** 2) @ R2.T + 0.3 * np.eye(2)
    conic = np.linalg.inv(S2)
    assert np.allclose(r.rec["conic"][0], [conic[0, 0], conic[0, 1], conic[1, 1]], rtol=1e-12)
    assert abs(r.rec["radius"][0] - 3 * math.sqrt(np.linalg.eigvalsh(S2).max())) < 1e-10


# ------------------------------------------------------------------ brute force

@pytest.mark.parametrize("n,W,H,tile,deg,seed", [(60, 32, 32, 16, 3, 1), (200, 48, 40, 16, 2, 2),
                                                  (120, 40, 24, 8, 1, 3), (80, 33, 35, 16, 0, 4),
                                                  (150, 64, 32, 32, 3, 5)])
def test_matches_brute_force(oracle_lib, n, W, H, tile, deg, seed):
    from oracle import brute
    g, cam, _ = scenes.tiny_scene(n=n, width=W, height=H, degree=deg, seed=seed)
    r = oracle_lib.render(g, cam, oracle_lib.Options(tile=tile))
    assert r.n_amb == 0     # no pixel sits inside a decision band (rect edges included)
    img, T, nbl = brute.render(g, cam, tile=tile)
    assert np.abs(img - r.image).max() < 1e-12
    assert np.abs(T - r.T).max() < 1e-12
    assert int(nbl.sum()) == r.n_blend
    pr = brute.project(g, cam)
    ok = r.rec["valid"]
    assert np.array_equal(ok, pr["ok"])
    assert np.abs(pr["r"][ok] - r.rec["radius"][ok]).max() < 1e-10


def test_keys_sorted_ranges_and_ties(oracle_lib):
    g, cam, _ = scenes.tiny_scene(n=100, width=48, height=48, degree=0, seed=7)
    # force exact depth ties between pairs of Gaussians (same mean, different shapes)
    g.means[1::2] = g.means[0::2]
    r = oracle_lib.render(g, cam)
    k = r.keys
    assert np.all(k[1:] >= k[:-1])
    tiles = (k >> np.uint64(32)).astype(np.int64)
    for t in range(r.ranges.shape[0]):
        s, e = r.ranges[t]
        assert np.all(tiles[s:e] == t)
        ids = r.vals[s:e]
        d = r.keys[s:e] & np.uint64(0xFFFFFFFF)
        tie = d[1:] == d[:-1]
        assert np.all(ids[1:][tie] > ids[:-1][tie])   # equal keys keep ascending index order
    assert r.ranges[:, 1].max() == r.num_pairs
    # every visible Gaussian appears exactly (rect area) times
    rc = r.rec["rect"]
    area = np.where(r.rec["visible"], (rc[:, 1] - rc[:, 0] + 1) * (rc[:, 3] - rc[:, 2] + 1), 0)
    assert np.array_equal(np.bincount(r.vals, minlength=g.n), area)


def _ranges_from_rectangles(r):
    """Tile ranges rebuilt from the visible Gaussians' tile rectangles alone: +1 / -1 at the ends
    of every rectangle row (differences along the tile rows), a prefix sum along each row for the
    per-tile counts, an exclusive scan over the tile ids for the starts; (0, 0) for an empty tile."""
    tx, ty = r.tiles_x, r.tiles_y
    diff = np.zeros((ty, tx + 1), np.int64)
    rc = r.rec["rect"][r.rec["visible"]]
    for tx0, tx1, ty0, ty1 in rc:
        diff[ty0:ty1 + 1, tx0] += 1
        diff[ty0:ty1 + 1, tx1 + 1] -= 1
    counts = np.cumsum(diff[:, :tx], axis=1).ravel()
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    out = np.stack([starts, starts + counts], 1)
    out[counts == 0] = 0
    return out


@pytest.mark.parametrize("case", ["tiny", "small"])
def test_tile_ranges_follow_from_rectangles(oracle_lib, case):
    # a Gaussian's pairs are exactly the tiles of its rectangle, so the ranges of the tile-sorted
    # pair list are fixed before any sort: per-tile counts from the rectangles, scanned over the
    # tile ids in order (what the GPU builds beside its depth sort)
    if case == "tiny":
        g, cam, _ = scenes.tiny_scene(n=300, width=100, height=70, degree=1, seed=11)
    else:
        g, cam, _ = scenes.small_cell(1)
    r = oracle_lib.render(g, cam)
    assert np.array_equal(_ranges_from_rectangles(r), r.ranges.astype(np.int64))
    assert r.ranges[:, 1].max() == r.num_pairs


def _brute_lists(uvrd, W, H, tile):
    """Per tile, by enumeration of its pixel samples: the Gaussians whose closed box
    [u - r, u + r] x [v - r, v + r] (edges rounded to FP32 as computed) contains one of the tile's
    pixels inside the image, ordered by (FP32 depth bits, index)."""
    tx_n, ty_n = (W + tile - 1) // tile, (H + tile - 1) // tile
    u, v, r, d = (uvrd[:, k].astype(np.float32) for k in range(4))
    ok = r >= 0
    x0, x1 = (u - r).astype(np.float32), (u + r).astype(np.float32)
    y0, y1 = (v - r).astype(np.float32), (v + r).astype(np.float32)
    bits = d.view(np.uint32)
    lists = []
    for t in range(tx_n * ty_n):
        ty, tx = divmod(t, tx_n)
        xs = np.arange(tx * tile, min(W, (tx + 1) * tile), dtype=np.float32)
        ys = np.arange(ty * tile, min(H, (ty + 1) * tile), dtype=np.float32)
        hitx = ((xs[None, :] >= x0[:, None]) & (xs[None, :] <= x1[:, None])).any(1)
        hity = ((ys[None, :] >= y0[:, None]) & (ys[None, :] <= y1[:, None])).any(1)
        ids = np.nonzero(ok & hitx & hity)[0]
        lists.append(sorted(ids.tolist(), key=lambda i: (int(bits[i]), i)))
    return lists


@pytest.mark.parametrize("W,H,tile,seed", [(48, 40, 16, 0), (33, 35, 8, 1), (70, 64, 32, 2)])
def test_pairs_from_fp32_matches_per_pixel_enumeration(oracle_lib, W, H, tile, seed):
    # given FP32 decision inputs (as another implementation would report them), the oracle's key
    # generation, stable sort and ranges equal a per-pixel enumeration of each tile; the inputs
    # include edges on pixel centres, rectangles off every image side, culled entries and exact
    # depth ties
    rng = np.random.default_rng(seed)
    n = 160
    u = rng.uniform(-20, W + 20, n).astype(np.float32)
    v = rng.uniform(-20, H + 20, n).astype(np.float32)
    r = rng.uniform(0.0, 14.0, n).astype(np.float32)
    u[:20] = np.round(u[:20])                      # u - r, u + r exactly on pixel samples
    r[:20] = np.round(r[:20])
    r[20:30] = -1.0                                # culled
    d = rng.uniform(0.5, 3.0, n).astype(np.float32)
    d[30:60:2] = d[31:61:2]                        # exact depth ties
    uvrd = np.stack([u, v, r, d], 1)
    keys, ids, ranges = oracle_lib.pairs_from_fp32(uvrd, W, H, tile)
    want = _brute_lists(uvrd, W, H, tile)
    assert ranges[:, 1].max() == len(ids) == sum(len(x) for x in want)
    for t, lst in enumerate(want):
        s, e = ranges[t]
        assert ids[s:e].tolist() == lst, t
        if not lst:
            assert s == e == 0
    assert np.all(keys[1:] >= keys[:-1])


def test_pairs_from_fp32_reproduces_the_forward_lists(oracle_lib):
    # the forward pass's own FP32 decision inputs give back its own lists
    g, cam, _ = scenes.small_cell(0)
    r = oracle_lib.render(g, cam)
    rec = r.rec
    uvrd = np.stack([rec["u32"], rec["v32"], np.where(rec["valid"], rec["r32"], -1.0), rec["depth32"]], 1)
    keys, ids, ranges = oracle_lib.pairs_from_fp32(uvrd, cam.width, cam.height, 16)
    assert np.array_equal(keys, r.keys) and np.array_equal(ids, r.vals)
    assert np.array_equal(ranges, r.ranges)


@pytest.mark.parametrize("case,budget", [("small", 3e-4), ("tiny", 3e-4), ("blob1080p", 5e-4)])
def test_ambiguous_pixel_budget(oracle_lib, case, budget):
    # Pixels whose compositing decision lies inside the FP32 error bands are excluded from the
    # image comparison; their count grows with the number of evaluations times the band width, so
    # it is bounded per pixel: about 2e-4 of the pixels at 1080p (224 evaluations a pixel), none
    # or a few on the small scenes.  The 1e-5 per pixel once proposed for these scenes would need
    # bands below the kernels' measured FP32 decision error.
    if case == "small":
        g, cam, _ = scenes.small_cell(0)
    elif case == "tiny":
        g, cam, _ = scenes.tiny_scene(n=300, width=100, height=61, degree=3, seed=6)
    else:
        g, cam, _ = scenes.blob_cell_1080p()
    r = oracle_lib.render(g, cam)
    px = cam.width * cam.height
    assert r.n_amb <= budget * px + 1, (r.n_amb, px)


# ------------------------------------------------------------------ invariants

def test_transmittance_monotone_and_bounded(oracle_lib):
    g, cam, _ = scenes.small_cell(0)
    r = oracle_lib.render(g, cam)
    assert (r.T >= 0).all() and (r.T <= 1).all()
    rng = np.random.default_rng(0)
    for _ in range(40):
        x, y = rng.integers(0, 128, 2)
        Ts, _ = r.pixel_trace(x, y)
        assert np.all(np.diff(Ts) <= 0) and (len(Ts) == 0 or Ts[-1] >= 1e-4)


def test_permutation_invariance(oracle_lib):
    g, cam, _ = scenes.small_cell(0)
    r = oracle_lib.render(g, cam)
    perm = np.random.default_rng(1).permutation(g.n)
    r2 = oracle_lib.render(g.subset(perm), cam)
    # Equal FP32 depths in one tile are ordered by input index, so only tie-free tiles must agree.
    tied = np.zeros(r.ranges.shape[0], bool)
    for t, (s, e) in enumerate(r.ranges):
        d = r.keys[s:e]
        tied[t] = np.any(d[1:] == d[:-1])
    assert tied.sum() <= 2
    mask = np.repeat(np.repeat((~tied).reshape(8, 8), 16, 0), 16, 1)
    assert np.abs(r.image - r2.image)[:, mask].max() < 1e-12
    inv = np.argsort(perm)
    w = np.broadcast_to(mask, (3, 128, 128)).astype(np.float64)
    gr = r.backward(w)
    gr2 = r2.backward(w)
    assert np.abs(gr["means"] - gr2["means"][inv]).max() < 1e-9 * (1 + np.abs(gr["means"]).max())


def test_tile_mask_renders_subset(oracle_lib):
    g, cam, _ = scenes.small_cell(0)
    full = oracle_lib.render(g, cam)
    mask = np.zeros(64, np.uint8)
    mask[[0, 9, 27, 63]] = 1
    part = oracle_lib.render(g, cam, tile_mask=mask)
    for t in np.nonzero(mask)[0]:
        ty, tx = divmod(int(t), 8)
        sl = np.s_[:, ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16]
        assert np.array_equal(full.image[sl], part.image[sl])


# ------------------------------------------------------------------ adjoint

def _fd_check(oracle_lib, g, cam, weights, opts=None, per_group=40, seed=0):
    sc = oracle_lib.Scene64.of(g)
    opts = opts or oracle_lib.Options()
    r0 = oracle_lib.render(sc, cam, opts)
    grads = r0.backward(weights)
    rng = np.random.default_rng(seed)
    names = ["means", "log_scales", "quats", "logits", "sh"]
    report = {}
    for name, P in zip(names, sc.params()):
        G = grads[name].reshape(-1)
        flat = P.reshape(-1)
        gmax = np.abs(G).max()
        used = 0
        for j in rng.choice(flat.size, min(flat.size, per_group), replace=False):
            x0 = flat[j]
            h = 1e-6 * max(1.0, abs(x0))
            flat[j] = x0 + h
            rp = oracle_lib.render(sc, cam, opts)
            flat[j] = x0 - h
            rm = oracle_lib.render(sc, cam, opts)
            flat[j] = x0
            if rp.decision_hash != r0.decision_hash or rm.decision_hash != r0.decision_hash:
                continue          # the perturbation crosses a threshold: no derivative there
            fd = ((rp.image * weights).sum() - (rm.image * weights).sum()) / (2 * h)
            assert abs(fd - G[j]) <= 1e-6 * abs(G[j]) + 1e-8 * gmax + 1e-12, (name, j, fd, G[j])
            used += 1
        report[name] = used
    return report


@pytest.mark.parametrize("seed,deg", [(2, 3), (5, 1)])
def test_adjoint_matches_central_differences(oracle_lib, seed, deg):
    g, cam, _ = scenes.tiny_scene(n=30, width=32, height=32, degree=deg, seed=seed)
    w = np.random.default_rng(seed).standard_normal((3, 32, 32))
    rep = _fd_check(oracle_lib, g, cam, w)
    assert all(v >= 20 for k, v in rep.items() if k != "logits") and rep["logits"] >= 15


def _group_dirs(rng, sc, ids, group):
    """One direction per target over one parameter group (random signs, scaled by max(1, |theta|)),
    in the raw-parameter layout mean 3, log-scale 3, quaternion 4, logit 1, SH 3K."""
    F = 11 + 3 * sc.K
    spans = {"means": (0, 3), "log_scales": (3, 6), "quats": (6, 10), "logits": (10, 11), "sh": (11, F)}
    a, b = spans[group]
    dirs = np.zeros((len(ids), F))
    flat = np.concatenate([sc.means, sc.log_scales, sc.quats, sc.logits[:, None], sc.sh.reshape(sc.n, -1)], 1)
    dirs[:, a:b] = rng.choice([-1.0, 1.0], (len(ids), b - a)) * np.maximum(1.0, np.abs(flat[ids, a:b]))
    return dirs


def test_tile_local_differences_equal_full_renders_and_the_adjoint(oracle_lib):
    # re-rendering only the perturbed Gaussian's tiles gives the full loss difference (every other
    # pixel is unchanged), and the directional derivative equals the adjoint's
    g, cam, _ = scenes.tiny_scene(n=60, width=64, height=48, degree=2, seed=13)
    sc = oracle_lib.Scene64.of(g)
    r0 = oracle_lib.render(sc, cam)
    w = np.random.default_rng(3).standard_normal((3, 48, 64))
    grads = r0.backward(w)
    rng = np.random.default_rng(4)
    vis = np.nonzero(r0.rec["visible"])[0]
    ids = rng.choice(vis, min(12, len(vis)), replace=False)
    eps = 1e-6
    flat_names = ["means", "log_scales", "quats", "logits", "sh"]
    used = 0
    for group in flat_names:
        dirs = _group_dirs(rng, sc, ids, group)
        fd, flags = r0.fd_directional(w, ids, dirs, eps)
        G = np.concatenate([grads["means"], grads["log_scales"], grads["quats"], grads["logits"][:, None],
                            grads["sh"].reshape(sc.n, -1)], 1)
        for k, i in enumerate(ids):
            if flags[k]:
                continue
            # the same difference from two full renders of the perturbed scene
            full = []
            for e in (eps, -eps):
                sp = oracle_lib.Scene64(sc.means.copy(), sc.log_scales.copy(), sc.quats.copy(), sc.logits.copy(),
                                        sc.sh.copy(), sc.sh_degree)
                d = dirs[k]
                sp.means[i] += e * d[0:3]
                sp.log_scales[i] += e * d[3:6]
                sp.quats[i] += e * d[6:10]
                sp.logits[i] += e * d[10]
                sp.sh[i] += e * d[11:].reshape(sc.K, 3)
                full.append((oracle_lib.render(sp, cam).image * w).sum())
            fd_full = (full[0] - full[1]) / (2 * eps)
            assert abs(fd[k] - fd_full) <= 1e-7 * (abs(fd_full) + 1.0), (group, i, fd[k], fd_full)
            an = float(G[i] @ dirs[k])
            assert abs(fd[k] - an) <= 1e-6 * (abs(an) + np.abs(G[i] * dirs[k]).sum()) + 1e-9, (group, i, fd[k], an)
            used += 1
    assert used >= 40


def test_adjoint_guard_band_and_white_background(oracle_lib):
    """Gaussians near/outside the image edge exercise the clamped Jacobian; bg != 0."""
    g, cam, _ = scenes.tiny_scene(n=40, width=32, height=32, degree=2, seed=11, box=2.5, dist=3.0)
    w = np.random.default_rng(1).standard_normal((3, 32, 32))
    _fd_check(oracle_lib, g, cam, w, oracle_lib.Options(bg=(1.0, 0.5, 0.2)), per_group=30)


def test_opacity_derivative_closed_form(oracle_lib):
    """Single head-on Gaussian: d pixel / d opacity = c exp(-rho^2 / (2 sigma^2))."""
    f, Z, s = 80.0, 5.0, 0.06
    cam = _cam_identity(64, 64, f)
    g = _gauss([[0, 0, Z]], [[math.log(s)] * 3], [[1, 0, 0, 0]], [0.2], [(0.7, 0.3, 0.1)])
    r = oracle_lib.render(g, cam)
    dimg = np.zeros((3, 64, 64))
    dimg[0, 32, 33] = 1.0
    gr = r.backward(dimg)
    sig2 = (f * math.exp(float(np.float32(math.log(s)))) / Z) ** 2 + 0.3
    rho2 = (33 - 32.0) ** 2
    assert abs(gr["g2d"][0, 5] - r.rec["rgb"][0, 0] * math.exp(-rho2 / (2 * sig2))) < 1e-12


def test_abs_gradient_statistic(oracle_lib):
    """The densification statistic sums |dL/du| + |dL/dv| of each pixel's own contribution.  With
    dL non-zero at one pixel each Gaussian has one such term, so the statistic equals |du| + |dv|
    of the adjoint (which the finite-difference pins cover); in general it is at least that
    (triangle inequality), with equality only where every pixel's terms share their signs."""
    g, cam, _ = scenes.tiny_scene(n=60, width=40, height=32, degree=1, seed=3)
    r = oracle_lib.render(g, cam)
    one = np.zeros((3, 32, 40))
    one[1, 17, 22] = 1.0
    gr = r.backward(one)
    assert np.abs(gr["g2d_abs"] - (np.abs(gr["g2d"][:, 0]) + np.abs(gr["g2d"][:, 1]))).max() < 1e-12
    assert (gr["g2d_abs"] > 0).sum() >= 2
    w = np.random.default_rng(3).standard_normal((3, 32, 40))
    gr = r.backward(w)
    lower = np.abs(gr["g2d"][:, 0]) + np.abs(gr["g2d"][:, 1])
    assert (gr["g2d_abs"] >= lower - 1e-12).all()
    assert (gr["g2d_abs"] > lower * (1 + 1e-6)).any()       # cancellation across pixels happens
    assert (gr["g2d_abs"][~r.rec["visible"]] == 0).all()


def test_alpha_clamp_closed_form(oracle_lib):
    """Single head-on Gaussian with opacity near 1: at the centre pixel alpha = min(0.99, o) = 0.99,
    so the pixel is 0.99 c and does not depend on the opacity, the mean or the conic (their
    derivatives are exactly 0 there; d pixel / d rgb = 0.99); 4 px away alpha < 0.99 and
    d pixel / d opacity = c exp(-rho^2 / (2 sigma^2)) as without the clamp."""
    f, Z, s = 80.0, 5.0, 0.19
    cam = _cam_identity(64, 64, f)
    g = _gauss([[0, 0, Z]], [[math.log(s)] * 3], [[1, 0, 0, 0]], [8.0], [(0.7, 0.3, 0.1)])
    r = oracle_lib.render(g, cam)
    c = r.rec["rgb"][0, 0]
    assert r.rec["opacity"][0] > 0.999
    assert abs(r.image[0, 32, 32] - 0.99 * c) < 1e-12
    dimg = np.zeros((3, 64, 64))
    dimg[0, 32, 32] = 1.0
    g2d = r.backward(dimg)["g2d"][0]
    assert np.all(g2d[:6] == 0.0), g2d            # du, dv, d conic (3), d opacity
    assert abs(g2d[6] - 0.99) < 1e-12 and g2d[7] == 0.0 and g2d[8] == 0.0
    dimg[0, 32, 32] = 0.0
    dimg[0, 32, 36] = 1.0
    sig2 = (f * math.exp(float(np.float32(math.log(s)))) / Z) ** 2 + 0.3
    G = math.exp(-16.0 / (2 * sig2))
    assert r.rec["opacity"][0] * G < 0.99
    g2d = r.backward(dimg)["g2d"][0]
    assert abs(g2d[5] - c * G) < 1e-12


# ------------------------------------------------------------------ loss (Eq. 1)

def test_ssim_identity_and_scipy(oracle_lib):
    from oracle import brute
    rng = np.random.default_rng(0)
    x = rng.random((3, 20, 27))
    y = rng.random((3, 20, 27))
    assert abs(oracle_lib.ssim(x, x) - 1.0) < 1e-12
    assert abs(oracle_lib.ssim(x, y) - brute.ssim(x, y)) < 1e-12
    L = oracle_lib.loss_l1_dssim(x, x, 0.2, grad=False)
    assert abs(L) < 1e-12


def test_ssim_constant_images_closed_form(oracle_lib):
    a, b = 0.3, 0.8
    x = np.full((3, 30, 30), a)
    y = np.full((3, 30, 30), b)
    m = oracle_lib.ssim_map(x, y)
    C1 = 0.01 ** 2
    assert abs(m[0, 15, 15] - (2 * a * b + C1) / (a * a + b * b + C1)) < 1e-12
    # at a corner the zero-padded window covers a fraction s of its mass
    w = np.exp(-((np.arange(11) - 5.0) ** 2) / 4.5); w /= w.sum()
    sfr = w[5:].sum() ** 2
    C2 = 0.03 ** 2
    e = ((2 * a * b * sfr ** 2 + C1) * (2 * a * b * sfr * (1 - sfr) + C2) /
         (((a * a + b * b) * sfr ** 2 + C1) * ((a * a + b * b) * sfr * (1 - sfr) + C2)))
    assert abs(m[0, 0, 0] - e) < 1e-12


def test_loss_gradient_central_differences(oracle_lib):
    rng = np.random.default_rng(5)
    x = rng.random((3, 17, 23))
    y = rng.random((3, 17, 23))
    L, G = oracle_lib.loss_l1_dssim(x, y, 0.2)
    l1 = np.abs(x - y).mean()
    assert abs(L - (0.8 * l1 + 0.2 * (1 - oracle_lib.ssim(x, y)))) < 1e-13
    for _ in range(40):
        c, i, j = rng.integers(0, 3), rng.integers(0, 17), rng.integers(0, 23)
        h = 1e-5
        if abs(x[c, i, j] - y[c, i, j]) < 4 * h:
            continue                        # the L1 kink lies inside the stencil
        x[c, i, j] += h
        Lp = oracle_lib.loss_l1_dssim(x, y, 0.2, grad=False)
        x[c, i, j] -= 2 * h
        Lm = oracle_lib.loss_l1_dssim(x, y, 0.2, grad=False)
        x[c, i, j] += h
        assert abs((Lp - Lm) / (2 * h) - G[c, i, j]) < 1e-6 * abs(G[c, i, j]) + 1e-10
