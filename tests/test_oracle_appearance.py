"""Pins of the appearance-model oracle (paper Sec. 4.2, Eq. 2-3, and the CNN of the supplementary
material).

Every operator is checked against something other than itself: the convolution against brute
force on a tiny input, the pixel shuffle, bilinear up-sampling and 32x average pooling against
their PyTorch library counterparts (FP64, CPU), every adjoint against the dot-product identity,
the whole model against a PyTorch composition with autograd, the full loss gradient against
central finite differences, and the special case M = 1 against the loss of Eq. 1.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
from oracle import appearance as OA


def test_conv_matches_brute_force():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 5, 4))
    w = rng.standard_normal((2, 3, 3, 3))
    b = rng.standard_normal(2)
    y = OA.conv(x, w, b)
    for o in range(2):
        for yy in range(5):
            for xx in range(4):
                s = b[o]
                for c in range(3):
                    for i in range(3):
                        for j in range(3):
                            sy, sx = yy + i - 1, xx + j - 1
                            if 0 <= sy < 5 and 0 <= sx < 4:
                                s += w[o, c, i, j] * x[c, sy, sx]
                assert y[o, yy, xx] == pytest.approx(s, abs=1e-12)


def test_operators_match_pytorch():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((8, 6, 7))
    w = rng.standard_normal((5, 8, 3, 3))
    b = rng.standard_normal(5)
    t = torch.from_numpy
    assert np.allclose(OA.conv(x, w, b), F.conv2d(t(x)[None], t(w), t(b), padding=1)[0].numpy(), atol=1e-12)
    assert np.array_equal(OA.shuffle(x), F.pixel_shuffle(t(x)[None], 2)[0].numpy())
    assert np.array_equal(OA.unshuffle(OA.shuffle(x)), x)
    for H, W in [(13, 17), (12, 14), (40, 9)]:
        ref = F.interpolate(t(x)[None], size=(H, W), mode="bilinear", align_corners=False)[0].numpy()
        assert np.allclose(OA.bilinear(x, H, W), ref, atol=1e-12)
    img = rng.random((3, 70, 100))
    assert np.allclose(OA.pool32(img), F.avg_pool2d(t(img)[None], 32)[0].numpy(), atol=1e-14)


def test_shuffle_follows_its_definition():
    x = np.arange(8 * 2 * 3, dtype=np.float64).reshape(8, 2, 3)
    y = OA.shuffle(x)
    for c4 in range(8):
        c, r = divmod(c4, 4)
        i, j = divmod(r, 2)
        for yy in range(2):
            for xx in range(3):
                assert y[c, 2 * yy + i, 2 * xx + j] == x[c4, yy, xx]


def test_bilinear_reproduces_linear_maps():
    # bilinear interpolation of a map that is affine in (x, y) is that affine map at the mapped
    # coordinates, wherever no clamp applies
    h, w, H, W = 9, 11, 20, 23
    ys, xs = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    f = (2.0 + 0.5 * xs - 0.25 * ys)[None]
    up = OA.bilinear(f, H, W)[0]
    sy = (np.arange(H) + 0.5) * h / H - 0.5
    sx = (np.arange(W) + 0.5) * w / W - 0.5
    inner = (sy >= 0) & (sy <= h - 1)
    innx = (sx >= 0) & (sx <= w - 1)
    expect = 2.0 + 0.5 * sx[None, :] - 0.25 * sy[:, None]
    assert np.allclose(up[np.ix_(inner, innx)], expect[np.ix_(inner, innx)], atol=1e-12)
    assert np.allclose(OA.bilinear(np.full((2, h, w), 3.5), H, W), 3.5, atol=1e-14)


def test_adjoints_satisfy_the_dot_product_identity():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((6, 9, 10))
    w = rng.standard_normal((4, 6, 3, 3))
    g = rng.standard_normal((4, 9, 10))
    zero = np.zeros(4)
    dx, dw, db = OA.conv_adj(x, w, g)
    lhs = np.sum(OA.conv(x, w, zero) * g)
    assert lhs == pytest.approx(np.sum(x * dx), rel=1e-12)
    assert lhs == pytest.approx(np.sum(w * dw), rel=1e-12)
    assert np.allclose(db, g.sum(axis=(1, 2)))
    gu = rng.standard_normal((6, 21, 17))
    assert np.sum(OA.bilinear(x, 21, 17) * gu) == pytest.approx(np.sum(x * OA.bilinear_adj(gu, 9, 10)), rel=1e-12)
    img = rng.standard_normal((3, 70, 100))
    gp = rng.standard_normal((3, 2, 3))
    assert np.sum(OA.pool32(img) * gp) == pytest.approx(np.sum(img * OA.pool32_adj(gp, 70, 100)), rel=1e-12)


def _torch_model(img, target, emb, weights, lam):
    """The same model written with PyTorch modules (FP64, autograd); the D-SSIM term is left out."""
    t = lambda a: torch.tensor(a, dtype=torch.float64, requires_grad=True)
    I, E = t(img), t(emb)
    Ws = [(t(w), t(b)) for w, b in weights]
    H, W = img.shape[1:]
    p = F.avg_pool2d(I[None], 32)
    D = torch.cat([p, E[None, :, None, None].expand(1, 64, p.shape[2], p.shape[3])], 1)
    a = F.conv2d(D, *Ws[0], padding=1)
    for k in range(1, 5):
        a = F.relu(F.conv2d(F.pixel_shuffle(a, 2), *Ws[k], padding=1))
    u = F.interpolate(a, size=(H, W), mode="bilinear", align_corners=False)
    M = F.conv2d(F.relu(F.conv2d(u, *Ws[5], padding=1)), *Ws[6], padding=1)[0]
    L = (1 - lam) * (I * M - torch.from_numpy(target)).abs().mean()
    L.backward()
    return L.item(), M.detach().numpy(), I.grad.numpy(), E.grad.numpy(), [(w.grad.numpy(), b.grad.numpy()) for w, b in Ws]


@pytest.fixture(scope="module")
def case():
    rng = np.random.default_rng(3)
    H, W = 70, 100                     # 2 x 3 cells of 32 x 32; 6 rows and 4 columns left over
    img = rng.random((3, H, W))
    target = rng.random((3, H, W))
    emb = rng.normal(0, 1, 64)
    weights = OA.init_weights(rng)
    return img, target, emb, weights


def test_model_and_gradients_match_pytorch_autograd(case):
    img, target, emb, weights = case
    lam = 0.2
    L, M, gi, ge, gw = OA.loss_and_grads(img, target, emb, weights, lam)
    Lt, Mt, git, get, gwt = _torch_model(img, target, emb, weights, lam)
    dssim, gs = oracle.loss_l1_dssim(img, target, 1.0)
    assert np.allclose(M, Mt, atol=1e-12)
    assert L == pytest.approx(Lt + lam * dssim, rel=1e-12)
    assert np.allclose(gi, git + lam * gs, atol=1e-14)
    assert np.allclose(ge, get, rtol=1e-10, atol=1e-16)
    for (dw, db), (dwt, dbt) in zip(gw, gwt):
        assert np.allclose(dw, dwt, rtol=1e-10, atol=1e-16)
        assert np.allclose(db, dbt, rtol=1e-10, atol=1e-16)


def test_gradients_match_central_differences(case):
    img, target, emb, weights = case
    lam = 0.2
    L, M, gi, ge, gw = OA.loss_and_grads(img, target, emb, weights, lam)
    loss = lambda im, e, ws: OA.loss_and_grads(im, target, e, ws, lam)[0]
    h = 1e-6
    rng = np.random.default_rng(4)

    def check(analytic, bump):
        num = (bump(h) - bump(-h)) / (2 * h)
        assert analytic == pytest.approx(num, rel=2e-4, abs=1e-9)

    for _ in range(6):
        c, y, x = rng.integers(3), rng.integers(64), rng.integers(96)    # inside the pooled cells

        def bump(d, c=c, y=y, x=x):
            im = img.copy()
            im[c, y, x] += d
            return loss(im, emb, weights)
        check(gi[c, y, x], bump)
    for k in rng.choice(64, 4, replace=False):
        check(ge[k], lambda d, k=k: loss(img, emb + d * np.eye(64)[k], weights))
    for layer in range(7):
        w, b = weights[layer]
        idx = tuple(rng.integers(s) for s in w.shape)

        def bump_w(d, layer=layer, idx=idx):
            ws = [(a.copy(), bb.copy()) for a, bb in weights]
            ws[layer][0][idx] += d
            return loss(img, emb, ws)

        def bump_b(d, layer=layer):
            ws = [(a.copy(), bb.copy()) for a, bb in weights]
            ws[layer][1][0] += d
            return loss(img, emb, ws)
        check(gw[layer][0][idx], bump_w)
        check(gw[layer][1][0], bump_b)


def test_identity_map_reduces_to_eq1(case):
    # with the last convolution zero and its bias 1, M = 1 and Eq. 3 is Eq. 1
    img, target, emb, weights = case
    ws = [(w.copy(), b.copy()) for w, b in weights]
    ws[6] = (np.zeros_like(ws[6][0]), np.ones(3))
    L, M, gi, ge, gw = OA.loss_and_grads(img, target, emb, ws, 0.2)
    L1, g1 = oracle.loss_l1_dssim(img, target, 0.2)
    assert np.array_equal(M, np.ones_like(M))
    assert L == pytest.approx(L1, rel=1e-12)
    assert np.allclose(gi, g1, atol=1e-15)
    assert np.all(ge == 0) and all(np.all(dw == 0) for dw, _ in gw[:6])
