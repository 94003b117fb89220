"""GPU parity of the decoupled appearance model (paper Sec. 4.2, Eq. 3, and the CNN of the
supplementary material) against the FP64 appearance oracle, through the C ABI.

Tolerances are those of FP32 arithmetic, which is what the method runs in.  The tensor-core
convolutions split every FP32 operand into two TF32 parts and form each product from three MMAs,
so products carry a relative error of about 2^-21 and accumulate in FP32; the other layers are
plain FP32.  The map M is held to 1e-4 of its range, the loss to 1e-5 relative, and every gradient
group (the embedding, each layer's weights and biases) to a relative L2 error of 2e-3 against the
FP64 oracle, with no allowance for reduced-precision operands.  The L1 term's sign is a decision
taken in floating point: where |I_r M - I| is within twice the map's bound the two sides may
legitimately differ, so dL/dI_r must agree element-wise (within 2e-3 of its scale) everywhere
except at such pixels.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import appearance as OA
from paper_2402_17427_gb300 import appearance as AP
from paper_2402_17427_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2402_17427_gb300 import _build
    _build.build()
    oracle.build()
    assert torch.cuda.is_available()


def _case(W, H, seed):
    """Seeded inputs: a smooth rendering with noise, an independent target, an embedding and a
    fan-in scaled CNN whose last bias is near 1 (so M stays near 1, as in training)."""
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.linspace(0, 1, H), np.linspace(0, 1, W), indexing="ij")
    base = np.stack([0.5 + 0.3 * np.sin(6 * xx + c) * np.cos(4 * yy - c) for c in range(3)])
    img = np.clip(base + 0.1 * rng.standard_normal((3, H, W)), 0, 1).astype(np.float32)
    target = np.clip(base * 0.9 + 0.05 + 0.1 * rng.standard_normal((3, H, W)), 0, 1).astype(np.float32)
    emb = rng.normal(0, 1, 64).astype(np.float32)
    weights = OA.init_weights(rng)
    weights[6] = (weights[6][0] * 0.5, 1.0 + 0.05 * rng.standard_normal(3))
    weights = [(w.astype(np.float32), b.astype(np.float32)) for w, b in weights]
    return img, target, emb, weights


def _flat(weights):
    return np.concatenate([np.concatenate([w.ravel(), b]) for w, b in weights]).astype(np.float32)


def _gpu(img, target, emb, weights, lam, grad=True):
    model = AP.AppearanceModel(1)
    model.params.copy_(torch.from_numpy(_flat(weights)))
    model.embeddings[0].copy_(torch.from_numpy(emb))
    out = model.loss(torch.from_numpy(img).cuda(), torch.from_numpy(target).cuda(), 0, lam, grad=grad, want_map=True)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _compare(W, H, seed, lam=0.2):
    img, target, emb, weights = _case(W, H, seed)
    g = _gpu(img, target, emb, weights, lam)
    w64 = [(w.astype(np.float64), b.astype(np.float64)) for w, b in weights]
    e64 = emb.astype(np.float64)
    L, M, gi, ge, gw = OA.loss_and_grads(img, target, e64, w64, lam)
    # the map and the loss
    span = M.max() - M.min()
    assert np.abs(g["map"] - M).max() <= 1e-4 * span, np.abs(g["map"] - M).max() / span
    assert g["loss"][0] == pytest.approx(L, rel=1e-5)
    # the gradient of the image, element-wise where the L1 sign is settled
    d = img.astype(np.float64) * M - target
    settled = np.abs(d) > 2e-4 * span
    scale = np.abs(gi).max()
    off = np.abs(g["grad_img"] - gi) > 2e-3 * scale
    assert not (off & settled).any()           # any disagreement is at a pixel whose sign is unsettled
    assert off.mean() <= (~settled).mean()
    # the embedding and every layer's weight and bias gradients
    errs = {"embedding": _rel(g["grad_embedding"], ge)}
    views = AP.layer_views(torch.from_numpy(g["grad_params"]))
    for k, ((gw_gpu, gb_gpu), (dw, db)) in enumerate(zip(views, gw)):
        if np.linalg.norm(dw) > 0:
            errs[f"w{k}"] = _rel(gw_gpu.numpy(), dw)
        if np.linalg.norm(db) > 0:
            errs[f"b{k}"] = _rel(gb_gpu.numpy(), db)
    assert max(errs.values()) <= 2e-3, errs
    return g


@pytest.mark.parametrize("W,H,seed", [(100, 70, 0), (330, 200, 1), (64, 32, 2), (47, 33, 6), (257, 129, 7)])
def test_appearance_matches_oracle(W, H, seed):
    # (100, 70): 3 x 2 pooled cells, 6 rows and 4 columns outside them, ragged head M-tiles
    # (16 x 8 pixels); (330, 200): 10 x 6 cells; (64, 32): the smallest shapes (1 x 2 cells);
    # (47, 33): one cell, up-sampling 16 -> 33 rows and 16 -> 47 columns (factors 2.06 and 2.94),
    # partial M-tiles on both edges; (257, 129): odd sizes, a last M-tile column of one pixel
    _compare(W, H, seed)


@pytest.mark.parametrize("lam", [0.0, 1.0])
def test_appearance_lambda_extremes(lam):
    # lambda = 0: L1 on I_a alone (no D-SSIM term); lambda = 1: D-SSIM on I_r alone, so the CNN
    # receives no gradient at all
    g = _compare(100, 70, 5, lam)
    if lam == 1.0:
        assert not g["grad_params"].any() and not g["grad_embedding"].any()


def test_appearance_full_size_matches_oracle():
    # the 1920 x 1080 training view the benchmark times
    _compare(1920, 1080, 3)


def test_forward_only_and_identity_map():
    img, target, emb, weights = _case(200, 96, 4)
    full = _gpu(img, target, emb, weights, 0.2)
    fwd = _gpu(img, target, emb, weights, 0.2, grad=False)
    assert np.array_equal(full["map"], fwd["map"]) and full["loss"][0] == fwd["loss"][0]
    # M = 1 (last convolution zero, bias 1): Eq. 3 is Eq. 1, and dL/dI_r is Eq. 1's gradient
    weights[6] = (np.zeros_like(weights[6][0]), np.ones(3, np.float32))
    g = _gpu(img, target, emb, weights, 0.2)
    assert np.array_equal(g["map"], np.ones_like(g["map"]))
    H, W = img.shape[1:]
    need = B.vg_loss_workspace_bytes(W, H)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    loss = torch.empty(1, device="cuda")
    grad = torch.empty(3, H, W, device="cuda")
    x, y = torch.from_numpy(img).cuda(), torch.from_numpy(target).cuda()
    B.vg_loss_l1_dssim(x.data_ptr(), y.data_ptr(), W, H, 0.2, ws.data_ptr(), need, loss.data_ptr(), grad.data_ptr(),
                       torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert g["loss"][0] == pytest.approx(loss.item(), rel=1e-6)
    assert np.array_equal(g["grad_img"], grad.cpu().numpy())
    assert not g["grad_embedding"].any()
    assert not g["grad_params"][:AP.param_count() - (3 * 16 * 9 + 3)].any()


def test_appearance_rejects_bad_arguments():
    assert B.vg_appearance_workspace_bytes(31, 100) == 0 and B.vg_appearance_workspace_bytes(100, 16385) == 0
    assert B.vg_appearance_param_count() == AP.param_count() == 255539
    dev = torch.zeros(16, device="cuda")
    p = dev.data_ptr()
    with pytest.raises(B.VGError):      # image too small
        B.vg_appearance_loss(p, p, 16, 64, p, p, 0.2, p, 1 << 30, p, None, None, None, None, 0)
    with pytest.raises(B.VGError):      # gradient pointers partly given
        B.vg_appearance_loss(p, p, 64, 64, p, p, 0.2, p, 1 << 30, p, None, p, None, p, 0)
    with pytest.raises(B.VGError):      # workspace too small
        B.vg_appearance_loss(p, p, 64, 64, p, p, 0.2, p, 16, p, None, None, None, None, 0)
    with pytest.raises(B.VGError):      # lambda outside [0, 1]
        B.vg_appearance_loss(p, p, 64, 64, p, p, 1.5, p, 1 << 30, p, None, None, None, None, 0)
