"""GPU parity of the colour-corrected evaluation (paper Sec. 5.1 metrics) against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import evaluate as OE
from paper_2402_17427_gb300 import rasterize as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2402_17427_gb300 import _build
    _build.build()
    import oracle
    oracle.build()
    assert torch.cuda.is_available()


def _run(x, y):
    out = R.color_corrected_metrics(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("H,W", [(270, 480), (37, 53)])
def test_corrected_metrics_match_oracle(H, W):
    rng = np.random.default_rng(H)
    y = rng.uniform(0, 1, (3, H, W)).astype(np.float32)
    A = np.array([[0.8, 0.1, 0.0], [0.05, 1.1, -0.1], [0.0, 0.2, 0.7]])
    x = np.clip((A @ y.reshape(3, -1)).reshape(y.shape) + 0.05 + 0.05 * rng.standard_normal(y.shape), 0, 1)
    x = x.astype(np.float32)
    out = _run(x, y)
    c, Ar, br = OE.color_correct(x, y)
    p_ref = OE.psnr(c, y)
    import oracle
    s_ref = oracle.ssim(c, y)
    assert abs(out[0] - p_ref) <= 1e-3, (out[0], p_ref)
    assert abs(out[1] - s_ref) <= 2e-5, (out[1], s_ref)
    assert np.allclose(out[2:11].reshape(3, 3), Ar, rtol=1e-4, atol=1e-5)
    assert np.allclose(out[11:14], br, rtol=1e-4, atol=1e-5)


def test_exactly_affine_rendering_is_corrected_to_the_truth():
    rng = np.random.default_rng(7)
    y = rng.uniform(0.1, 0.9, (3, 64, 96)).astype(np.float32)
    x = (0.5 * y + 0.2).astype(np.float32)
    out = _run(x, y)
    assert out[1] == pytest.approx(1.0, abs=1e-5) and out[0] > 60.0


def test_constant_rendering_fits_the_channel_means():
    rng = np.random.default_rng(8)
    y = rng.uniform(0, 1, (3, 40, 40)).astype(np.float32)
    x = np.full_like(y, 0.3)
    out = _run(x, y)
    c, _, _ = OE.color_correct(x, y)
    assert abs(out[0] - OE.psnr(c, y)) <= 1e-3
