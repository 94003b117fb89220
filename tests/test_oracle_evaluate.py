"""Pins of the colour-corrected evaluation oracle (paper Sec. 5.1, metrics after a per-image
least-squares colour alignment)."""
import numpy as np
import pytest

from oracle import evaluate as OE


def test_correction_recovers_a_known_affine_map():
    rng = np.random.default_rng(0)
    y = rng.uniform(0.2, 0.8, (3, 40, 50))
    A = np.array([[1.2, 0.1, -0.05], [0.0, 0.9, 0.1], [0.05, -0.1, 1.1]])
    b = np.array([0.02, -0.03, 0.01])
    # the rendering is the inverse map of the truth: correcting it must give the truth back
    x = (np.linalg.inv(A) @ (y.reshape(3, -1) - b[:, None])).reshape(y.shape)
    c, Ah, bh = OE.color_correct(x, y)
    assert np.allclose(Ah, A, atol=1e-10) and np.allclose(bh, b, atol=1e-10)
    assert np.abs(c - y).max() < 1e-10


def test_psnr_closed_form_and_clipping():
    y = np.zeros((3, 8, 8))
    x = np.full((3, 8, 8), 0.1)
    assert OE.psnr(x, y) == pytest.approx(20.0)          # mse 0.01
    # a constant rendering cannot explain a varying target: the fit is the per-channel mean
    rng = np.random.default_rng(1)
    t = rng.uniform(0, 1, (3, 16, 16))
    c, _, _ = OE.color_correct(np.full_like(t, 0.3), t)
    assert np.allclose(c, t.mean(axis=(1, 2))[:, None, None])
    # corrected values are clipped to the image range
    c2, _, _ = OE.color_correct(t, np.clip(2.0 * t - 0.5, -1, 2))
    assert c2.min() >= 0.0 and c2.max() <= 1.0


def test_metrics_of_an_exact_match():
    rng = np.random.default_rng(2)
    t = rng.uniform(0, 1, (3, 24, 20))
    p, s = OE.corrected_metrics(0.5 * t + 0.25, t)     # exactly affine: corrected to the truth
    assert s == pytest.approx(1.0, abs=1e-12) and p > 200
