"""Oracle for the evaluation metrics with colour correction (paper Sec. 5.1, "Metrics"), FP64.

TEST INFRASTRUCTURE ONLY (tests and the benchmark's CPU baseline); shares no code with the CUDA
kernels.

Before PSNR and SSIM are measured, each rendered image is aligned to its ground truth by solving
a per-image least-squares problem on the RGB values.  Reading: an affine map of the rendered
colour, y ~ A x + b (A 3x3, b 3), fitted over all pixels; the corrected image A x + b is clipped to
[0, 1] (the image range); PSNR = -10 log10(mean squared error) with peak 1; SSIM is the same 11x11
Gaussian-window SSIM as the loss (Eq. 1), averaged over pixels and channels.  When the normal
equations are singular (e.g. a constant rendering) any least-squares solution gives the same
fitted values, which is what the metrics use.
"""
from __future__ import annotations

import numpy as np


def color_correct(img: np.ndarray, target: np.ndarray):
    """img, target: [3, H, W].  Returns (corrected image [3,H,W], A [3,3], b [3])."""
    x = np.asarray(img, np.float64).reshape(3, -1).T
    y = np.asarray(target, np.float64).reshape(3, -1).T
    X = np.concatenate([x, np.ones((x.shape[0], 1))], axis=1)
    beta, *_ = np.linalg.lstsq(X, y, rcond=None)       # [4, 3]
    fitted = X @ beta
    out = np.clip(fitted, 0.0, 1.0).T.reshape(np.shape(img))
    return out, beta[:3].T, beta[3]


def psnr(img: np.ndarray, target: np.ndarray) -> float:
    mse = float(np.mean((np.asarray(img, np.float64) - np.asarray(target, np.float64)) ** 2))
    return float("inf") if mse == 0.0 else -10.0 * np.log10(mse)


def corrected_metrics(img: np.ndarray, target: np.ndarray):
    """(PSNR, SSIM) of the colour-corrected rendering."""
    import oracle
    c, _, _ = color_correct(img, target)
    return psnr(c, target), oracle.ssim(c, target)
