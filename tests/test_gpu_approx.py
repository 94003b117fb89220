"""The approximate operations the compositing kernels use, on the GPU at hand, through the C ABI.

The adjoint of the alpha blending (paper Sec. 3) walks each pixel's list back to front and divides
the transmittance by 1 - alpha with the approximate reciprocal; for a splat that does not reach the
pixel alpha is 0, and the kernel then relies on the reciprocal of 1 being exactly 1 (the pixel's
transmittance is left bit for bit).  The other checks bound both operations' error against FP64:
the reciprocal to 2 ulp over alpha's whole range (1 - alpha in [0.01, 1]), the base-2 exponential
to 2^-21 relative over the exponents the compositing evaluates (log2 of alpha_min .. 0).
"""
import numpy as np
import pytest
import torch

from paper_2402_17427_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2402_17427_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()


def _apply(kind, x):
    xin = torch.from_numpy(np.asarray(x, np.float32)).cuda()
    out = torch.full_like(xin, float("nan"))
    B.vg_approx_probe(kind, xin.data_ptr(), out.data_ptr(), xin.numel(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_reciprocal_of_one_is_exactly_one():
    x = np.array([1.0, 2.0, 0.5, 4.0, 0.25], np.float32)
    assert np.array_equal(_apply(0, x), (1.0 / x).astype(np.float32))
    # 1 - alpha for alpha = 0 as the kernel forms it (1 + (-0))
    one = np.float32(1.0) + np.float32(-0.0)
    assert _apply(0, [one])[0] == np.float32(1.0)


def test_reciprocal_error_over_the_alpha_range():
    x = np.linspace(0.01, 1.0, 100001, dtype=np.float32)
    got = _apply(0, x).astype(np.float64)
    ref = 1.0 / x.astype(np.float64)
    ulp = np.spacing(ref.astype(np.float32)).astype(np.float64)
    assert float(np.max(np.abs(got - ref) / ulp)) <= 2.0


def test_exp2_error_over_the_compositing_exponents():
    x = np.linspace(np.log2(1.0 / 255.0), 0.0, 100001, dtype=np.float32)
    got = _apply(1, x).astype(np.float64)
    ref = np.exp2(x.astype(np.float64))
    assert float(np.max(np.abs(got - ref) / ref)) <= 2.0 ** -21
    assert _apply(1, [0.0])[0] == np.float32(1.0)
