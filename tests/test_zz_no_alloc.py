"""The allocation-free loss entry point (vg_loss_l1_dssim_noalloc) against the regular one.

Callers that cannot allocate device memory between steps (hosts that plan all device memory up
front, latency-critical loops) use the variant whose scratch lives in the library itself.  It
must give the same loss and gradient as vg_loss_l1_dssim, on consecutive calls that reuse the
shared scratch, and refuse images larger than its fixed scratch.  This file is collected last
so that a run stopping at the first failure has already run every other test.
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
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _regular(x, y, lam):
    W, H = x.shape[2], x.shape[1]
    need = B.vg_loss_workspace_bytes(W, H)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    loss = torch.empty((), dtype=torch.float32, device="cuda")
    grad = torch.empty_like(x)
    B.vg_loss_l1_dssim(x.data_ptr(), y.data_ptr(), W, H, lam, ws.data_ptr(), need, loss.data_ptr(),
                       grad.data_ptr(), _stream())
    return loss, grad


def _noalloc(x, y, lam):
    W, H = x.shape[2], x.shape[1]
    loss = torch.empty((), dtype=torch.float32, device="cuda")
    grad = torch.empty_like(x)
    B.vg_loss_l1_dssim_noalloc(x.data_ptr(), y.data_ptr(), W, H, lam, loss.data_ptr(), grad.data_ptr(), _stream())
    return loss, grad


def test_noalloc_loss_matches_regular_entry_point_on_consecutive_calls():
    rng = np.random.default_rng(123)
    # two calls in a row with different sizes: the second reuses the shared scratch
    for (H, W), lam in [((864, 1152), 0.2), ((75, 101), 0.5)]:
        x = torch.from_numpy(rng.random((3, H, W)).astype(np.float32)).cuda()
        y = torch.from_numpy(rng.random((3, H, W)).astype(np.float32)).cuda()
        l_ref, g_ref = _regular(x, y, lam)
        l_na, g_na = _noalloc(x, y, lam)
        torch.cuda.synchronize()
        assert abs(float(l_na) - float(l_ref)) <= 1e-6 * abs(float(l_ref)) + 1e-7
        assert torch.allclose(g_na, g_ref, rtol=1e-5, atol=1e-9 * float(g_ref.abs().max()))


def test_noalloc_loss_rejects_images_beyond_its_scratch():
    H, W = 1025, 1024      # one row more than VG_LOSS_NOALLOC_MAX_PIXELS allows
    assert H * W > B.VG_LOSS_NOALLOC_MAX_PIXELS
    x = torch.zeros((3, H, W), dtype=torch.float32, device="cuda")
    with pytest.raises(B.VGError) as e:
        _noalloc(x, x, 0.2)
    assert e.value.status == B.VG_ERR_CAPACITY


def test_noalloc_loss_rejects_a_side_beyond_16384_as_an_argument_error():
    # few pixels, but one side over the 16384 every entry point accepts
    x = torch.zeros((3, 1, 20000), dtype=torch.float32, device="cuda")
    with pytest.raises(B.VGError) as e:
        _noalloc(x, x, 0.2)
    assert e.value.status == B.VG_ERR_INVALID
