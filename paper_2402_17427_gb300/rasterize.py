"""PyTorch front end of the CUDA rasteriser: device memory, streams and autograd plumbing.

Everything numeric runs in libvgrast.so; this module only allocates tensors (the caller-owned
workspace and outputs), passes raw pointers and the current stream, and wires the backward
entry point into ``torch.autograd``.  The backward pass keeps no per-sample state: the saved
context is the workspace (projected Gaussians, tile lists), the final transmittance and the
last-contributor index per pixel, from which the kernels recompute transmittance (paper Sec. 3,
"differentiable rasterizer"; memory O(pixels + pairs), which is what lets one GPU hold the
20M-Gaussian cells).
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np
import torch

from . import binding as B
from .scenes import Camera


@dataclasses.dataclass
class RasterSettings:
    tile_size: int = 16
    chunk: int = 128
    bg: tuple = (0.0, 0.0, 0.0)
    dilation: float = 0.3
    alpha_max: float = 0.99
    alpha_min: float = 1.0 / 255.0
    t_min: float = 1e-4
    guard: float = 1.3
    stop_rule: int = 0
    count_blends: bool = False
    test_stall: bool = False      # diagnostic: make the compaction's look-back give up (tests only)

    def c(self, accumulate: bool = False) -> B.vg_raster_opts:
        o = B.vg_raster_opts()
        o.tile_size, o.chunk = self.tile_size, self.chunk
        o.bg[:] = [float(v) for v in self.bg]
        o.dilation, o.alpha_max, o.alpha_min = self.dilation, self.alpha_max, self.alpha_min
        o.t_min, o.guard, o.stop_rule = self.t_min, self.guard, self.stop_rule
        o.flags = (B.VG_FLAG_COUNT_BLENDS if self.count_blends else 0) | \
                  (B.VG_FLAG_ACCUMULATE_GRADS if accumulate else 0) | \
                  (B.VG_FLAG_TEST_STALL_LOOKBACK if self.test_stall else 0)
        return o


def camera_c(cam: Camera) -> B.vg_camera:
    c = B.vg_camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.world_to_cam[:] = [float(v) for v in cam.world_to_cam.ravel()]
    c.cam_pos[:] = [float(v) for v in np.asarray(cam.cam_pos, np.float32)]
    c.near_plane = float(cam.near)
    return c


def gaussians_c(means, log_scales, quats, logits, sh, degree: int) -> B.vg_gaussians:
    for t in (means, log_scales, quats, logits, sh):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError("Gaussian parameters must be contiguous float32 CUDA tensors")
    g = B.vg_gaussians()
    g.means, g.log_scales, g.quats = means.data_ptr(), log_scales.data_ptr(), quats.data_ptr()
    g.opacity_logits, g.sh = logits.data_ptr(), sh.data_ptr()
    g.n, g.sh_degree = int(means.shape[0]), int(degree)
    return g


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


class Workspace:
    """Caller-owned device workspace of one view, grown when a render needs more pairs."""

    def __init__(self, device=None, pair_capacity: int | None = None):
        self.device = torch.device(device or "cuda")
        self.capacity = pair_capacity
        self.buf = None
        self.key = None

    def ensure(self, n: int, width: int, height: int, opts: B.vg_raster_opts, capacity: int | None = None):
        # first guess one pair per Gaussian (a render that needs more reports it and is re-run
        # with the count it needed); the capacity only grows
        cap = int(capacity or self.capacity or max(1 << 16, n))
        self.capacity = cap
        need = B.vg_workspace_bytes(n, width, height, cap, opts)
        if need == 0:
            raise ValueError("invalid rasteriser sizes")
        if self.buf is None or self.buf.numel() < need:
            self.buf = torch.empty(need, dtype=torch.uint8, device=self.device)
        self.key = (n, width, height, cap, opts.tile_size)
        return self.buf, need


class Rasterizer:
    """Forward / backward of one cell seen by one camera, with a persistent workspace.

    ``check='sync'`` reads the device counters after every forward (one host synchronisation)
    and re-renders with a larger pair list when it overflowed.  ``check='defer'`` never
    synchronises; call :meth:`verify` later to make sure no render overflowed.
    """

    def __init__(self, settings: RasterSettings | None = None, device=None, pair_capacity=None, check="sync"):
        self.settings = settings or RasterSettings()
        self.ws = Workspace(device, pair_capacity)
        self.check = check
        self.counters = None
        self._pending = []

    def forward(self, means, log_scales, quats, logits, sh, degree, cam: Camera, events=None, key_inputs=None):
        """key_inputs: optional float32 CUDA tensor [n, 4] that receives the FP32 (u, v, r, depth)
        each Gaussian's tile rectangle and sort key were decided from (parity tests)."""
        opts = self.settings.c()
        if events is not None:
            opts.events = ctypes.pointer(events)
        if key_inputs is not None:
            if not (key_inputs.is_cuda and key_inputs.dtype == torch.float32 and key_inputs.is_contiguous()
                    and key_inputs.numel() >= 4 * int(means.shape[0])):
                raise ValueError("key_inputs must be a contiguous float32 CUDA tensor of n x 4 entries")
            opts.key_inputs = key_inputs.data_ptr()
        g = gaussians_c(means, log_scales, quats, logits, sh, degree)
        camc = camera_c(cam)
        dev = means.device
        H, W = cam.height, cam.width
        rgb = torch.empty((3, H, W), dtype=torch.float32, device=dev)
        T = torch.empty((H, W), dtype=torch.float32, device=dev)
        last = torch.empty((H, W), dtype=torch.int32, device=dev)
        counters = torch.empty(B.VG_CNT_LEN, dtype=torch.int64, device=dev)   # every entry written by the call
        for _attempt in range(4):
            buf, nbytes = self.ws.ensure(g.n, W, H, opts)
            B.vg_rasterize_forward(g, camc, opts, buf.data_ptr(), nbytes, self.ws.capacity, rgb.data_ptr(),
                                   T.data_ptr(), last.data_ptr(), counters.data_ptr(), _stream())
            if self.check != "sync":
                self._pending.append(counters)
                break
            c = counters.cpu()
            if c[B.VG_CNT_STATUS] & B.VG_STATUS_WAIT_TIMEOUT:
                raise B.VGError(B.VG_ERR_TIMEOUT, "vg_rasterize_forward")
            if not (c[B.VG_CNT_STATUS] & B.VG_STATUS_PAIR_OVERFLOW):
                break
            self.ws.capacity = int(c[B.VG_CNT_PAIRS] * 1.25) + 1024
        self.counters = counters
        return rgb, T, last

    def verify(self):
        """Raises if any deferred render overflowed its pair list or timed out."""
        for c in self._pending:
            c = c.cpu()
            if c[B.VG_CNT_STATUS]:
                raise B.VGError(B.VG_ERR_CAPACITY if c[B.VG_CNT_STATUS] & 1 else B.VG_ERR_TIMEOUT, "deferred render")
        self._pending.clear()

    def backward(self, means, log_scales, quats, logits, sh, degree, cam: Camera, T, last, dL_drgb,
                 grads=None, accumulate=False, means2d_abs=None, events=None):
        opts = self.settings.c(accumulate=accumulate)
        if events is not None:
            opts.events = ctypes.pointer(events)
        g = gaussians_c(means, log_scales, quats, logits, sh, degree)
        if grads is None:
            grads = tuple(torch.empty_like(t) for t in (means, log_scales, quats, logits, sh))
        buf, nbytes = self.ws.buf, self.ws.buf.numel()
        dL = dL_drgb.contiguous()
        B.vg_rasterize_backward(g, camera_c(cam), opts, buf.data_ptr(), nbytes, self.ws.capacity, T.data_ptr(),
                                last.data_ptr(), dL.data_ptr(), *(t.data_ptr() for t in grads),
                                means2d_abs.data_ptr() if means2d_abs is not None else None, _stream())
        return grads


class _RasterizeFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, log_scales, quats, logits, sh, degree, cam, rasterizer):
        rgb, T, last = rasterizer.forward(means, log_scales, quats, logits, sh, degree, cam)
        ctx.save_for_backward(means, log_scales, quats, logits, sh, T, last)
        ctx.degree, ctx.cam, ctx.rasterizer = degree, cam, rasterizer
        ctx.mark_non_differentiable(T, last)
        return rgb, T, last

    @staticmethod
    def backward(ctx, dL_drgb, _dT, _dlast):
        means, log_scales, quats, logits, sh, T, last = ctx.saved_tensors
        grads = ctx.rasterizer.backward(means, log_scales, quats, logits, sh, ctx.degree, ctx.cam, T, last,
                                        dL_drgb)
        return (*grads, None, None, None)


def rasterize(means, log_scales, quats, logits, sh, degree: int, cam: Camera, rasterizer: Rasterizer | None = None):
    """Differentiable render: returns the image [3,H,W]; gradients flow to the raw parameters."""
    r = rasterizer or Rasterizer()
    rgb, _T, _last = _RasterizeFn.apply(means, log_scales, quats, logits, sh, degree, cam, r)
    return rgb


class LossL1DSSIM:
    """Eq. 1 loss on the GPU: returns (loss scalar tensor, dL/dimage)."""

    def __init__(self, lam: float = 0.2):
        self.lam = lam
        self.buf = None
        self.loss = None
        self.grad = None
        self.calls = 0          # forward calls on this workspace (the SSIM maps they leave behind)

    def _workspace(self, img):
        _, H, W = img.shape
        need = B.vg_loss_workspace_bytes(W, H)
        if self.buf is None or self.buf.numel() < need:
            self.buf = torch.empty(need, dtype=torch.uint8, device=img.device)
        self.calls += 1
        return W, H

    def __call__(self, img: torch.Tensor, target: torch.Tensor, reuse: bool = False):
        W, H = self._workspace(img)
        if reuse and self.grad is not None and self.grad.shape == img.shape:
            loss, grad = self.loss, self.grad
        else:
            loss = torch.empty((), dtype=torch.float32, device=img.device)
            grad = torch.empty_like(img)
            self.loss, self.grad = loss, grad
        B.vg_loss_l1_dssim(img.contiguous().data_ptr(), target.contiguous().data_ptr(), W, H, self.lam,
                           self.buf.data_ptr(), self.buf.numel(), loss.data_ptr(), grad.data_ptr(), _stream())
        return loss, grad

    def value(self, img: torch.Tensor, target: torch.Tensor):
        """The loss alone; the workspace keeps what grad_scaled needs."""
        W, H = self._workspace(img)
        loss = torch.empty((), dtype=torch.float32, device=img.device)
        B.vg_loss_l1_dssim(img.data_ptr(), target.data_ptr(), W, H, self.lam, self.buf.data_ptr(), self.buf.numel(),
                           loss.data_ptr(), None, _stream())
        return loss

    def grad_scaled(self, img: torch.Tensor, target: torch.Tensor, scale: torch.Tensor, buf: torch.Tensor):
        """scale * dL/dimage from the state the last value() call left in `buf`."""
        _, H, W = img.shape
        grad = torch.empty_like(img)
        B.vg_loss_l1_dssim_grad(img.data_ptr(), target.data_ptr(), W, H, self.lam, buf.data_ptr(), buf.numel(),
                                scale.data_ptr(), grad.data_ptr(), _stream())
        return grad


class _LossFn(torch.autograd.Function):
    """Forward computes the loss only; backward runs the gradient pass scaled on the device by the
    incoming gradient (no separate elementwise product)."""

    @staticmethod
    def forward(ctx, img, target, lossobj):
        img, target = img.contiguous(), target.contiguous()
        loss = lossobj.value(img, target)
        ctx.save_for_backward(img, target)
        ctx.lossobj, ctx.buf, ctx.call = lossobj, lossobj.buf, lossobj.calls
        return loss

    @staticmethod
    def backward(ctx, g):
        img, target = ctx.saved_tensors
        if ctx.lossobj.buf is ctx.buf and ctx.lossobj.calls != ctx.call:
            raise RuntimeError("the loss workspace was used by another forward before this backward")
        scale = g.detach().to(torch.float32).contiguous()
        return ctx.lossobj.grad_scaled(img, target, scale, ctx.buf), None, None


def l1_dssim_loss(img, target, lam: float = 0.2, lossobj: LossL1DSSIM | None = None):
    """Differentiable Eq. 1 loss ((1 - lam) L1 + lam D-SSIM) computed by the CUDA kernels."""
    return _LossFn.apply(img, target, lossobj or LossL1DSSIM(lam))


def to_device(g, device="cuda"):
    """Gaussian parameter tensors (float32, contiguous) on the device."""
    return [torch.from_numpy(np.ascontiguousarray(a)).to(device) for a in g.arrays()]


def color_corrected_metrics(img: torch.Tensor, target: torch.Tensor):
    """PSNR and SSIM of a rendering after the per-image least-squares colour correction of the
    evaluation protocol (Sec. 5.1).  img, target: CUDA float32 [3, H, W].  Returns a CUDA float32
    [14] tensor: PSNR, SSIM, A (3x3, row-major), b (3)."""
    img, target = img.contiguous(), target.contiguous()
    H, W = int(img.shape[1]), int(img.shape[2])
    need = B.vg_eval_workspace_bytes(W, H)
    ws = torch.empty(need, dtype=torch.uint8, device=img.device)
    out = torch.empty(14, dtype=torch.float32, device=img.device)
    B.vg_eval_color_corrected(img.data_ptr(), target.data_ptr(), W, H, ws.data_ptr(), need, out.data_ptr(), _stream())
    return out
