"""Per-cell optimiser step on the GPU (paper Sec. 3, Sec. 5.1) through include/vgoptim.h: a fused
Adam update of every parameter group, the densification statistics of each rendered view and the
clone / split / prune densification (every 200 iterations between 1,000 and 30,000).

The learning rates and densification thresholds below are the settings of 3D Gaussian Splatting,
which the paper keeps for everything it does not change; the schedule of the position learning
rate is the caller's (pass the current value to each step).
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import binding as B
from .rasterize import _stream, gaussians_c

PARAM_NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")


@dataclass
class AdamSettings:
    lr_means: float = 1.6e-4        # times the scene extent, decayed by the caller's schedule
    lr_log_scales: float = 5e-3
    lr_quats: float = 1e-3
    lr_opacity: float = 5e-2
    lr_sh_dc: float = 2.5e-3
    lr_sh_rest: float = 2.5e-3 / 20
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15


@dataclass
class DensifySettings:
    grad_threshold: float = 2e-4
    percent_dense: float = 0.01
    scene_extent: float = 1.0
    min_opacity: float = 0.005
    max_world_scale_frac: float = 0.1    # of the scene extent
    start: int = 1000
    stop: int = 30000
    every: int = 200

    def c(self) -> B.vg_densify_opts:
        o = B.vg_densify_opts()
        o.grad_threshold, o.percent_dense, o.scene_extent = self.grad_threshold, self.percent_dense, self.scene_extent
        o.min_opacity, o.max_world_scale = self.min_opacity, self.max_world_scale_frac * self.scene_extent
        return o

    def due(self, iteration: int) -> bool:
        return self.start <= iteration <= self.stop and iteration % self.every == 0


def _ptrs(ts) -> B.vg_param_ptrs:
    p = B.vg_param_ptrs()
    p.means, p.log_scales, p.quats, p.opacity_logits, p.sh = (t.data_ptr() for t in ts)
    return p


class Adam:
    """Adam moments of one cell's parameters, updated in place by one fused launch per step."""

    def __init__(self, params, settings: AdamSettings | None = None):
        self.s = settings or AdamSettings()
        self.m = tuple(torch.zeros_like(t) for t in params)
        self.v = tuple(torch.zeros_like(t) for t in params)
        self.t = 0

    def step(self, params, grads, degree: int, lr_means: float | None = None):
        self.t += 1
        o = B.vg_adam_opts()
        o.lr[:] = [self.s.lr_means if lr_means is None else lr_means, self.s.lr_log_scales, self.s.lr_quats,
                   self.s.lr_opacity, self.s.lr_sh_dc, self.s.lr_sh_rest]
        o.beta1, o.beta2, o.eps, o.step = self.s.beta1, self.s.beta2, self.s.eps, self.t
        B.vg_adam_step(_ptrs(params), gaussians_c(*grads, degree), _ptrs(self.m), _ptrs(self.v), o, _stream())


class DensifyStats:
    """Accumulated view-space gradient norm and view count of every Gaussian."""

    def __init__(self, n: int, device):
        self.accum = torch.zeros(n, dtype=torch.float32, device=device)
        self.count = torch.zeros(n, dtype=torch.int32, device=device)

    def add_view(self, rasterizer, n: int, camera):
        """After rasterizer.backward for `camera`: reads the 2D mean gradients from its workspace."""
        ws = rasterizer.ws
        opts = rasterizer.settings.c()
        B.vg_densify_accumulate(ws.buf.data_ptr(), ws.buf.numel(), n, camera.width, camera.height, ws.capacity, opts,
                                self.accum.data_ptr(), self.count.data_ptr(), _stream())


def densify_with(params, adam: Adam, stats: DensifyStats, degree: int, settings: DensifySettings,
                 normals: torch.Tensor):
    """Clone / split / prune with the given split draws (CUDA float32 [n, 2, 3] standard normals).
    Returns the new parameter tensors; `adam` and `stats` are replaced by the new model's moments
    and fresh statistics."""
    n = int(params[0].shape[0])
    dev = params[0].device
    cap = 2 * n
    out = tuple(torch.empty((cap,) + tuple(t.shape[1:]), dtype=t.dtype, device=dev) for t in params)
    mo = tuple(torch.empty_like(t) for t in out)
    vo = tuple(torch.empty_like(t) for t in out)
    need = B.vg_densify_workspace_bytes(n)
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    cnt = torch.empty((), dtype=torch.int64, device=dev)
    B.vg_densify(gaussians_c(*params, degree), gaussians_c(*adam.m, degree), gaussians_c(*adam.v, degree),
                 stats.accum.data_ptr(), stats.count.data_ptr(), normals.contiguous().data_ptr(), settings.c(),
                 ws.data_ptr(), need, _ptrs(out), _ptrs(mo), _ptrs(vo), cnt.data_ptr(), _stream())
    m = int(cnt)
    if m < 0:
        raise RuntimeError("vg_densify: a bounded device wait gave up")
    new = tuple(t[:m].contiguous() for t in out)
    adam.m = tuple(t[:m].contiguous() for t in mo)
    adam.v = tuple(t[:m].contiguous() for t in vo)
    stats.__init__(m, dev)
    return new


def densify(params, adam: Adam, stats: DensifyStats, degree: int, settings: DensifySettings,
            generator: torch.Generator | None = None):
    """Clone / split / prune with split draws from `generator`."""
    n = int(params[0].shape[0])
    normals = torch.randn((n, 2, 3), device=params[0].device, generator=generator)
    return densify_with(params, adam, stats, degree, settings, normals)
