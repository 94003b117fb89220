"""Batched multi-cell rendering: many cells, each with its own camera, in one launch per stage.

VastGaussian optimises the cells of a partitioned scene independently and in parallel
(Sec. 4.1; Sec. 5.1 trains one cell per GPU).  Here the cells of one training step share a
GPU: ``vg_render_batch`` projects all cells' Gaussians in one launch, sorts all of their
(tile, Gaussian) pairs in one sort, and composites every (cell, tile) work item in one
persistent launch per tile size whose blocks pull the largest tile lists first;
``vg_render_batch_backward`` mirrors it.  Cells may use different tile sizes.

The autotuner picks, per cell, the tile size (8, 16 or 32) and the shared-memory chunk depth
that minimise the measured forward + backward time of that cell alone, and caches the choice by
(Gaussian-count bucket, pixel count, pairs-per-visible bucket).  The depth-sort bit width needs
no tuning: every render sorts exactly the significant bits of its keys (computed on the device).
"""
from __future__ import annotations

import math

import torch

from . import binding as B
from .rasterize import RasterSettings, Workspace, camera_c, gaussians_c, _stream


class BatchRasterizer:
    """Forward / backward of n cells x 1 camera each through the batch C ABI."""

    def __init__(self, settings=None, device=None, pair_capacity=None, check="sync"):
        self.settings = settings            # list of RasterSettings (one per cell) or None
        self.device = torch.device(device or "cuda")
        self.capacity = pair_capacity
        self.buf = None
        self.check = check
        self.counters = None
        self._pending = []

    def _opts(self, n, accumulate=False, events=None):
        st = self.settings or [RasterSettings()] * n
        arr = []
        for s in st:
            o = s.c(accumulate=accumulate)
            arr.append(o)
        if events is not None:
            import ctypes
            arr[0].events = ctypes.pointer(events)
        return arr

    def _ensure(self, gs, cams, opts, n_total):
        cap = int(self.capacity or max(1 << 16, n_total))
        self.capacity = cap
        need = B.vg_batch_workspace_bytes(gs, cams, opts, cap)
        if need == 0:
            raise ValueError("invalid batch")
        if self.buf is None or self.buf.numel() < need:
            self.buf = torch.empty(need, dtype=torch.uint8, device=self.device)
        return need

    def forward(self, cells, degree, cameras, events=None, key_inputs=None):
        """cells: list of (means, log_scales, quats, logits, sh) tensors.  Returns [(rgb, T, last)].
        key_inputs: optional float32 CUDA tensor [total n, 4] receiving every Gaussian's FP32
        (u, v, r, depth) decision inputs, cells concatenated in order (parity tests)."""
        gs = [gaussians_c(*c, degree) for c in cells]
        cams = [camera_c(c) for c in cameras]
        opts = self._opts(len(cells), events=events)
        if key_inputs is not None:
            total = sum(int(c[0].shape[0]) for c in cells)
            if not (key_inputs.is_cuda and key_inputs.dtype == torch.float32 and key_inputs.is_contiguous()
                    and key_inputs.numel() >= 4 * total):
                raise ValueError("key_inputs must be a contiguous float32 CUDA tensor of total n x 4 entries")
            opts[0].key_inputs = key_inputs.data_ptr()
        outs = []
        for cam in cameras:
            outs.append((torch.empty((3, cam.height, cam.width), dtype=torch.float32, device=self.device),
                         torch.empty((cam.height, cam.width), dtype=torch.float32, device=self.device),
                         torch.empty((cam.height, cam.width), dtype=torch.int32, device=self.device)))
        counters = torch.empty(B.VG_CNT_LEN, dtype=torch.int64, device=self.device)   # every entry written by the call
        n_total = sum(int(c[0].shape[0]) for c in cells)
        for _ in range(4):
            nbytes = self._ensure(gs, cams, opts, n_total)
            B.vg_render_batch(gs, cams, opts, self.buf.data_ptr(), nbytes, self.capacity,
                              [o[0].data_ptr() for o in outs], [o[1].data_ptr() for o in outs],
                              [o[2].data_ptr() for o in outs], counters.data_ptr(), _stream())
            if self.check != "sync":
                self._pending.append(counters)
                break
            c = counters.cpu()
            if c[B.VG_CNT_STATUS] & B.VG_STATUS_WAIT_TIMEOUT:
                raise B.VGError(B.VG_ERR_TIMEOUT, "vg_render_batch")
            if not c[B.VG_CNT_STATUS] & B.VG_STATUS_PAIR_OVERFLOW:
                break
            self.capacity = int(c[B.VG_CNT_PAIRS] * 1.25) + 1024
        self.counters = counters
        return outs

    def read_state(self, cells, degree, cameras):
        """Tile ranges [total tiles, 2] and Gaussian ids of every pair (global numbering, cells in
        order) left by the last forward, as NumPy arrays."""
        import numpy as np
        gs = [gaussians_c(*c, degree) for c in cells]
        cams = [camera_c(c) for c in cameras]
        opts = self._opts(len(cells))
        tiles = 0
        for s, cam in zip(self.settings or [RasterSettings()] * len(cells), cameras):
            ts = s.tile_size
            tiles += ((cam.width + ts - 1) // ts) * ((cam.height + ts - 1) // ts)
        ranges = torch.zeros((tiles, 2), dtype=torch.int32, device=self.device)
        ids = torch.zeros(self.capacity, dtype=torch.int32, device=self.device)
        B.vg_read_batch_state(self.buf.data_ptr(), self.buf.numel(), gs, cams, opts, self.capacity,
                              ranges.data_ptr(), ids.data_ptr(), None, None, _stream())
        torch.cuda.synchronize()
        return ranges.cpu().numpy().astype(np.int64), ids.cpu().numpy().view(np.uint32)

    def verify(self):
        for c in self._pending:
            c = c.cpu()
            if c[B.VG_CNT_STATUS]:
                raise B.VGError(B.VG_ERR_CAPACITY if c[B.VG_CNT_STATUS] & 1 else B.VG_ERR_TIMEOUT, "deferred batch")
        self._pending.clear()

    def backward(self, cells, degree, cameras, outs, dLs, grads=None, events=None):
        gs = [gaussians_c(*c, degree) for c in cells]
        cams = [camera_c(c) for c in cameras]
        opts = self._opts(len(cells), events=events)
        if grads is None:
            grads = [tuple(torch.empty_like(t) for t in c) for c in cells]
        dLs = [d.contiguous() for d in dLs]
        B.vg_render_batch_backward(gs, cams, opts, self.buf.data_ptr(), self.buf.numel(), self.capacity,
                                   [o[1].data_ptr() for o in outs], [o[2].data_ptr() for o in outs],
                                   [d.data_ptr() for d in dLs],
                                   [g[0].data_ptr() for g in grads], [g[1].data_ptr() for g in grads],
                                   [g[2].data_ptr() for g in grads], [g[3].data_ptr() for g in grads],
                                   [g[4].data_ptr() for g in grads], _stream())
        return grads


def _bucket(x: float) -> int:
    return int(round(math.log2(max(1.0, x)) * 2))


class AutoTuner:
    """Per-cell tile size / chunk choice by measurement, cached by a coarse workload key."""

    TILES = (8, 16, 32)
    CHUNKS = (32, 64, 128)

    def __init__(self, base: RasterSettings | None = None, trials: int = 3):
        self.base = base or RasterSettings()
        self.trials = trials
        self.cache = {}
        self.log = []

    def key(self, n, cam, pairs, visible):
        return (_bucket(n), cam.width * cam.height, _bucket(pairs / max(1, visible)))

    def _time(self, params, degree, cam, settings):
        from .rasterize import Rasterizer
        r = Rasterizer(settings, device=params[0].device, check="sync")
        rgb, T, last = r.forward(*params, degree, cam)
        dL = torch.ones_like(rgb) / rgb.numel()
        r.backward(*params, degree, cam, T, last, dL)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(self.trials):
            rgb, T, last = r.forward(*params, degree, cam)
            r.backward(*params, degree, cam, T, last, dL)
        e1.record()
        torch.cuda.synchronize()
        c = r.counters.cpu()
        return e0.elapsed_time(e1) / self.trials, int(c[B.VG_CNT_PAIRS]), int(c[B.VG_CNT_VISIBLE])

    def choose(self, params, degree, cam) -> RasterSettings:
        import dataclasses
        ms0, P, V = self._time(params, degree, cam, self.base)
        k = self.key(int(params[0].shape[0]), cam, P, V)
        if k in self.cache:
            return self.cache[k]
        best, best_ms = self.base, ms0
        for ts in self.TILES:
            for ch in self.CHUNKS:
                s = dataclasses.replace(self.base, tile_size=ts, chunk=ch)
                if s == self.base:
                    continue
                ms, _, _ = self._time(params, degree, cam, s)
                if ms < best_ms:
                    best, best_ms = s, ms
        self.cache[k] = best
        self.log.append({"key": k, "tile": best.tile_size, "chunk": best.chunk, "ms": best_ms, "default_ms": ms0})
        return best
