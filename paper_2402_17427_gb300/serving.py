"""Continuous-batching novel-view server over a merged scene.

VastGaussian merges its optimised cells into one scene (Sec. 4.3) and renders it in real time
(Sec. 5).  This server keeps every cell's Gaussians resident on the device, takes novel-view
requests as they arrive, admits them into batches while stream slots and the memory budget
allow, and renders each batch with one ``vg_render_views`` call (every view culls the cells
whose boxes miss its frustum).  Several slots, each with its own CUDA stream and workspace, let
batches admitted while others are still on the GPU overlap with them on the device.  Latency is
completion time minus arrival time, measured on the host clock by polling CUDA events.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np
import torch

from . import binding as B
from .rasterize import RasterSettings, camera_c, gaussians_c, to_device


def extent_aabb(g, sigmas: float = 3.0) -> np.ndarray:
    """Box around a cell's Gaussians including `sigmas` times their largest scale."""
    m = np.asarray(g.means, np.float64)
    r = sigmas * np.exp(np.asarray(g.log_scales, np.float64).max(axis=1))[:, None]
    return np.concatenate([(m - r).min(0), (m + r).max(0)]).astype(np.float32)


@dataclasses.dataclass
class ServeStats:
    requests: int
    duration_s: float
    latencies_ms: list
    p50_ms: float
    p99_ms: float
    mean_ms: float
    throughput_rps: float
    mpix_per_s: float
    batches: int
    mean_batch: float
    max_inflight: int
    max_inflight_bytes: int
    rerenders: int
    mean_cells_per_view: float

    def summary(self) -> dict:
        d = dataclasses.asdict(self)
        d.pop("latencies_ms")
        return d


def admit(queue_bytes, inflight_bytes: int, any_inflight: bool, budget: int, max_batch: int) -> int:
    """How many requests from the head of the queue (their in-flight device bytes, in arrival order)
    the next batch takes: as many as fit the memory budget next to what is already in flight, up
    to max_batch.  A request larger than the whole budget is still served, alone, once nothing else
    is in flight; otherwise requests that do not fit wait in the queue."""
    k, est = 0, 0
    for e in queue_bytes:
        if k == max_batch:
            break
        if inflight_bytes + est + e > budget and (k > 0 or any_inflight):
            break
        k += 1
        est += e
    return k


class _Slot:
    def __init__(self, device):
        self.stream = torch.cuda.Stream(device=device)
        self.buf = None
        self.busy = False


class SceneServer:
    """Renders novel views of resident cells; see :meth:`render` and :meth:`serve`."""

    def __init__(self, cells, device="cuda", settings: RasterSettings | None = None, slots: int = 3,
                 max_batch: int = 8, mem_budget_gb: float = 32.0, pairs_per_mpix: float = 4e6):
        self.device = torch.device(device)
        self.settings = settings or RasterSettings()
        self.degree = cells[0].gaussians.sh_degree
        self.params = [to_device(c.gaussians, self.device) for c in cells]
        self.gs = [gaussians_c(*p, self.degree) for p in self.params]
        self.n = np.array([c.gaussians.n for c in cells], np.int64)
        self.aabbs = np.ascontiguousarray(np.stack([extent_aabb(c.gaussians) for c in cells]), np.float32)
        self.slots = [_Slot(self.device) for _ in range(slots)]
        self.max_batch = max_batch
        self.budget = int(mem_budget_gb * (1 << 30))
        self.ppm0 = pairs_per_mpix           # prior before the first observation
        self.ppm = None                      # largest (Gaussian, tile) pairs per megapixel seen
        self.resident_bytes = sum(sum(t.numel() * 4 for t in p) for p in self.params)

    # -------------------------------------------------------------------------------- one batch
    def _ppm(self) -> float:
        return self.ppm if self.ppm is not None else self.ppm0

    def _capacity(self, cams):
        """Pair-list capacity for a batch: its megapixels times the largest pairs-per-megapixel any
        batch has needed so far (never lowered, so a capacity that held once holds again), with a
        25 % margin."""
        mpix = sum(c.width * c.height for c in cams) / 1e6
        return max(1 << 16, int(mpix * self._ppm() * 1.25))

    def _observe(self, cams, counters):
        mpix = sum(c.width * c.height for c in cams) / 1e6
        seen = float(counters[B.VG_CNT_PAIRS]) / max(mpix, 1e-6)
        self.ppm = seen if self.ppm is None else max(self.ppm, seen)

    def _launch(self, slot: _Slot, cams, capacity: int):
        opts = [self.settings.c() for _ in cams]
        camc = [camera_c(c) for c in cams]
        need = B.vg_views_workspace_bytes(self.gs, self.aabbs, camc, opts, capacity)
        if need == 0:
            raise ValueError("invalid views")
        with torch.cuda.stream(slot.stream):
            if slot.buf is None or slot.buf.numel() < need:
                slot.buf = torch.empty(need, dtype=torch.uint8, device=self.device)
            outs = [(torch.empty((3, c.height, c.width), dtype=torch.float32, device=self.device),
                     torch.empty((c.height, c.width), dtype=torch.float32, device=self.device),
                     torch.empty((c.height, c.width), dtype=torch.int32, device=self.device)) for c in cams]
            counters = torch.empty(B.VG_CNT_LEN, dtype=torch.int64, device=self.device)   # all written by the call
            kept = B.vg_render_views(self.gs, self.aabbs, camc, opts, slot.buf.data_ptr(), need, capacity,
                                     [o[0].data_ptr() for o in outs], [o[1].data_ptr() for o in outs],
                                     [o[2].data_ptr() for o in outs], counters.data_ptr(), slot.stream.cuda_stream)
            # counters go to pinned host memory on this slot's stream: reading them after the
            # event completes needs no synchronisation with the other slots
            host = torch.empty(B.VG_CNT_LEN, dtype=torch.int64, pin_memory=True)
            host.copy_(counters, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(slot.stream)
        return outs, host, ev, kept, need

    def render(self, cams, capacity: int | None = None):
        """Synchronous render of a list of views; returns [(rgb, T, last)] and the counters."""
        cap = capacity or self._capacity(cams)
        slot = self.slots[0]
        for _ in range(4):
            outs, counters, ev, kept, _ = self._launch(slot, cams, cap)
            ev.synchronize()
            c = counters
            self._observe(cams, c)
            if not (int(c[B.VG_CNT_STATUS]) & B.VG_STATUS_PAIR_OVERFLOW):
                return outs, c, kept
            cap = int(c[B.VG_CNT_PAIRS] * 1.25) + 1024
        raise B.VGError(B.VG_ERR_CAPACITY, "render")

    # -------------------------------------------------------------------------------- the loop
    def _bytes(self, cam) -> int:
        """Device memory one request holds while in flight: its image buffers and its share of
        the batch workspace (pairs at 64 B, visible Gaussians at about 200 B)."""
        px = cam.width * cam.height
        return 20 * px + int(64 * 1.25 * self._ppm() * px / 1e6) + int(200 * self.n.sum() / 4)

    def serve(self, requests, keep_outputs: bool = False, time_limit_s: float | None = None,
              warmup_s: float = 0.0):
        """Runs the request stream in real time.  Returns ServeStats (and outputs by rid if kept).

        Requests that arrive before ``warmup_s`` are served but left out of the statistics."""
        reqs = sorted(requests, key=lambda r: r.arrival_s)
        queue = collections.deque()
        inflight = []
        lat = {}
        outputs = {}
        nxt = 0
        batches = 0
        batch_sizes = []
        rerenders = 0
        max_inflight = 0
        max_inflight_bytes = 0
        kept_cells = []
        inflight_bytes = 0
        torch.cuda.synchronize(self.device)
        t0 = time.perf_counter()
        while len(lat) < len(reqs):
            now = time.perf_counter() - t0
            if time_limit_s is not None and now > time_limit_s:
                break
            while nxt < len(reqs) and reqs[nxt].arrival_s <= now:
                queue.append(reqs[nxt])
                nxt += 1
            # completions
            for b in list(inflight):
                slot, batch, outs, counters, ev, est = b
                if not ev.query():
                    continue
                done = time.perf_counter() - t0
                inflight.remove(b)
                slot.busy = False
                inflight_bytes -= est
                c = counters
                self._observe([r.camera for r in batch], c)
                if int(c[B.VG_CNT_STATUS]) & B.VG_STATUS_PAIR_OVERFLOW:
                    # the estimate was too low: render these requests again, first in line
                    rerenders += 1
                    queue.extendleft(reversed(batch))
                    continue
                for r, o in zip(batch, outs):
                    lat[r.rid] = (done - r.arrival_s) * 1e3
                    if keep_outputs:
                        outputs[r.rid] = o
            # admission: a free slot and room in the memory budget
            free = [s for s in self.slots if not s.busy]
            k = 0
            if queue and free:
                head = [self._bytes(queue[i].camera) for i in range(min(len(queue), self.max_batch))]
                k = admit(head, inflight_bytes, bool(inflight), self.budget, self.max_batch)
            if k > 0:
                batch = [queue.popleft() for _ in range(k)]
                est = sum(head[:k])
                slot = free[0]
                cams = [r.camera for r in batch]
                outs, counters, ev, kept, _ = self._launch(slot, cams, self._capacity(cams))
                kept_cells += kept
                slot.busy = True
                inflight.append((slot, batch, outs, counters, ev, est))
                inflight_bytes += est
                batches += 1
                batch_sizes.append(len(batch))
                max_inflight = max(max_inflight, len(inflight))
                max_inflight_bytes = max(max_inflight_bytes, inflight_bytes)
                continue
            # nothing to do right now: wait briefly for an arrival or a completion
            if inflight or (nxt < len(reqs)):
                wait = 2e-4 if inflight else max(0.0, min(2e-3, reqs[nxt].arrival_s - now))
                time.sleep(wait)
        torch.cuda.synchronize(self.device)
        dur = time.perf_counter() - t0
        served = [r for r in reqs if r.rid in lat and r.arrival_s >= warmup_s]
        L = np.array([lat[r.rid] for r in served]) if served else np.zeros(1)
        mpix = sum(r.camera.width * r.camera.height for r in served) / 1e6
        dur = dur - warmup_s
        stats = ServeStats(requests=len(served), duration_s=dur, latencies_ms=L.tolist(),
                           p50_ms=float(np.percentile(L, 50)), p99_ms=float(np.percentile(L, 99)),
                           mean_ms=float(L.mean()), throughput_rps=len(served) / dur, mpix_per_s=mpix / dur,
                           batches=batches, mean_batch=float(np.mean(batch_sizes)) if batch_sizes else 0.0,
                           max_inflight=max_inflight, max_inflight_bytes=int(max_inflight_bytes),
                           rerenders=rerenders,
                           mean_cells_per_view=float(np.mean(kept_cells)) if kept_cells else 0.0)
        return (stats, outputs) if keep_outputs else stats
