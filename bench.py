#!/usr/bin/env python3
"""Benchmark of the differentiable tile rasteriser: fwd+bwd training steps per second.

One step = forward render (projection + SH colour, depth sort, pair generation, tile sort,
front-to-back compositing) of one cell seen by one camera, the Eq. 1 loss
(0.8 L1 + 0.2 D-SSIM) and its gradient, and the backward render down to the raw parameters,
all through the C ABI of libvgrast.so.  Workload: 1,000,000 Gaussians drawn from 64 blobs over a
100x20x100 m volume, SH degree 3, one 1920x1080 camera on a 30 m orbit pitched down 45 deg
(synthetic, seeded).  Inputs are resident in HBM when the timed region starts; the parameters
(236 MB) are larger than L2, so no explicit L2 flush is done between steps.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle instead (bounded tile
samples extrapolated to a full step).  Under torchrun every rank renders its own replica
(the path has no exchange step) and rank 0 reports the aggregate.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd training steps/s (1 view, 1M Gaussians, SH3, 1920x1080, L1+0.2 D-SSIM)"
WORKLOAD = ("single-cell training step: 1,000,000 Gaussians from 64 blobs in 100x20x100 m, SH degree 3, "
            "1920x1080 camera on a 30 m orbit at 30 m altitude pitched -45 deg; forward + loss + backward")
# Algorithmic FP32-pipe operations of the compositing loops (see the design notes):
#   forward : 11 per (pixel, Gaussian) evaluation + 7 per composited evaluation
#   backward: 11 per evaluation (recomputed decision) + 37 per composited evaluation
OPS_EVAL, OPS_BLEND_FWD, OPS_BLEND_BWD = 11, 7, 37
# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the compositing kernels
# on this workload, from one ncu capture each (summarised under profiles/).  A figure holds only for
# the kernel source it was taken from: when the sources' hash differs it is reported as null.  The
# hash is re-recorded only after an edit that leaves the kernels' device source unchanged (the
# header's host-side workspace layout, host declarations, comments).
TRAFFIC_SOURCES = ("paper_2402_17427_gb300/csrc/blend.cu", "paper_2402_17427_gb300/csrc/vg_common.cuh",
                   "paper_2402_17427_gb300/csrc/internal.h")
PROFILED_TRAFFIC = {
    "sources_sha256": "41622bed1adda167cb60d63ef8b9ece17d6e7f7cf8280c257725cd320cd9aed1",
    "blend": 18660864 + 1536768,
    "blend_backward": 67457536 + 1475328,
}
# Warp instructions issued per launch (smsp__inst_executed.sum) of the compositing kernels on this
# workload, from the same captures; held to the same source hash.
PROFILED_INSTRUCTIONS = {
    "sources_sha256": "41622bed1adda167cb60d63ef8b9ece17d6e7f7cf8280c257725cd320cd9aed1",
    "blend": 259017717,
    "blend_backward": 357429896,
}


def _sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for rel in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def profiled_traffic(kernel):
    return PROFILED_TRAFFIC.get(kernel) if _sources_sha256() == PROFILED_TRAFFIC["sources_sha256"] else None


def profiled_instructions(kernel):
    return PROFILED_INSTRUCTIONS.get(kernel) if _sources_sha256() == PROFILED_INSTRUCTIONS["sources_sha256"] else None


def alu_peaks(dev, local):
    """Measured throughput of the FP32 FMA pipe (scalar and packed f32x2, lane operations) and of
    the special-function unit's ex2.approx on this GPU, from the library's probe kernels: a grid of
    8 blocks of 256 threads per SM, 8 independent chains a thread, best of 5 timed launches, with
    the SM clock sampled meanwhile."""
    import torch
    from paper_2402_17427_gb300 import binding as B
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, iters = sms * 8, 16384
    scratch = torch.empty(blocks * 256, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    clocks = ClockSampler(local)
    clocks.start()
    out = {}
    t_end = time.time() + 0.6          # long enough for a few clock samples
    best = {0: 1e30, 1: 1e30, 2: 1e30}
    while True:
        for kind in (0, 1, 2):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            B.vg_alu_probe(kind, blocks, iters, scratch.data_ptr(), stream)
            b.record()
            torch.cuda.synchronize()
            best[kind] = min(best[kind], a.elapsed_time(b))
        if time.time() > t_end:
            break
    clk = clocks.stop()
    ops = blocks * 256 * iters * 8
    out["ffma_tops"] = ops / (best[0] * 1e-3) / 1e12
    out["ffma2_lane_tops"] = 2 * ops / (best[1] * 1e-3) / 1e12
    out["ex2_tops"] = ops / (best[2] * 1e-3) / 1e12
    out["sm_mhz"] = clk["sm_mhz"] if clk else None
    out["sms"] = sms
    if clk and clk.get("sm_mhz"):
        f = clk["sm_mhz"] * 1e6
        out["ffma_per_sm_clk"] = out["ffma_tops"] * 1e12 / (sms * f)
        out["ffma2_lanes_per_sm_clk"] = out["ffma2_lane_tops"] * 1e12 / (sms * f)
        out["ex2_per_sm_clk"] = out["ex2_tops"] * 1e12 / (sms * f)
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle work for the CPU baseline")
    ap.add_argument("--cpu-single-thread", action="store_true",
                    help="also time the CPU baseline on one host thread (adds about a minute)")
    ap.add_argument("--no-patterns", action="store_true", help="skip the batched-cells and serving measurements")
    ap.add_argument("--serve-seconds", type=float, default=30.0)
    ap.add_argument("--only-pattern", choices=["appearance", "evaluation", "optimiser", "partition", "memory_scale",
                                               "batched_cells", "serving"],
                    help="run one pattern measurement on one GPU, print its JSON and exit (no step line)")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------ dist

def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def slowest_ms(pg, ms, device):
    """Per-step time of the whole job: the slowest rank's (max over ranks); ms itself with no group.
    Every rank must call it (a collective)."""
    if pg is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_rate(ws, ms):
    """Steps per second of the whole job: each of the ws ranks runs one step of its own replica in
    every ms-long step of the slowest rank."""
    return ws * 1000.0 / ms


# ------------------------------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------------------ CPU oracle

def oracle_step_time(g, cam, target, budget_s: float, seed: int = 0, threads: int | None = None):
    """Seconds one full step takes on the FP64 oracle, from a bounded sample (on all host cores
    unless `threads` is given).

    The projection, pair generation and sort of all N Gaussians run in full (an empty tile mask);
    compositing + adjoint run on a random sample of tiles and are scaled by total/sampled tiles;
    the loss runs on a 270x480 crop and is scaled by the pixel ratio.
    """
    import oracle
    threads = threads or os.cpu_count() or 1
    opts = oracle.Options(n_threads=threads)
    sc = oracle.Scene64.of(g)
    tiles_x, tiles_y = (cam.width + 15) // 16, (cam.height + 15) // 16
    ntiles = tiles_x * tiles_y
    t0 = time.perf_counter()
    oracle.render(sc, cam, opts, tile_mask=np.zeros(ntiles, np.uint8))
    t_proj = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    k = 8
    per_tile = None
    spent = t_proj
    while True:
        tiles = rng.choice(ntiles, k, replace=False)
        mask = np.zeros(ntiles, np.uint8)
        mask[tiles] = 1
        t0 = time.perf_counter()
        r = oracle.render(sc, cam, opts, tile_mask=mask)
        w = np.zeros((3, cam.height, cam.width))
        pm = np.repeat(np.repeat(mask.reshape(tiles_y, tiles_x).astype(bool), 16, 0), 16, 1)[:cam.height, :cam.width]
        w[:, pm] = 1.0 / w.size
        r.backward(w)
        dt = time.perf_counter() - t0
        spent += dt
        per_tile = max(1e-9, dt - t_proj) / k
        if spent > 0.5 * budget_s or k >= ntiles // 4:
            break
        k = min(ntiles // 4, max(2 * k, int(k * 0.5 * budget_s / max(dt, 1e-3))))
    crop = (slice(None), slice(0, min(270, cam.height)), slice(0, min(480, cam.width)))
    x = np.ascontiguousarray(r.image[crop])
    y = np.ascontiguousarray(np.asarray(target, np.float64)[crop])
    t0 = time.perf_counter()
    oracle.loss_l1_dssim(x, y, 0.2)
    t_loss = (time.perf_counter() - t0) * (cam.width * cam.height) / (x.shape[1] * x.shape[2])
    step = t_proj + per_tile * ntiles + t_loss
    sample = (f"full projection+sort of {g.n} Gaussians, compositing+adjoint of {k} of {ntiles} tiles "
              f"(scaled x{ntiles / k:.1f}), loss on a {x.shape[2]}x{x.shape[1]} crop (scaled by pixels)")
    return step, threads, sample


def oracle_sampled_step(g, cam, target, frac: float, seed: int):
    """One sampled step of the oracle: the projection and pair sort of every Gaussian, compositing
    and adjoint of a random `frac` of the tiles, the loss on a 480x270 crop.  Returns (seconds this
    took, the full-step seconds it stands for, threads, sample description)."""
    import oracle
    threads = os.cpu_count() or 1
    opts = oracle.Options(n_threads=threads)
    sc = oracle.Scene64.of(g)
    tiles_x, tiles_y = (cam.width + 15) // 16, (cam.height + 15) // 16
    ntiles = tiles_x * tiles_y
    k = max(1, int(round(frac * ntiles)))
    rng = np.random.default_rng(seed)
    mask = np.zeros(ntiles, np.uint8)
    mask[rng.choice(ntiles, k, replace=False)] = 1
    t0 = time.perf_counter()
    oracle.render(sc, cam, opts, tile_mask=np.zeros(ntiles, np.uint8))
    t_proj = time.perf_counter() - t0
    t0 = time.perf_counter()
    r = oracle.render(sc, cam, opts, tile_mask=mask)
    w = np.zeros((3, cam.height, cam.width))
    pm = np.repeat(np.repeat(mask.reshape(tiles_y, tiles_x).astype(bool), 16, 0), 16, 1)[:cam.height, :cam.width]
    w[:, pm] = 1.0 / w.size
    r.backward(w)
    t_tiles = max(1e-9, time.perf_counter() - t0 - t_proj)
    crop = (slice(None), slice(0, min(270, cam.height)), slice(0, min(480, cam.width)))
    x = np.ascontiguousarray(r.image[crop])
    y = np.ascontiguousarray(np.asarray(target, np.float64)[crop])
    t0 = time.perf_counter()
    oracle.loss_l1_dssim(x, y, 0.2)
    t_loss = time.perf_counter() - t0
    px_ratio = (cam.width * cam.height) / (x.shape[1] * x.shape[2])
    actual = t_proj + (t_proj + t_tiles) + t_loss        # the sampled render projects again
    full = t_proj + t_tiles * ntiles / k + t_loss * px_ratio
    sample = (f"per step: projection and pair sort of all {g.n} Gaussians, compositing + adjoint of a random "
              f"{k} of {ntiles} tiles (scaled x{ntiles / k:.2f}), loss on a {x.shape[2]}x{x.shape[1]} crop (scaled "
              f"x{px_ratio:.1f}); value = full steps per second from the scaled times, ms_per_step = the sampled "
              "step's own time")
    return actual, full, threads, sample


def run_reference(args, ws, rank):
    """The oracle as the reference arm: each step a bounded sample of the same workload on the host
    cores, reported as full steps per second, with ms_per_step the time the sampled steps took."""
    if rank != 0:
        return
    from paper_2402_17427_gb300 import scenes
    import oracle
    oracle.build()
    g, cam, target = scenes.blob_cell_1080p()
    actual, full = [], []
    for i in range(args.warmup + args.steps):
        a, f, threads, sample = oracle_sampled_step(g, cam, target, 0.125, seed=i)
        if i >= args.warmup:
            actual.append(a)
            full.append(f)
    v = 1.0 / float(np.mean(full))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(actual)) * 1e3,
            "full_step_ms": float(np.mean(full)) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------ patterns

def batch_pattern(dev, steps=10, warmup=3):
    """Eight uneven aerial cells trained together (one batched call per stage) against the same
    cells trained one after another (three calls per cell), fwd + loss + bwd, same GPU."""
    import torch
    from paper_2402_17427_gb300 import batch as BT, rasterize as R, scenes
    cells = scenes.aerial_cells(step=0)
    params = [[t.to(dev) for t in R.to_device(c.gaussians, "cpu")] for c in cells]
    cams = [c.camera for c in cells]
    targets = [torch.from_numpy(c.target).to(dev) for c in cells]
    tuner = BT.AutoTuner()
    settings = [tuner.choose(p, 3, cam) for p, cam in zip(params, cams)]
    grads = [tuple(torch.empty_like(t) for t in p) for p in params]
    losses = [R.LossL1DSSIM(0.2) for _ in cells]
    br = BT.BatchRasterizer(settings, device=dev)
    ras = [R.Rasterizer(s, device=dev) for s in settings]

    def batched():
        outs = br.forward(params, 3, cams)
        dLs = [losses[k](outs[k][0], targets[k], reuse=True)[1] for k in range(len(cells))]
        br.backward(params, 3, cams, outs, dLs, grads=grads)

    def sequential():
        for k in range(len(cells)):
            rgb, T, last = ras[k].forward(*params[k], 3, cams[k])
            _, dL = losses[k](rgb, targets[k], reuse=True)
            ras[k].backward(*params[k], 3, cams[k], T, last, dL, grads=grads[k])

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    batched()
    sequential()
    br.check = "defer"
    for r in ras:
        r.check = "defer"
    ms_b = timed(batched)
    ms_s = timed(sequential)
    br.verify()
    for r in ras:
        r.verify()
    return {"workload": "8 aerial cells (0.3M..3.0M Gaussians, 11.8M total, SH3), 1152x864 nadir view each, "
                        "fwd + L1/D-SSIM + bwd for all cells",
            "batched_steps_per_s": 1000.0 / ms_b, "sequential_steps_per_s": 1000.0 / ms_s,
            "batched_ms": ms_b, "sequential_ms": ms_s, "speedup": ms_s / ms_b,
            "tiles": [s.tile_size for s in settings], "chunks": [s.chunk for s in settings]}


def _time_cuda(fn, reps=10, warmup=3):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def partition_pattern(dev, hbm_gbs):
    """Scene partition on the device (Sec. 4.1, 4.3): airspace boxes of 16 cells (20M points),
    visibility of those boxes in 4000 cameras, and the seamless merge of 16 cells whose Gaussians
    (1.25M each, SH3) cover their 20%-expanded rectangles.  Inputs are drawn on the device from a
    fixed seed."""
    import math
    import torch
    from paper_2402_17427_gb300 import partition as PT, scenes
    g = torch.Generator(device=dev)
    g.manual_seed(6000)
    n_cells, per, cell = 16, 1_250_000, 250.0
    cells, regions, offs = [], [], [0]
    for k in range(n_cells):
        x0, z0 = cell * (k % 4), cell * (k // 4)
        lo = torch.tensor([x0 - 0.1 * cell, 0.0, z0 - 0.1 * cell], device=dev)
        ext = torch.tensor([1.2 * cell, 60.0, 1.2 * cell], device=dev)
        means = lo + ext * torch.rand((per, 3), device=dev, generator=g)
        cells.append((means, torch.randn((per, 3), device=dev, generator=g) - 2.0,
                      torch.randn((per, 4), device=dev, generator=g), torch.randn((per,), device=dev, generator=g),
                      torch.randn((per, 16, 3), device=dev, generator=g)))
        regions.append((x0, x0 + cell, z0, z0 + cell))
        offs.append(offs[-1] + per)
    points = torch.cat([c[0] for c in cells]).contiguous()
    t_box = _time_cuda(lambda: PT.airspace_boxes(points, offs, 0.0))
    boxes = PT.airspace_boxes(points, offs, 0.0)
    rng = np.random.default_rng(6001)
    cams = []
    for i in range(4000):
        W, H = scenes.RESOLUTIONS[i % 3]
        yaw, pitch = rng.uniform(0, 2 * math.pi), math.radians(rng.uniform(-90, -30))
        eye = (rng.uniform(0, 1000), rng.uniform(20, 150), rng.uniform(0, 1000))
        cams.append(scenes.camera_from_forward(eye, scenes.yaw_pitch_forward(yaw, pitch), W, H))
    table = PT.camera_table(cams)      # marshalled once; the timed call is the C-ABI call
    t_vis = _time_cuda(lambda: PT.camera_visibility(boxes, table))
    vis, sel = PT.camera_visibility(boxes, table)
    t_merge = _time_cuda(lambda: PT.merge_cells(cells, regions, 3), reps=5, warmup=2)
    merged = PT.merge_cells(cells, regions, 3)
    m, total = int(merged[0].shape[0]), n_cells * per
    # algorithmic bytes: every mean read (12 B), the 236 B of each kept Gaussian read and written
    merge_bytes = 12 * total + 2 * 236 * m
    box_bytes = 12 * total
    return {"workload": "16 cells x 1.25M Gaussians (SH3) over 20%-expanded 250 m cells; 4000 cameras "
                        "(720p/1080p/4K, 20-150 m, pitch -90..-30 deg)",
            "airspace_boxes_ms": t_box, "airspace_boxes_gbs": box_bytes / (t_box * 1e-3) / 1e9,
            "visibility_ms": t_vis, "visibility_pairs_per_s": 4000 * n_cells / (t_vis * 1e-3),
            "cameras_selected_per_cell_mean": float(sel.float().sum(0).mean()),
            "merge_ms": t_merge, "merged": m, "merge_gbs": merge_bytes / (t_merge * 1e-3) / 1e9,
            "merge_hbm_frac": merge_bytes / (t_merge * 1e-3) / 1e9 / hbm_gbs,
            "note": "times include each call's argument marshalling and output allocation"}


def optimiser_pattern(dev, hbm_gbs):
    """The optimiser step at the benchmark cell's size (1M Gaussians, SH3): one fused Adam update
    of every parameter, and one clone / split / prune pass with a mix of decisions."""
    import torch
    from paper_2402_17427_gb300 import optim as OP
    n, K = 1_000_000, 16
    g = torch.Generator(device=dev)
    g.manual_seed(8000)
    shapes = [(n, 3), (n, 3), (n, 4), (n,), (n, K, 3)]
    params = [torch.randn(sh, device=dev, generator=g) for sh in shapes]
    params[1] = params[1] * 0.8 + math.log(0.05)
    params[3] = params[3] * 3.0
    grads = [torch.randn(sh, device=dev, generator=g) * 1e-2 for sh in shapes]
    adam = OP.Adam(params)
    t_adam = _time_cuda(lambda: adam.step(params, grads, 3), reps=20, warmup=3)
    # each parameter scalar: p, g, m, v read and p, m, v written
    scalars = n * (3 + 3 + 4 + 1 + 3 * K)
    adam_bytes = 7 * 4 * scalars
    acc = torch.empty(n, device=dev).exponential_(1.0 / 3e-4, generator=g)
    cnt = torch.randint(0, 4, (n,), device=dev, generator=g, dtype=torch.int32)
    normals = torch.randn((n, 2, 3), device=dev, generator=g)
    ds = OP.DensifySettings(scene_extent=10.0)
    state = {}

    def one():
        a = OP.Adam.__new__(OP.Adam)
        a.m, a.v = adam.m, adam.v
        st = OP.DensifyStats.__new__(OP.DensifyStats)
        st.accum, st.count = acc, cnt
        state["new"] = OP.densify_with(params, a, st, 3, ds, normals)

    t_dens = _time_cuda(one, reps=5, warmup=2)
    m = int(state["new"][0].shape[0])
    # read: every Gaussian's decision inputs and its parameters + moments (3 x 236 B) once;
    # written: 3 x 236 B per emitted Gaussian
    dens_bytes = n * (12 + 4 + 4 + 4) + 3 * 236 * (n + m)
    return {"workload": "1M Gaussians, SH3 (59 floats each); densify with random statistics "
                        "(prune / keep / clone / split mix)",
            "adam_ms": t_adam, "adam_gbs": adam_bytes / (t_adam * 1e-3) / 1e9,
            "adam_hbm_frac": adam_bytes / (t_adam * 1e-3) / 1e9 / hbm_gbs,
            "densify_ms": t_dens, "densify_out": m, "densify_gbs": dens_bytes / (t_dens * 1e-3) / 1e9,
            "densify_hbm_frac": dens_bytes / (t_dens * 1e-3) / 1e9 / hbm_gbs,
            "note": "densify time includes its output allocation"}


def evaluation_pattern(dev, hbm_gbs):
    """Colour-corrected PSNR / SSIM (Sec. 5.1) of a 1920x1080 rendering against its target."""
    import torch
    from paper_2402_17427_gb300 import rasterize as R
    g = torch.Generator(device=dev)
    g.manual_seed(7000)
    y = torch.rand((3, 1080, 1920), device=dev, generator=g)
    x = (0.8 * y + 0.1 + 0.05 * torch.randn((3, 1080, 1920), device=dev, generator=g)).clamp(0, 1)
    t = _time_cuda(lambda: R.color_corrected_metrics(x, y), reps=20, warmup=3)
    out = R.color_corrected_metrics(x, y).cpu().tolist()
    # algorithmic bytes: both images read by the two fitting passes and the correction, the
    # corrected image written, then read with the target by the SSIM pass
    px = 1920 * 1080
    nbytes = (3 * 2 + 1 + 2) * 3 * 4 * px
    return {"workload": "1920x1080 rendering vs target (affine colour shift + noise)", "ms": t,
            "images_per_s": 1000.0 / t, "psnr": out[0], "ssim": out[1],
            "gbs": nbytes / (t * 1e-3) / 1e9, "hbm_frac": nbytes / (t * 1e-3) / 1e9 / hbm_gbs}


def appearance_pattern(dev, bf16_tflops):
    """The appearance loss of Eq. 3 (Sec. 4.2) on one 1920x1080 training view, forward and
    backward: pooling, the CNN and its adjoint, the map, L1 and D-SSIM, every gradient."""
    import torch
    from paper_2402_17427_gb300 import appearance as AP
    g = torch.Generator(device=dev)
    g.manual_seed(9000)
    H, W = 1080, 1920
    y = torch.rand((3, H, W), device=dev, generator=g)
    x = (0.9 * y + 0.05 + 0.05 * torch.randn((3, H, W), device=dev, generator=g)).clamp(0, 1)
    model = AP.AppearanceModel(4, seed=9001, device=dev)
    t_full = _time_cuda(lambda: model.loss(x, y, 1), reps=20, warmup=3)
    t_fwd = _time_cuda(lambda: model.loss(x, y, 1, grad=False), reps=20, warmup=3)
    # algorithmic FLOPs of the network as defined (dense 3x3 convolutions), forward; the backward
    # pass costs two such products per layer (input gradient, weight gradient)
    h, w = H // 32, W // 32
    fwd = 0
    for k, (c, o) in enumerate(AP.LAYERS):
        px = (h << min(k, 4)) * (w << min(k, 4)) if k < 5 else H * W
        fwd += 2 * px * o * 9 * c
    tf32_peak = bf16_tflops * 1.1 / 2.25      # dense TF32 / BF16 nominal ratio
    return {"workload": "1920x1080 view, 64-float embedding, CNN 67->256->...->16 at 528x960, "
                        "bilinear to 1080p, 16->16->3 head; lambda 0.2",
            "fwd_bwd_ms": t_full, "fwd_ms": t_fwd, "views_per_s": 1000.0 / t_full,
            "gflop_fwd_bwd": 3 * fwd / 1e9,
            "tflops_fwd_bwd": 3 * fwd / (t_full * 1e-3) / 1e12,
            "tf32_frac": 3 * fwd / (t_full * 1e-3) / 1e12 / tf32_peak,
            "tf32_peak_tflops": tf32_peak,
            "peak_source": "MEASURED_PEAKS.json bf16_tflops x 1.1 / 2.25 (nominal TF32 / BF16)"}


def memory_scale_pattern(dev, steps=5, warmup=2):
    """The differentiable cell at memory scale (pattern 3): 20M Gaussians (SH3) on urban facades
    and ground, one 1920x1080 view, a training step through the torch.autograd.Functions (render,
    Eq. 1 loss, backward from the stored final transmittance) with every gradient returned."""
    import torch
    from paper_2402_17427_gb300 import binding as B, rasterize as R, scenes
    g, cam, target = scenes.urban_cell_20m()
    params = [t.to(dev).requires_grad_(True) for t in R.to_device(g, "cpu")]
    tgt = torch.from_numpy(target).to(dev)
    ras = R.Rasterizer(device=dev, check="sync")
    lossobj = R.LossL1DSSIM(0.2)

    def step():
        img = R.rasterize(*params, g.sh_degree, cam, ras)
        L = R.l1_dssim_loss(img, tgt, 0.2, lossobj)
        return torch.autograd.grad(L, params)

    step()                         # sizes the pair list (one synchronous check)
    torch.cuda.synchronize()
    ras.check = "defer"
    torch.cuda.reset_peak_memory_stats(dev)
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = B.vg_kernel_launches()
    e0.record()
    for _ in range(steps):
        grads = step()
    e1.record()
    torch.cuda.synchronize()
    launches = (B.vg_kernel_launches() - launches0) / steps
    ras.verify()
    ms = e0.elapsed_time(e1) / steps
    cnt = ras.counters.cpu().numpy()
    assert all(bool(torch.isfinite(t).all()) for t in grads)
    return {"workload": "urban cell: 20,000,000 Gaussians (SH3) on ~150 building facades and ground in "
                        "500x500x60 m, one 1920x1080 view at 80 m pitched -45 deg; render + L1/D-SSIM + "
                        "backward through torch.autograd, gradients of all 20M",
            "ms_per_step": ms, "steps_per_s": 1000.0 / ms,
            "peak_device_bytes": int(torch.cuda.max_memory_allocated(dev)),
            "parameter_bytes": int(sum(t.numel() * 4 for t in params)),
            "workspace_bytes": int(ras.ws.buf.numel()), "pair_capacity": int(ras.ws.capacity),
            "pairs": int(cnt[B.VG_CNT_PAIRS]), "visible": int(cnt[B.VG_CNT_VISIBLE]),
            "library_launches_per_step": launches}


def serving_pattern(dev, seconds=30.0):
    """The merged 20M-Gaussian city (16 cells) served under a 200 req/s Poisson stream."""
    from paper_2402_17427_gb300 import scenes, serving
    cells = scenes.merged_city()
    srv = serving.SceneServer(cells, device=dev, slots=3, max_batch=8)
    reqs = scenes.request_stream(duration_s=seconds)
    srv.render([r.camera for r in reqs[:4]])      # allocate workspaces, learn the pairs ratio
    st = srv.serve(reqs, warmup_s=2.0)
    d = st.summary()
    d["workload"] = ("merged city: 16 cells, 20M Gaussians SH3 resident; Poisson 200 req/s for %.0f s; "
                     "50%% 1280x720, 35%% 1920x1080, 15%% 3840x2160; first 2 s excluded" % seconds)
    d["resident_gb"] = srv.resident_bytes / 1e9
    # The same server offered more than it can take (Poisson 3000 req/s for 4 s, same resolution
    # mix): the queue grows, so the throughput over the run, drain included, is the service
    # capacity, and latencies are queueing-dominated.  Once with batches of up to max_batch
    # requests, once with one request a batch (the same 3 slots in flight).
    keys = ("requests", "duration_s", "throughput_rps", "mpix_per_s", "mean_batch", "batches", "max_inflight",
            "p50_ms", "p99_ms", "rerenders")
    sat = {}
    for name, mb in (("batched", srv.max_batch), ("one_per_batch", 1)):
        full = srv.max_batch
        srv.max_batch = mb
        try:
            st = srv.serve(scenes.request_stream(seed=5001, rate_hz=3000.0, duration_s=4.0), warmup_s=0.5)
        finally:
            srv.max_batch = full
        sat[name] = {k: v for k, v in st.summary().items() if k in keys}
    sat["offered_rps"] = 3000.0
    sat["batching_speedup"] = sat["batched"]["throughput_rps"] / max(sat["one_per_batch"]["throughput_rps"], 1e-9)
    d["saturated"] = sat
    return d


# ------------------------------------------------------------------------------------------ GPU arm

def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import torch
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    from paper_2402_17427_gb300 import _build, binding as B, rasterize as R, scenes
    if rank == 0:
        _build.build()
    if args.only_pattern:
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            pass
        dev = torch.device("cuda", local)
        fn = {"appearance": lambda: appearance_pattern(dev, float(peaks.get("bf16_tflops", 1900.0))),
              "evaluation": lambda: evaluation_pattern(dev, float(peaks.get("hbm_gbs", 6800.0))),
              "optimiser": lambda: optimiser_pattern(dev, float(peaks.get("hbm_gbs", 6800.0))),
              "partition": lambda: partition_pattern(dev, float(peaks.get("hbm_gbs", 6800.0))),
              "memory_scale": lambda: memory_scale_pattern(dev),
              "batched_cells": lambda: batch_pattern(dev),
              "serving": lambda: serving_pattern(dev, args.serve_seconds)}[args.only_pattern]
        if rank == 0:
            print(json.dumps({"pattern": args.only_pattern, **fn()}), flush=True)
        return
    if pg:
        pg.barrier()
    g, cam, target = scenes.blob_cell_1080p()
    dev = torch.device("cuda", local)
    params = [t.to(dev) for t in R.to_device(g, "cpu")]
    target_t = torch.from_numpy(target).to(dev)
    ras = R.Rasterizer(R.RasterSettings(), device=dev, check="sync")
    lossf = R.LossL1DSSIM(0.2)

    def step(evf=None, evb=None, prm=None, tgt=None, lf=None, lev=None):
        prm = params if prm is None else prm
        tgt = target_t if tgt is None else tgt
        rgb, T, last = ras.forward(*prm, g.sh_degree, cam, events=evf)
        if lev:
            lev[0].record()
        L, dL = (lf or lossf)(rgb, tgt, reuse=True)
        if lev:
            lev[1].record()
        grads = ras.backward(*prm, g.sh_degree, cam, T, last, dL, grads=step.grads, events=evb)
        return L, T, last

    step.grads = tuple(torch.empty_like(t) for t in params)
    # size the pair list once (synchronous check), then run without host synchronisation
    step()
    torch.cuda.synchronize()
    ras.check = "defer"
    # exact evaluation / blend counts of one step (untimed)
    ras.settings.count_blends = True
    _, _, last = step()
    torch.cuda.synchronize()
    cnt = ras.counters.cpu().numpy()
    evals_f, blends_f = int(cnt[B.VG_CNT_EVALS]), int(cnt[B.VG_CNT_BLENDS])
    evals_run_f = int(cnt[B.VG_CNT_EVALS_RUN])
    evals_b = int(last.to(torch.int64).sum().item())
    P, V = int(cnt[B.VG_CNT_PAIRS]), int(cnt[B.VG_CNT_VISIBLE])
    # the backward's executed pixel slots (same step's workspace, counting backward)
    cnt_t = torch.empty(B.VG_CNT_LEN, dtype=torch.int64, device=dev)
    B.vg_read_counters(ras.ws.buf.data_ptr(), ras.ws.buf.numel(), cnt_t.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    evals_run_b = int(cnt_t[B.VG_CNT_EVALS_RUN_BWD].item())
    ras.settings.count_blends = False

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    K = args.steps
    stage_ev = []
    for _k in range(K):
        evs = B.vg_stage_events()
        keep = []
        for s in range(B.VG_STAGE_COUNT):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()      # torch creates the CUDA event on first record; the library records it again
            b.record()
            keep += [a, b]
            evs.begin[s], evs.end[s] = a.cuda_event, b.cuda_event
        stage_ev.append((evs, keep))
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = B.vg_kernel_launches()
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(K)]   # each step's start, for the spread
    start.record()
    for k in range(K):
        marks[k].record()
        step(stage_ev[k][0], stage_ev[k][0])
    end.record()
    torch.cuda.synchronize()
    launches = B.vg_kernel_launches() - launches0
    per_step = [marks[k].elapsed_time(marks[k + 1] if k + 1 < K else end) for k in range(K)]
    clk = clocks.stop()
    if pg:
        pg.barrier()
    ras.verify()
    ms = slowest_ms(pg, start.elapsed_time(end) / K, dev)
    stage_ms = {}
    names = ["project", "sort", "blend", "blend_backward", "project_backward"]
    for s, nm in enumerate(names):
        stage_ms[nm] = float(np.mean([stage_ev[k][1][2 * s].elapsed_time(stage_ev[k][1][2 * s + 1]) for k in range(K)]))
    # the loss call (Eq. 1, both SSIM passes and the reduction), timed in further steps after the
    # timed region (its two events inside it would add to the step), and what no stage covers:
    # launch gaps between the calls and the small kernels outside the stages
    KL = min(K, 50)
    lev = [[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in range(KL)]
    for k in range(KL):
        step(lev=lev[k])
    torch.cuda.synchronize()
    ras.verify()
    stage_ms["loss"] = float(np.mean([a.elapsed_time(b) for a, b in lev]))
    stage_ms["unstaged"] = float(ms - sum(stage_ms.values()))

    # e2e: the same step from pinned host buffers, every step's inputs copied in and its loss copied
    # out inside the timed region.  Two device input sets: step k computes on one while step k+1's
    # inputs are copied into the other on a copy stream (a training loop fed from host memory).
    e2e = None
    if not args.no_e2e:
        host = [t.cpu().pin_memory() for t in params]
        host_target = target_t.cpu().pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in host) + host_target.numel() * 4
        dsets = [params, [torch.empty_like(t) for t in params]]
        dtg = [target_t, torch.empty_like(target_t)]
        comp, cs, ds = torch.cuda.current_stream(), torch.cuda.Stream(), torch.cuda.Stream()
        ready = [torch.cuda.Event(), torch.cuda.Event()]
        free = [torch.cuda.Event(), torch.cuda.Event()]
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        lossfs = [R.LossL1DSSIM(0.2), R.LossL1DSSIM(0.2)]   # step k writes its loss into set k % 2

        def upload(b):
            with torch.cuda.stream(cs):
                cs.wait_event(free[b])        # the step that last read input set b has finished
                for d, h in zip(dsets[b], host):
                    d.copy_(h, non_blocking=True)
                dtg[b].copy_(host_target, non_blocking=True)
                ready[b].record(cs)

        def run(n, out):
            free[0].record(comp)
            free[1].record(comp)
            copied[0].record(comp)
            copied[1].record(comp)
            upload(0)
            for i in range(n):
                b = i & 1
                if i + 1 < n:
                    upload(1 - b)
                comp.wait_event(ready[b])
                comp.wait_event(copied[b])    # step i - 2's loss, in the same set, has reached the host
                L = step(prm=dsets[b], tgt=dtg[b], lf=lossfs[b])[0]
                free[b].record(comp)
                # the step's loss, device to host, on a third stream so that the next step's kernels
                # do not queue behind the copy
                with torch.cuda.stream(ds):
                    ds.wait_event(free[b])
                    out[i].copy_(L.view(-1)[:1], non_blocking=True)
                    copied[b].record(ds)

        ke = max(3, K // 2)
        losses = torch.empty((ke, 1), dtype=torch.float32).pin_memory()
        run(2, losses)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run(ke, losses)
        comp.wait_stream(ds)       # the timed region ends after the last loss has reached the host
        e1.record()
        torch.cuda.synchronize()
        assert bool(torch.isfinite(losses).all())       # every step's loss, read on the host
        ems = slowest_ms(pg, e0.elapsed_time(e1) / ke, dev)
        # the copies alone (same tensors, same copy stream, nothing computing): the host-to-device
        # link's rate, and the step rate it alone would allow
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(2):
            upload(0)
        torch.cuda.synchronize()
        c0.record(cs)
        for _ in range(5):
            upload(0)
        c1.record(cs)
        torch.cuda.synchronize()
        copy_ms = c0.elapsed_time(c1) / 5
        e2e = {"value": job_rate(ws, ems), "unit": "steps/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": 4, "pipelined": "inputs of step k+1 copied during step k",
               "h2d_copy_ms": copy_ms, "h2d_gbs": h2d / copy_ms / 1e6,
               "copy_bound_steps_per_s": job_rate(ws, copy_ms)}
        ras.verify()

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return

    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    alu = alu_peaks(dev, local)
    # measured FP32 FMA pipe rate in lane operations: the packed form (two lanes an instruction)
    # reaches the pipe's rate with half the issue slots, so it is the larger of the two probes
    peak_ops = max(alu["ffma_tops"], alu["ffma2_lane_tops"])
    fwd_ops = OPS_EVAL * evals_f + OPS_BLEND_FWD * blends_f
    bwd_ops = OPS_EVAL * evals_b + OPS_BLEND_BWD * blends_f
    # the same per-evaluation counts over the slots the kernels execute after their warp culling
    fwd_ops_x = OPS_EVAL * evals_run_f + OPS_BLEND_FWD * blends_f
    bwd_ops_x = OPS_EVAL * evals_run_b + OPS_BLEND_BWD * blends_f
    kern = {"blend": fwd_ops / (stage_ms["blend"] * 1e-3) / 1e12,
            "blend_backward": bwd_ops / (stage_ms["blend_backward"] * 1e-3) / 1e12}
    kern_x = {"blend": fwd_ops_x / (stage_ms["blend"] * 1e-3) / 1e12,
              "blend_backward": bwd_ops_x / (stage_ms["blend_backward"] * 1e-3) / 1e12}
    dom = max(("blend", "blend_backward"), key=lambda k: stage_ms[k])
    clk_mhz = (clk or {}).get("sm_mhz") or alu.get("sm_mhz") or 2070.0
    inst = profiled_instructions(dom)
    issue_frac = (inst / (sms * 4 * clk_mhz * 1e6 * stage_ms[dom] * 1e-3)) if inst else None
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    F = 11 + 3 * 16
    N, px = g.n, cam.width * cam.height
    step_bytes = N * (4 * F + 12) + V * (8 * F + 156) + 116 * P + 76 * px
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        try:
            t, threads, sample = oracle_step_time(g, cam, target, args.cpu_budget)
            cpu = {"value": 1.0 / t, "unit": "steps/s", "cores": threads, "kind": "oracle", "sample": sample}
            if args.cpu_single_thread:
                t1, _, sample1 = oracle_step_time(g, cam, target, args.cpu_budget, seed=1, threads=1)
                cpu["single_thread"] = {"value": 1.0 / t1, "unit": "steps/s", "cores": 1, "sample": sample1}
        except Exception as e:  # the oracle is test infrastructure; report, never fail the GPU number
            cpu = {"value": None, "unit": "steps/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"failed: {e}"}
    patterns = None
    if not args.no_patterns and ws == 1:
        try:
            patterns = {"batched_cells": batch_pattern(dev), "serving": serving_pattern(dev, args.serve_seconds),
                        "memory_scale": memory_scale_pattern(dev),
                        "partition": partition_pattern(dev, hbm), "evaluation": evaluation_pattern(dev, hbm),
                        "optimiser": optimiser_pattern(dev, hbm),
                        "appearance": appearance_pattern(dev, bf16_peak)}
        except Exception as e:  # report, never lose the main number
            patterns = {"error": repr(e)}
    line = {
        "metric": METRIC, "value": job_rate(ws, ms), "unit": "steps/s", "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "step_ms": {"median": float(np.median(per_step)), "p90": float(np.percentile(per_step, 90)),
                    "min": float(np.min(per_step)), "max": float(np.max(per_step))},
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "gaussians": N, "width": cam.width, "height": cam.height,
                   "sh_degree": g.sh_degree, "tile": 16, "visible": V, "pairs": P,
                   "l2": "inputs larger than L2 (236 MB of parameters per step), no flush",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "roofline": {"bound": "alu", "kernel": dom, "achieved": kern[dom], "peak": peak_ops,
                     "unit": "FP32 Tops/s", "frac": kern[dom] / peak_ops, "traffic": profiled_traffic(dom),
                     "achieved_executed": kern_x[dom], "frac_executed": kern_x[dom] / peak_ops,
                     "issue_frac": issue_frac,
                     "peak_source": "measured: vg_alu_probe FP32 FMA lane rate on this GPU (the larger of the "
                                    f"scalar and packed probes; {sms} SMs, SM clock {alu.get('sm_mhz')} MHz during "
                                    "the probe)",
                     "alu_probe": alu},
        "stage_ms": stage_ms,
        "blends": {"evals_fwd": evals_f, "blends_fwd": blends_f, "evals_bwd": evals_b,
                   "evals_run_fwd": evals_run_f, "evals_run_bwd": evals_run_b,
                   "fwd_evals_per_s": evals_f / (stage_ms["blend"] * 1e-3),
                   "bwd_evals_per_s": evals_b / (stage_ms["blend_backward"] * 1e-3),
                   "fwd_tops": kern["blend"], "bwd_tops": kern["blend_backward"]},
        "step_hbm": {"bytes": int(step_bytes), "achieved_gbs": step_bytes / (ms * 1e-3) / 1e9, "peak_gbs": hbm,
                     "frac": step_bytes / (ms * 1e-3) / 1e9 / hbm, "peak_source": "MEASURED_PEAKS.json hbm_gbs"},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
        "patterns": patterns,
    }
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
