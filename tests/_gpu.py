"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI, read back its
state, and pick the Gaussians that can reach a set of sampled tiles so the oracle only has to
project those.  Nothing here computes any part of the rasteriser itself."""
from __future__ import annotations

import math

import numpy as np
import torch

import oracle
from paper_2402_17427_gb300 import binding as B
from paper_2402_17427_gb300 import rasterize as R


def run_forward(g, cam, settings=None, capacity=None, check="sync"):
    """Forward through the C ABI; returns (rasterizer, device params, dict of numpy results)."""
    settings = settings or R.RasterSettings()
    r = R.Rasterizer(settings, pair_capacity=capacity, check=check)
    params = R.to_device(g)
    rgb, T, last = r.forward(*params, g.sh_degree, cam)
    torch.cuda.synchronize()
    out = dict(image=rgb.cpu().numpy(), T=T.cpu().numpy(), last=last.cpu().numpy().astype(np.int64),
               counters=r.counters.cpu().numpy(), rgb_t=rgb, T_t=T, last_t=last)
    return r, params, out


def read_state(r: R.Rasterizer, g, cam):
    opts = r.settings.c()
    tiles_x = (cam.width + opts.tile_size - 1) // opts.tile_size
    tiles_y = (cam.height + opts.tile_size - 1) // opts.tile_size
    dev = r.ws.buf.device
    ranges = torch.zeros((tiles_x * tiles_y, 2), dtype=torch.int32, device=dev)
    ids = torch.zeros(r.ws.capacity, dtype=torch.int32, device=dev)
    proj = torch.zeros((max(g.n, 1), 12), dtype=torch.float32, device=dev)
    touched = torch.zeros(max(g.n, 1), dtype=torch.int32, device=dev)
    B.vg_read_render_state(r.ws.buf.data_ptr(), r.ws.buf.numel(), g.n, cam.width, cam.height, r.ws.capacity, opts,
                           ranges.data_ptr(), ids.data_ptr(), proj.data_ptr(), touched.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return dict(ranges=ranges.cpu().numpy().astype(np.int64), ids=ids.cpu().numpy().view(np.uint32),
                proj=proj.cpu().numpy()[:g.n], touched=touched.cpu().numpy()[:g.n])


def run_backward(r, params, g, cam, out, dL, means2d_abs=None):
    dL_t = torch.from_numpy(np.ascontiguousarray(dL, np.float32)).cuda()
    grads = r.backward(*params, g.sh_degree, cam, out["T_t"], out["last_t"], dL_t, means2d_abs=means2d_abs)
    torch.cuda.synchronize()
    names = ["means", "log_scales", "quats", "logits", "sh"]
    return {k: v.cpu().numpy().astype(np.float64) for k, v in zip(names, grads)}


def oracle_opts(settings: R.RasterSettings, **kw) -> oracle.Options:
    return oracle.Options(tile=settings.tile_size, stop_rule=settings.stop_rule, bg=tuple(settings.bg),
                          dilation=settings.dilation, alpha_max=settings.alpha_max, alpha_min=settings.alpha_min,
                          t_min=settings.t_min, guard=settings.guard, **kw)


def tile_lists_equal(orc, gpu_state, tiles, exclude_ids=()):
    """Per sampled tile, the GPU list must equal the oracle list (Gaussian ids, in order) once the
    Gaussians whose rectangle edges are ambiguous are removed from both.  Returns mismatches."""
    ex = set(int(i) for i in exclude_ids)
    bad = []
    for t in tiles:
        s, e = orc.ranges[t]
        want = [int(i) for i in orc.vals[s:e] if int(i) not in ex]
        gs, ge = gpu_state["ranges"][t]
        got = [int(i) for i in gpu_state["ids"][gs:ge] if int(i) not in ex]
        if want != got:
            bad.append(t)
    return bad


def reachable_subset(g, cam, tiles, tile_size, guard=1.3, dilation=0.3, margin_px=4.0):
    """Indices (ascending) of every Gaussian whose tile rectangle could contain one of `tiles`.

    A conservative bound: the 2D covariance's largest eigenvalue is at most its trace, which is at
    most (|J row 0|^2 + |J row 1|^2) * max scale^2 + 2 dilation; with the guard-band clamp
    |J row 0|^2 <= (fx/z)^2 (1 + limx^2).  The subset keeps the original order, so ties in the
    depth sort are broken exactly as in the full set.
    """
    means = np.asarray(g.means, np.float64)
    R_ = np.asarray(cam.R, np.float64)
    p = means @ R_.T + np.asarray(cam.t, np.float64)
    z = p[:, 2]
    front = z > cam.near * 0.999
    zs = np.where(front, z, 1.0)
    limx = guard * 0.5 * cam.width / cam.fx
    limy = guard * 0.5 * cam.height / cam.fy
    smax2 = np.exp(2.0 * np.asarray(g.log_scales, np.float64).max(1))
    tr = ((cam.fx / zs) ** 2 * (1 + limx ** 2) + (cam.fy / zs) ** 2 * (1 + limy ** 2)) * smax2 + 2 * dilation
    rb = 3.0 * np.sqrt(tr) * 1.001 + margin_px
    u = cam.fx * p[:, 0] / zs + cam.cx
    v = cam.fy * p[:, 1] / zs + cam.cy
    tiles_x = (cam.width + tile_size - 1) // tile_size
    keep = np.zeros(len(means), bool)
    for t in tiles:
        ty, tx = divmod(int(t), tiles_x)
        x0, x1 = tx * tile_size, (tx + 1) * tile_size - 1
        y0, y1 = ty * tile_size, (ty + 1) * tile_size - 1
        dx = np.maximum(0.0, np.maximum(x0 - u, u - x1))
        dy = np.maximum(0.0, np.maximum(y0 - v, v - y1))
        keep |= front & (dx <= rb) & (dy <= rb)
    return np.nonzero(keep)[0]


def conservative_tile_rects(g, cam, tile_size, guard=1.3, dilation=0.3, margin_px=4.0):
    """For every Gaussian, a tile rectangle that contains every tile its own rectangle can reach
    (the bound of reachable_subset): returns (ok, tx0, tx1, ty0, ty1), ok false for a Gaussian
    behind the near plane or whose bound misses the image."""
    means = np.asarray(g.means, np.float64)
    R_ = np.asarray(cam.R, np.float64)
    p = means @ R_.T + np.asarray(cam.t, np.float64)
    z = p[:, 2]
    front = z > cam.near * 0.999
    zs = np.where(front, z, 1.0)
    limx = guard * 0.5 * cam.width / cam.fx
    limy = guard * 0.5 * cam.height / cam.fy
    smax2 = np.exp(2.0 * np.asarray(g.log_scales, np.float64).max(1))
    tr = ((cam.fx / zs) ** 2 * (1 + limx ** 2) + (cam.fy / zs) ** 2 * (1 + limy ** 2)) * smax2 + 2 * dilation
    rb = 3.0 * np.sqrt(tr) * 1.001 + margin_px
    u = cam.fx * p[:, 0] / zs + cam.cx
    v = cam.fy * p[:, 1] / zs + cam.cy
    tiles_x = (cam.width + tile_size - 1) // tile_size
    tiles_y = (cam.height + tile_size - 1) // tile_size
    x0 = np.floor((u - rb) / tile_size)
    x1 = np.floor((u + rb) / tile_size)
    y0 = np.floor((v - rb) / tile_size)
    y1 = np.floor((v + rb) / tile_size)
    ok = front & (x1 >= 0) & (x0 <= tiles_x - 1) & (y1 >= 0) & (y0 <= tiles_y - 1)
    clip = lambda a, hi: np.clip(np.nan_to_num(a, nan=0.0, posinf=hi, neginf=0.0), 0, hi).astype(np.int64)
    return ok, clip(x0, tiles_x - 1), clip(x1, tiles_x - 1), clip(y0, tiles_y - 1), clip(y1, tiles_y - 1)


def subset_reaching(rects, mask, tiles_x, tiles_y):
    """Indices (ascending) of the Gaussians whose conservative rectangle meets a tile of `mask`
    (uint8 [tiles]), by a 2D prefix sum over the mask."""
    ok, x0, x1, y0, y1 = rects
    m = np.asarray(mask, np.int64).reshape(tiles_y, tiles_x)
    S = np.zeros((tiles_y + 1, tiles_x + 1), np.int64)
    S[1:, 1:] = m.cumsum(0).cumsum(1)
    cnt = S[y1 + 1, x1 + 1] - S[y0, x1 + 1] - S[y1 + 1, x0] + S[y0, x0]
    return np.nonzero(ok & (cnt > 0))[0]


def group_errors(gpu, ref, keep_mask):
    """Per parameter group: relative L2 error over the kept Gaussians, and the worst element
    error normalised by (|ref| + 1e-3 max|ref|)."""
    out = {}
    for k in ("means", "log_scales", "quats", "logits", "sh"):
        a = gpu[k][keep_mask].reshape(-1)
        b = ref[k][keep_mask].reshape(-1)
        nb = np.linalg.norm(b)
        rel = np.linalg.norm(a - b) / max(nb, 1e-30)
        scale = np.abs(b).max() if b.size else 1.0
        elem = (np.abs(a - b) / (np.abs(b) + 1e-3 * scale + 1e-30)).max() if b.size else 0.0
        out[k] = (float(rel), float(elem), float(nb))
    return out
