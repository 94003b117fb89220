"""Oracle for the per-cell optimiser step (paper Sec. 3 and Sec. 5.1): Adam on the raw Gaussian
parameters and the adaptive densification that is triggered by the accumulated view-space
positional gradient (clone / split / prune every 200 iterations between iterations 1,000 and
30,000; the other settings are those of 3D Gaussian Splatting, which the paper defers to).

TEST INFRASTRUCTURE ONLY (tests and the benchmark's CPU baseline); shares no code with the CUDA
kernels.  Arrays are NumPy; Adam runs in FP64 on FP32 inputs; the densification decisions are
taken in FP32 with the same comparisons the kernel makes, so they agree bit for bit.

Readings (the paper is silent; each is stated where the kernel implements it):
* Adam: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, p -= lr (m / (1 - b1^t)) /
  (sqrt(v / (1 - b2^t)) + eps), one learning rate per group: means, log-scales, quaternions,
  opacity logits, SH degree-0 coefficients, higher SH coefficients.
* Statistic: for every Gaussian seen by a view, the norm of dL/d(projected mean) in normalised
  device units (dL/du W/2, dL/dv H/2) is added to its accumulator and its view count grows by 1.
* Densification of Gaussian i, in this order:
    1. prune when its opacity is below min_opacity (logit < log(min_opacity / (1 - min_opacity)));
    2. with g = accum / count (FP32, 0 when count = 0), densify when g >= grad_threshold:
       clone (emit the Gaussian and a copy) when max log-scale <= log(percent_dense * extent),
       else split (emit two children, not the Gaussian);
    3. otherwise emit the Gaussian.
  A split child j (j = 0, 1) has mean mu + R(q) (s * z_j) with z_j ~ N(0, I) given as input
  (s = exp(log-scale), R the rotation of the normalised quaternion), log-scale log-scale - ln 1.6
  (in FP32), and
  the parent's other parameters.  Every emitted Gaussian whose max log-scale exceeds
  log(max_world_scale) is then dropped.  Outputs keep the input order (a clone's copy right after
  it, a split's two children in its place); the Adam moments of survivors are kept, those of
  copies and children start at 0, and every statistic restarts at 0.
"""
from __future__ import annotations

import numpy as np

GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh_dc", "sh_rest")
LN16 = np.float32(np.log(1.6))   # a split child's scale is its parent's / 1.6


def adam_step(p, g, m, v, lr, step, b1=0.9, b2=0.999, eps=1e-15):
    """One Adam update of an FP32 array (FP64 arithmetic).  Returns new (p, m, v) as float64."""
    p, g, m, v = (np.asarray(a, np.float64) for a in (p, g, m, v))
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def accumulate(accum, count, ids, du, dv, width, height):
    """Adds the view-space gradient norms of the Gaussians `ids` (dL/du, dL/dv in pixels)."""
    accum = np.asarray(accum, np.float64).copy()
    count = np.asarray(count, np.int64).copy()
    nrm = np.sqrt((np.asarray(du, np.float64) * (width / 2.0)) ** 2 + (np.asarray(dv, np.float64) * (height / 2.0)) ** 2)
    np.add.at(accum, ids, nrm)
    np.add.at(count, ids, 1)
    return accum, count


def _rot(q):
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def thresholds(grad_threshold, percent_dense, extent, min_opacity, max_world_scale):
    """FP32 thresholds the decisions compare against (as the kernel receives them)."""
    return (np.float32(grad_threshold), np.float32(np.log(percent_dense * extent)),
            np.float32(np.log(min_opacity / (1.0 - min_opacity))), np.float32(np.log(max_world_scale)))


def decide(log_scales, logits, accum, count, th):
    """Action per Gaussian: 0 prune, 1 keep, 2 clone, 3 split (FP32 decisions)."""
    tg, tdense, tlogit, _ = th
    ls = np.asarray(log_scales, np.float32)
    lg = np.asarray(logits, np.float32)
    acc = np.asarray(accum, np.float32)
    cnt = np.asarray(count)
    with np.errstate(divide="ignore", invalid="ignore"):
        g = np.where(cnt > 0, acc / cnt.astype(np.float32), np.float32(0))
    act = np.ones(len(lg), np.int64)
    big = ls.max(axis=1) > tdense
    dens = g >= tg
    act[dens & ~big] = 2
    act[dens & big] = 3
    act[lg < tlogit] = 0
    return act


def densify(params, moments, accum, count, normals, th):
    """params: dict of FP32 arrays (means, log_scales, quats, opacity_logits, sh); moments: dict
    name -> (m, v) arrays; normals: [N, 2, 3] standard normal samples.  Returns (new params,
    new moments) as float64 arrays, in output order."""
    act = decide(params["log_scales"], params["opacity_logits"], accum, count, th)
    tmax = th[3]
    out = {k: [] for k in params}
    mom = {k: ([], []) for k in moments}
    n = len(act)
    for i in range(n):
        base = {k: np.asarray(params[k][i], np.float64) for k in params}
        emitted = []
        if act[i] == 1:
            emitted.append((base, True))
        elif act[i] == 2:
            emitted.append((base, True))
            emitted.append((base, False))
        elif act[i] == 3:
            s = np.exp(base["log_scales"])
            R = _rot(base["quats"])
            # child log-scale: the parent's minus ln 1.6, both in FP32 (an output parameter)
            lsc = (np.asarray(params["log_scales"][i], np.float32) - LN16).astype(np.float64)
            for j in range(2):
                child = dict(base)
                child["means"] = base["means"] + R @ (s * normals[i, j])
                child["log_scales"] = lsc
                emitted.append((child, False))
        for e, old in emitted:
            if np.float32(np.max(e["log_scales"])) > tmax:
                continue
            for k in params:
                out[k].append(e[k])
            for k in moments:
                if old:
                    mom[k][0].append(np.asarray(moments[k][0][i], np.float64))
                    mom[k][1].append(np.asarray(moments[k][1][i], np.float64))
                else:
                    mom[k][0].append(np.zeros_like(np.asarray(moments[k][0][i], np.float64)))
                    mom[k][1].append(np.zeros_like(np.asarray(moments[k][1][i], np.float64)))
    res = {k: np.array(out[k]) for k in params}
    resm = {k: (np.array(mom[k][0]), np.array(mom[k][1])) for k in moments}
    return res, resm, act
