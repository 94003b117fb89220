"""Independent brute-force renderer and SSIM (NumPy/SciPy, FP64) that pin the C++ oracle.

TEST INFRASTRUCTURE ONLY.  Nothing here is shared with ``vg_oracle.cpp``: rotations come from
``scipy.spatial.transform.Rotation``, the projection Jacobian from a complex-step derivative of
the pinhole map, spherical harmonics from ``scipy.special.sph_harm_y`` (complex, with the
Condon-Shortley phase) and the 2D radius from ``numpy.linalg.eigvalsh``.  Each pixel loops over
ALL Gaussians with the tile predicate, sorts the candidates by depth (ties by index) and
composites front to back (paper Sec. 3: projected, assigned to tiles, sorted, alpha-blended).
It is meant for tiny scenes (N <= a few hundred, images up to ~64x64).
"""
from __future__ import annotations

import math

import numpy as np


def real_sh(degree: int, d: np.ndarray) -> np.ndarray:
    """Real SH basis [N, (degree+1)^2] at unit directions d [N,3], index l^2 + l + m.

    Real form of the complex harmonics Y_l^m (which carry the Condon-Shortley phase):
    m > 0: sqrt2 Re Y_l^m;  m < 0: sqrt2 Im Y_l^|m|;  m = 0: Y_l^0.
    """
    from scipy.special import sph_harm_y
    theta = np.arccos(np.clip(d[:, 2], -1.0, 1.0))
    phi = np.mod(np.arctan2(d[:, 1], d[:, 0]), 2 * np.pi)
    cols = []
    for l in range(degree + 1):
        for m in range(-l, l + 1):
            Y = sph_harm_y(l, abs(m), theta, phi)
            if m == 0:
                cols.append(Y.real)
            elif m > 0:
                cols.append(math.sqrt(2.0) * Y.real)
            else:
                cols.append(math.sqrt(2.0) * Y.imag)
    return np.stack(cols, axis=1)


def _pinhole(p, fx, fy, cx, cy):
    return np.stack([fx * p[..., 0] / p[..., 2] + cx, fy * p[..., 1] / p[..., 2] + cy], axis=-1)


def project(g, cam, dilation=0.3, guard=1.3):
    """Per-Gaussian 2D quantities in FP64 (dict of arrays)."""
    from scipy.spatial.transform import Rotation
    from scipy.special import expit
    means = np.asarray(g.means, np.float64)
    R = np.asarray(cam.R, np.float64)
    t = np.asarray(cam.t, np.float64)
    p = means @ R.T + t
    z = p[:, 2]
    q = np.asarray(g.quats, np.float64)
    qn = np.linalg.norm(q, axis=1)
    ok = (z > cam.near) & (qn > 0)
    # scipy wants scalar-last quaternions
    Rq = Rotation.from_quat(q[:, [1, 2, 3, 0]] / np.where(qn > 0, qn, 1.0)[:, None]).as_matrix()
    s2 = np.exp(2.0 * np.asarray(g.log_scales, np.float64))
    Sigma = np.einsum("nij,nj,nkj->nik", Rq, s2, Rq)
    # Jacobian of the pinhole map at the guard-band clamped point, by complex step
    limx = guard * 0.5 * cam.width / cam.fx
    limy = guard * 0.5 * cam.height / cam.fy
    zs = np.where(ok, z, 1.0)
    pc = np.stack([np.clip(p[:, 0] / zs, -limx, limx) * zs, np.clip(p[:, 1] / zs, -limy, limy) * zs, zs], 1)
    h = 1e-30
    J = np.zeros((means.shape[0], 2, 3))
    for k in range(3):
        pe = pc.astype(np.complex128)
        pe[:, k] += 1j * h
        J[:, :, k] = _pinhole(pe, cam.fx, cam.fy, cam.cx, cam.cy).imag / h
    T = J @ R
    cov2 = np.einsum("nij,njk,nlk->nil", T, Sigma, T) + dilation * np.eye(2)
    det = np.linalg.det(cov2)
    ok &= det > 0
    conic = np.linalg.inv(np.where(ok[:, None, None], cov2, np.eye(2)))
    lam = np.linalg.eigvalsh(np.where(ok[:, None, None], cov2, np.eye(2)))[:, 1]
    r = 3.0 * np.sqrt(lam)
    uv = _pinhole(np.where(ok[:, None], p, 1.0), cam.fx, cam.fy, cam.cx, cam.cy)
    dirs = means - np.asarray(cam.cam_pos, np.float64)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    Y = real_sh(g.sh_degree, dirs)
    rgb = np.maximum(0.0, np.einsum("nk,nkc->nc", Y, np.asarray(g.sh, np.float64)) + 0.5)
    return dict(ok=ok, uv=uv, depth=z, conic=conic, cov2=cov2, r=r, rgb=rgb,
                opacity=expit(np.asarray(g.opacity_logits, np.float64)))


def render(g, cam, tile=16, alpha_max=0.99, alpha_min=1.0 / 255.0, t_min=1e-4, bg=(0, 0, 0),
           dilation=0.3, guard=1.3):
    """Per-pixel brute force: returns (image [3,H,W], T [H,W], n_blended [H,W])."""
    pr = project(g, cam, dilation, guard)
    W, H = cam.width, cam.height
    u, v, r = pr["uv"][:, 0], pr["uv"][:, 1], pr["r"]
    xlo = np.maximum(0, np.ceil(u - r)); xhi = np.minimum(W - 1, np.floor(u + r))
    ylo = np.maximum(0, np.ceil(v - r)); yhi = np.minimum(H - 1, np.floor(v + r))
    vis = pr["ok"] & (xlo <= xhi) & (ylo <= yhi)
    tx0, tx1 = xlo // tile, xhi // tile
    ty0, ty1 = ylo // tile, yhi // tile
    img = np.zeros((3, H, W))
    Tout = np.ones((H, W))
    nbl = np.zeros((H, W), np.int64)
    idx = np.arange(len(u))
    for y in range(H):
        for x in range(W):
            tx, ty = x // tile, y // tile
            cand = idx[vis & (tx0 <= tx) & (tx <= tx1) & (ty0 <= ty) & (ty <= ty1)]
            cand = cand[np.lexsort((cand, pr["depth"][cand]))]
            T, C = 1.0, np.zeros(3)
            for i in cand:
                d = np.array([x - u[i], y - v[i]])
                power = -0.5 * d @ pr["conic"][i] @ d
                if power > 0:
                    continue
                alpha = min(alpha_max, pr["opacity"][i] * math.exp(power))
                if alpha < alpha_min:
                    continue
                Tn = T * (1 - alpha)
                if Tn < t_min:
                    break
                C += pr["rgb"][i] * alpha * T
                T = Tn
                nbl[y, x] += 1
            img[:, y, x] = C + T * np.asarray(bg, np.float64)
            Tout[y, x] = T
    return img, Tout, nbl


def ssim(x, y):
    """Mean SSIM with an 11-tap Gaussian window (sigma 1.5), zero padding, via scipy.ndimage."""
    from scipy.ndimage import correlate1d
    w = np.exp(-((np.arange(11) - 5.0) ** 2) / (2 * 1.5 ** 2))
    w /= w.sum()

    def blur(a):
        return correlate1d(correlate1d(a, w, axis=-1, mode="constant"), w, axis=-2, mode="constant")

    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mx, my = blur(x), blur(y)
    sxx = blur(x * x) - mx * mx
    syy = blur(y * y) - my * my
    sxy = blur(x * y) - mx * my
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    s = (2 * mx * my + C1) * (2 * sxy + C2) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    return float(s.mean())
