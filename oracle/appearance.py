"""Oracle for decoupled appearance modelling (paper Sec. 4.2, Eq. 2-3; CNN of the supplementary
material), NumPy in FP64.

TEST INFRASTRUCTURE ONLY (tests and the benchmark's CPU baseline); shares no code with the CUDA
kernels.

The rendered image I_r [3, H, W] is downsampled 32 times, an appearance embedding l [64] is
concatenated to every pixel (67 channels), and a CNN produces a transformation map M [3, H, W];
the appearance-variant image is I_a = I_r * M (pixel-wise) and the loss is
    L = (1 - lambda) L1(I_a, I) + lambda D-SSIM(I_r, I)                                  (Eq. 3)
CNN: 3x3 conv 67 -> 256; four up-sampling blocks (pixel shuffle x2, 3x3 conv C/4 -> C/2, ReLU)
taking 256 channels to 16 at 16x the resolution; bilinear up-sampling to H x W; 3x3 conv, ReLU,
3x3 conv to 3 channels.

Readings (the paper is silent): the downsampling is the mean over non-overlapping 32 x 32
blocks (H // 32 by W // 32 of them; remaining rows and columns do not enter); convolutions have
biases and zero padding 1; the first convolution and the last have no activation; the hidden
width of the two final convolutions is 16; the pixel shuffle puts input channel 4c + 2i + j at
output channel c, offset (i, j); bilinear up-sampling maps output pixel y to input coordinate
(y + 1/2) h / H - 1/2, clamped below at 0, between rows floor and floor + 1 (the last row is
repeated); gradients flow to I_r through both terms and through the CNN input; L1 is the mean over
3 H W and D-SSIM is 1 - SSIM as in Eq. 1.
"""
from __future__ import annotations

import numpy as np

EMBED = 64
LAYERS = [(67, 256), (64, 128), (32, 64), (16, 32), (8, 16), (16, 16), (16, 3)]   # (in, out) channels


def init_weights(rng, scale=1.0):
    """Seeded weights [(w [O, C, 3, 3], b [O])] with a fan-in scaling."""
    out = []
    for c, o in LAYERS:
        std = scale / np.sqrt(9 * c)
        out.append((rng.normal(0, std, (o, c, 3, 3)), rng.normal(0, 0.1, o)))
    return out


# ---------------------------------------------------------------- operators and their adjoints

def pool32(x):
    C, H, W = x.shape
    h, w = H // 32, W // 32
    return x[:, :32 * h, :32 * w].reshape(C, h, 32, w, 32).mean(axis=(2, 4))


def pool32_adj(g, H, W):
    C, h, w = g.shape
    out = np.zeros((C, H, W))
    out[:, :32 * h, :32 * w] = np.repeat(np.repeat(g, 32, axis=1), 32, axis=2) / 1024.0
    return out


def conv(x, w, b):
    """3x3, zero padding 1: y[o, y, x] = b[o] + sum_{c, i, j} w[o, c, i, j] x[c, y + i - 1, x + j - 1].

    Evaluated on the padded image flattened with row pitch P = W + 2: output (y, x) and tap (i, j)
    read flat element (y + i) P + x + j, so each tap is one matrix product over a contiguous
    window; the two extra columns of every output row are computed and dropped."""
    C, H, W = x.shape
    P = W + 2
    xp = np.pad(x, ((0, 0), (1, 2), (1, 1))).reshape(C, (H + 3) * P)
    y = np.empty((w.shape[0], H * P))
    y[:] = b[:, None]
    for i in range(3):
        for j in range(3):
            o = i * P + j
            y += w[:, :, i, j] @ xp[:, o:o + H * P]
    return np.ascontiguousarray(y.reshape(-1, H, P)[:, :, :W])


def conv_adj(x, w, g):
    """Adjoints of conv: (dL/dx, dL/dw, dL/db) from g = dL/dy (same flat windows as conv, with g
    zero in the dropped columns)."""
    C, H, W = x.shape
    P = W + 2
    O = g.shape[0]
    xp = np.pad(x, ((0, 0), (1, 2), (1, 1))).reshape(C, (H + 3) * P)
    ge = np.zeros((O, H, P))
    ge[:, :, :W] = g
    ge = ge.reshape(O, H * P)
    gxp = np.zeros((C, (H + 3) * P))
    dw = np.empty_like(w)
    for i in range(3):
        for j in range(3):
            o = i * P + j
            dw[:, :, i, j] = ge @ xp[:, o:o + H * P].T
            gxp[:, o:o + H * P] += w[:, :, i, j].T @ ge
    gx = gxp.reshape(C, H + 3, P)[:, 1:H + 1, 1:W + 1]
    return np.ascontiguousarray(gx), dw, g.sum(axis=(1, 2))


def shuffle(x):
    C4, h, w = x.shape
    C = C4 // 4
    return x.reshape(C, 2, 2, h, w).transpose(0, 3, 1, 4, 2).reshape(C, 2 * h, 2 * w)


def unshuffle(y):
    C, H, W = y.shape
    return y.reshape(C, H // 2, 2, W // 2, 2).transpose(0, 2, 4, 1, 3).reshape(4 * C, H // 2, W // 2)


def _bilinear_taps(n_in, n_out):
    s = (np.arange(n_out) + 0.5) * (n_in / n_out) - 0.5
    s = np.maximum(s, 0.0)
    i0 = np.minimum(np.floor(s).astype(np.int64), n_in - 1)
    i1 = np.minimum(i0 + 1, n_in - 1)
    return i0, i1, s - i0


def bilinear(x, H, W):
    C, h, w = x.shape
    y0, y1, fy = _bilinear_taps(h, H)
    x0, x1, fx = _bilinear_taps(w, W)
    top = x[:, y0][:, :, x0] * (1 - fx) + x[:, y0][:, :, x1] * fx
    bot = x[:, y1][:, :, x0] * (1 - fx) + x[:, y1][:, :, x1] * fx
    return top * (1 - fy)[:, None] + bot * fy[:, None]


def bilinear_adj(g, h, w):
    C, H, W = g.shape
    y0, y1, fy = _bilinear_taps(h, H)
    x0, x1, fx = _bilinear_taps(w, W)
    out = np.zeros((C, h, w))
    for yy, wy in ((y0, 1 - fy), (y1, fy)):
        for xx, wx in ((x0, 1 - fx), (x1, fx)):
            np.add.at(out, (slice(None), yy[:, None], xx[None, :]), g * wy[:, None] * wx[None, :])
    return out


# ---------------------------------------------------------------- the model

def forward(img, emb, weights):
    """Activations of the appearance CNN; returns (M, cache)."""
    _, H, W = img.shape
    p = pool32(img)
    D = np.concatenate([p, np.broadcast_to(emb[:, None, None], (EMBED,) + p.shape[1:])], axis=0)
    acts = [D]
    a = conv(D, *weights[0])                       # no activation
    acts.append(a)
    for k in range(1, 5):
        a = np.maximum(conv(shuffle(a), *weights[k]), 0.0)
        acts.append(a)
    U = bilinear(a, H, W)
    Hh = np.maximum(conv(U, *weights[5]), 0.0)
    M = conv(Hh, *weights[6])
    return M, dict(acts=acts, U=U, Hh=Hh)


def loss_and_grads(img, target, emb, weights, lam):
    """Eq. 3 and its gradients with respect to the rendering, the embedding and the weights."""
    import oracle
    img = np.asarray(img, np.float64)
    target = np.asarray(target, np.float64)
    _, H, W = img.shape
    M, c = forward(img, emb, weights)
    Ia = img * M
    n = img.size
    l1 = np.abs(Ia - target).mean()
    dssim, g_ssim = oracle.loss_l1_dssim(img, target, 1.0)        # lambda = 1: 1 - SSIM and its gradient
    L = (1 - lam) * l1 + lam * dssim
    gIa = (1 - lam) * np.sign(Ia - target) / n
    gM = gIa * img
    g_img = gIa * M + lam * g_ssim
    grads = [None] * 7
    gHh, grads[6], gb6 = conv_adj(c["Hh"], weights[6][0], gM)
    grads[6] = (grads[6], gb6)
    gHh = gHh * (c["Hh"] > 0)
    gU, dw5, db5 = conv_adj(c["U"], weights[5][0], gHh)
    grads[5] = (dw5, db5)
    acts = c["acts"]
    g = bilinear_adj(gU, *acts[5].shape[1:]) * (acts[5] > 0)
    for k in range(4, 0, -1):            # block k maps acts[k] to acts[k + 1]
        gs, dw, db = conv_adj(shuffle(acts[k]), weights[k][0], g)
        grads[k] = (dw, db)
        g = unshuffle(gs)
        if k > 1:                        # acts[1] is the first convolution's output, no ReLU
            g = g * (acts[k] > 0)
    gD, dw0, db0 = conv_adj(acts[0], weights[0][0], g)
    grads[0] = (dw0, db0)
    g_img = g_img + pool32_adj(gD[:3], H, W)
    g_emb = gD[3:].sum(axis=(1, 2))
    return L, M, g_img, g_emb, grads
