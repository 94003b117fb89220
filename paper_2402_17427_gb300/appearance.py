"""Decoupled appearance modelling on the GPU (paper Sec. 4.2, Eq. 2-3) through include/vgappearance.h.

Each training view i has an appearance embedding l_i (64 floats).  The CNN of the supplementary
material turns the 32x-downsampled rendering, with l_i appended to every pixel, into a
transformation map M_i, and the loss of a view is
    L = (1 - lambda) L1(I_r * M_i, I) + lambda D-SSIM(I_r, I)                             (Eq. 3)
The embeddings and the CNN are optimised with the Gaussians (learning rate 0.001 for both,
Sec. 5.1) and discarded after training.
"""
from __future__ import annotations

import math

import torch

from . import binding as B
from .rasterize import _stream

EMBED = 64
LAYERS = ((67, 256), (64, 128), (32, 64), (16, 32), (8, 16), (16, 16), (16, 3))   # (C, O) of each 3x3 conv
LEARNING_RATE = 1e-3


def param_count() -> int:
    return sum(o * c * 9 + o for c, o in LAYERS)


def layer_views(params: torch.Tensor):
    """(weight [O, C, 3, 3], bias [O]) views of a flat parameter (or gradient) tensor."""
    out, off = [], 0
    for c, o in LAYERS:
        w = params[off:off + o * c * 9].view(o, c, 3, 3)
        off += o * c * 9
        out.append((w, params[off:off + o]))
        off += o
    return out


def init_params(seed: int = 0, device="cuda") -> torch.Tensor:
    """Seeded initialisation: weights N(0, 1 / (9 C)) (fan-in scaling), biases N(0, 0.1^2)."""
    gen = torch.Generator().manual_seed(seed)
    parts = []
    for c, o in LAYERS:
        parts.append(torch.randn(o * c * 9, generator=gen, dtype=torch.float64) / math.sqrt(9 * c))
        parts.append(torch.randn(o, generator=gen, dtype=torch.float64) * 0.1)
    return torch.cat(parts).float().to(device)


class AppearanceModel:
    """The CNN's parameters and one embedding per training view, with the loss of Eq. 3."""

    def __init__(self, n_views: int, seed: int = 0, device="cuda"):
        assert B.vg_appearance_param_count() == param_count()
        self.params = init_params(seed, device)
        gen = torch.Generator().manual_seed(seed + 1)
        self.embeddings = torch.randn(n_views, EMBED, generator=gen).to(device)
        self._ws = None

    def _workspace(self, W: int, H: int, device):
        need = B.vg_appearance_workspace_bytes(W, H)
        if need == 0:
            raise ValueError(f"image size {W}x{H} outside 32..16384")
        if self._ws is None or self._ws.numel() < need or self._ws.device != device:
            self._ws = torch.empty(need, dtype=torch.uint8, device=device)
        return self._ws, need

    def loss(self, img: torch.Tensor, target: torch.Tensor, view: int, lam: float = 0.2, grad: bool = True,
             want_map: bool = False):
        """Eq. 3 for view `view`.  img, target: CUDA float32 [3, H, W].  Returns a dict with
        'loss' ([1]), optionally 'map' ([3, H, W]) and, when grad, 'grad_img', 'grad_embedding'
        ([64]) and 'grad_params' (flat, same layout as params)."""
        img, target = img.contiguous(), target.contiguous()
        H, W = int(img.shape[1]), int(img.shape[2])
        dev = img.device
        ws, need = self._workspace(W, H, dev)
        out = {"loss": torch.empty(1, dtype=torch.float32, device=dev)}
        if want_map:
            out["map"] = torch.empty(3, H, W, dtype=torch.float32, device=dev)
        if grad:
            out["grad_img"] = torch.empty(3, H, W, dtype=torch.float32, device=dev)
            out["grad_embedding"] = torch.empty(EMBED, dtype=torch.float32, device=dev)
            out["grad_params"] = torch.empty_like(self.params)
        emb = self.embeddings[view].contiguous()
        p = lambda k: out[k].data_ptr() if k in out else None
        B.vg_appearance_loss(img.data_ptr(), target.data_ptr(), W, H, emb.data_ptr(), self.params.data_ptr(),
                             float(lam), ws.data_ptr(), need, out["loss"].data_ptr(), p("map"), p("grad_img"),
                             p("grad_embedding"), p("grad_params"), _stream())
        return out
