"""GB300-native (sm_103a) differentiable tile rasteriser for 3D Gaussian splatting.

The rasteriser R of VastGaussian (arXiv 2402.17427, Sec. 3) — EWA projection, SH colour, 16x16
tile binning, depth sort, front-to-back alpha compositing and its adjoint — as hand-written
CUDA kernels behind a C ABI (``include/vgrast.h``, ``libvgrast.so``).  Python modules:

* ``binding``   — ctypes binding of the C ABI (same names);
* ``rasterize`` — torch front end: workspaces, streams, ``torch.autograd.Function``;
* ``batch``     — many cells in one launch per stage, with the per-cell autotuner;
* ``serving``   — continuous-batching novel-view server over the merged scene;
* ``scenes``    — seeded synthetic scenes and cameras.

Submodules are imported lazily so that ``scenes`` works without torch or a GPU.
"""
__all__ = ["binding", "rasterize", "scenes", "build"]


def build(force: bool = False) -> str:
    from ._build import build as _b
    return _b(force=force)
