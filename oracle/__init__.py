"""CPU oracle (FP64) for the differentiable Gaussian rasteriser and its loss.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()`` and by the
benchmark's CPU-baseline leg, never by the product package.  ``vg_oracle.cpp`` holds the
renderer, tile lists, adjoint and L1 + D-SSIM loss (paper Sec. 3, Eq. 1); ``brute.py`` is an
independent NumPy brute-force renderer that pins it.

Every function here takes plain NumPy arrays (float32 scene parameters are widened to float64
exactly) and a camera described by plain numbers, so nothing from the CUDA path is involved.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "vg_oracle.cpp")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (OpenMP when available).  Returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("Rt", ctypes.c_double * 12), ("cam_pos", ctypes.c_double * 3),
                ("near_plane", ctypes.c_double)]


class _Opts(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("stop_rule", ctypes.c_int32),
                ("bg", ctypes.c_double * 3),
                ("dilation", ctypes.c_double), ("alpha_max", ctypes.c_double),
                ("alpha_min", ctypes.c_double), ("t_min", ctypes.c_double), ("guard", ctypes.c_double),
                ("band_alpha", ctypes.c_double), ("band_t", ctypes.c_double),
                ("band_power", ctypes.c_double), ("band_rect", ctypes.c_double),
                ("n_threads", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("tile_mask", ctypes.c_void_p)]


class _Scene(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("logits", ctypes.c_void_p), ("sh", ctypes.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.c_void_p
            L.or_forward.restype = P
            L.or_forward.argtypes = [ctypes.POINTER(_Scene), ctypes.POINTER(_Camera), ctypes.POINTER(_Opts)]
            L.or_free.argtypes = [P]
            L.or_num_pairs.restype = ctypes.c_int64
            L.or_num_pairs.argtypes = [P]
            L.or_stats.argtypes = [P, P]
            L.or_decision_hash.restype = ctypes.c_uint64
            L.or_decision_hash.argtypes = [P]
            L.or_get_image.argtypes = [P, P, P, P, P]
            L.or_get_pairs.argtypes = [P, P, P, P]
            L.or_get_records.argtypes = [P, P, P, P, P]
            L.or_pixel_trace.restype = ctypes.c_int32
            L.or_pixel_trace.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int32]
            L.or_backward.argtypes = [P, P, P, P, P, P, P, P, P]
            L.or_sh_basis.argtypes = [ctypes.c_int, P, P, P]
            L.or_fd_directional.argtypes = [P, P, ctypes.c_int64, P, P, ctypes.c_double, P, P]
            L.or_fd_directional.restype = None
            L.or_pairs_from_fp32.restype = ctypes.c_int64
            L.or_pairs_from_fp32.argtypes = [ctypes.c_int64, P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int64, P, P, P]
            L.or_ssim_map.restype = ctypes.c_double
            L.or_ssim_map.argtypes = [P, P, ctypes.c_int, ctypes.c_int, P]
            L.or_loss_l1_dssim.restype = ctypes.c_double
            L.or_loss_l1_dssim.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_double, P]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Options:
    """Rasteriser settings (the method's constants) and the oracle's ambiguity bands."""
    tile: int = 16
    stop_rule: int = 0
    bg: tuple = (0.0, 0.0, 0.0)
    dilation: float = 0.3
    alpha_max: float = 0.99
    alpha_min: float = 1.0 / 255.0
    t_min: float = 1e-4
    guard: float = 1.3
    # Relative decision bands: wide enough for the FP32 error with which another implementation
    # (the CUDA kernels) takes the same decisions.  Measured on GB300 against this oracle: final
    # transmittance within 7.5e-6 relative (so t_min decisions within that), no pixel off by more
    # than 1e-4 outside bands a quarter of these and the first flips at a sixteenth; the radius r
    # within 1.2e-5 relative.
    band_alpha: float = 5e-6
    band_t: float = 2.5e-5
    band_power: float = 2.5e-6
    band_rect: float = 2.5e-5
    n_threads: int = 0

    def c(self, tile_mask=None):
        o = _Opts()
        o.tile, o.stop_rule = self.tile, self.stop_rule
        o.bg[:] = [float(x) for x in self.bg]
        o.dilation, o.alpha_max, o.alpha_min = self.dilation, self.alpha_max, self.alpha_min
        o.t_min, o.guard = self.t_min, self.guard
        o.band_alpha, o.band_t, o.band_power, o.band_rect = (self.band_alpha, self.band_t,
                                                             self.band_power, self.band_rect)
        o.n_threads = self.n_threads
        o.tile_mask = tile_mask.ctypes.data if tile_mask is not None else None
        return o


def _camera(cam) -> _Camera:
    c = _Camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    Rt = np.concatenate([np.asarray(cam.R, np.float64), np.asarray(cam.t, np.float64)[:, None]], 1)
    c.Rt[:] = [float(x) for x in Rt.ravel()]
    c.cam_pos[:] = [float(x) for x in np.asarray(cam.cam_pos, np.float64)]
    c.near_plane = float(cam.near)
    return c


class Scene64:
    """FP64 copy of a Gaussian set (keeps the arrays alive for the C side)."""

    def __init__(self, means, log_scales, quats, logits, sh, sh_degree):
        f = lambda a: np.ascontiguousarray(np.asarray(a, np.float64))
        self.means, self.log_scales, self.quats = f(means), f(log_scales), f(quats)
        self.logits, self.sh = f(logits).reshape(-1), f(sh)
        self.sh_degree = int(sh_degree)
        self.n = self.means.shape[0]
        self.K = (self.sh_degree + 1) ** 2
        self.sh = self.sh.reshape(self.n, self.K, 3)

    @classmethod
    def of(cls, g):
        return cls(g.means, g.log_scales, g.quats, g.opacity_logits, g.sh, g.sh_degree)

    def c(self) -> _Scene:
        s = _Scene()
        s.n, s.sh_degree = self.n, self.sh_degree
        s.means, s.log_scales, s.quats = self.means.ctypes.data, self.log_scales.ctypes.data, self.quats.ctypes.data
        s.logits, s.sh = self.logits.ctypes.data, self.sh.ctypes.data
        return s

    def params(self):
        return [self.means, self.log_scales, self.quats, self.logits, self.sh]


class Render:
    """Result of one oracle forward pass (owns the C handle)."""

    def __init__(self, scene: Scene64, cam, opts: Options, tile_mask=None):
        L = lib()
        self._L = L
        self.scene, self.cam, self.opts = scene, cam, opts
        self._sc, self._cm = scene.c(), _camera(cam)
        mask = None if tile_mask is None else np.ascontiguousarray(tile_mask, np.uint8)
        self._op = opts.c(mask)
        self.h = L.or_forward(ctypes.byref(self._sc), ctypes.byref(self._cm), ctypes.byref(self._op))
        H, W = cam.height, cam.width
        self.tiles_x = (W + opts.tile - 1) // opts.tile
        self.tiles_y = (H + opts.tile - 1) // opts.tile
        self.image = np.zeros((3, H, W))
        self.T = np.zeros((H, W))
        self.last = np.zeros((H, W), np.int32)
        self.amb = np.zeros((H, W), np.uint8)
        L.or_get_image(self.h, _ptr(self.image), _ptr(self.T), _ptr(self.last), _ptr(self.amb))
        P = L.or_num_pairs(self.h)
        self.keys = np.zeros(P, np.uint64)
        self.vals = np.zeros(P, np.uint32)
        self.ranges = np.zeros((self.tiles_x * self.tiles_y, 2), np.int32)
        L.or_get_pairs(self.h, _ptr(self.keys), _ptr(self.vals), _ptr(self.ranges))
        n = scene.n
        f64 = np.zeros((n, 13))
        f32 = np.zeros((n, 4), np.float32)
        i32 = np.zeros((n, 9), np.int32)
        arect = np.zeros((n, 4), np.int32)
        L.or_get_records(self.h, _ptr(f64), _ptr(f32), _ptr(i32), _ptr(arect))
        self.rec = dict(u=f64[:, 0], v=f64[:, 1], conic=f64[:, 2:5], opacity=f64[:, 5], radius=f64[:, 6],
                        rgb=f64[:, 7:10], depth=f64[:, 10], cov2=f64[:, 11:13],
                        depth32=f32[:, 0], u32=f32[:, 1], v32=f32[:, 2], r32=f32[:, 3],
                        valid=i32[:, 0].astype(bool), visible=i32[:, 1].astype(bool),
                        rect=i32[:, 2:6], rect_amb=i32[:, 6].astype(bool), grad_amb=i32[:, 7].astype(bool),
                        union_rect=arect)
        st = np.zeros(4, np.int64)
        L.or_stats(self.h, _ptr(st))
        self.n_eval, self.n_blend, self.n_visible, self.n_amb = (int(x) for x in st)
        self.decision_hash = int(L.or_decision_hash(self.h))

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self._L.or_free(h)
            self.h = None

    @property
    def num_pairs(self) -> int:
        return int(self.keys.size)

    def tile_list(self, t):
        s, e = self.ranges[t]
        return self.vals[s:e]

    def pixel_trace(self, x, y, cap=4096):
        T = np.zeros(cap)
        g = np.zeros(cap, np.uint32)
        n = self._L.or_pixel_trace(self.h, int(x), int(y), _ptr(T), _ptr(g), cap)
        return T[:min(n, cap)], g[:min(n, cap)]

    def fd_directional(self, w, ids, dirs, eps: float = 1e-6):
        """Central differences of L = sum(w * image) along dirs[k] (raw parameters of Gaussian
        ids[k] in the layout mean 3, log-scale 3, quaternion 4, logit 1, SH 3K), re-rendering only
        that Gaussian's tiles.  Returns (derivatives [m], flags [m]); flag 1 marks a perturbation
        that changed a decision (not a derivative)."""
        w = np.ascontiguousarray(np.asarray(w, np.float64))
        ids = np.ascontiguousarray(np.asarray(ids, np.int64))
        dirs = np.ascontiguousarray(np.asarray(dirs, np.float64).reshape(len(ids), -1))
        assert dirs.shape[1] == 11 + 3 * self.scene.K
        out = np.zeros(len(ids))
        flags = np.zeros(len(ids), np.int32)
        self._L.or_fd_directional(self.h, _ptr(w), len(ids), _ptr(ids), _ptr(dirs), float(eps), _ptr(out),
                                  _ptr(flags))
        return out, flags

    def backward(self, dL_dimg):
        """Gradients w.r.t. raw parameters, plus the per-Gaussian 2D gradients [n, 9] and the
        densification statistic g2d_abs [n] (sum over pixels of |dL/du| + |dL/dv| per pixel)."""
        s = self.scene
        dimg = np.ascontiguousarray(np.asarray(dL_dimg, np.float64))
        out = dict(means=np.zeros((s.n, 3)), log_scales=np.zeros((s.n, 3)), quats=np.zeros((s.n, 4)),
                   logits=np.zeros(s.n), sh=np.zeros((s.n, s.K, 3)), g2d=np.zeros((s.n, 9)), g2d_abs=np.zeros(s.n))
        self._L.or_backward(self.h, _ptr(dimg), _ptr(out["means"]), _ptr(out["log_scales"]),
                            _ptr(out["quats"]), _ptr(out["logits"]), _ptr(out["sh"]), _ptr(out["g2d"]),
                            _ptr(out["g2d_abs"]))
        return out


def render(gaussians_or_scene, cam, opts: Options | None = None, tile_mask=None) -> Render:
    sc = gaussians_or_scene if isinstance(gaussians_or_scene, Scene64) else Scene64.of(gaussians_or_scene)
    return Render(sc, cam, opts or Options(), tile_mask)


def pairs_from_fp32(uvrd, width: int, height: int, tile: int = 16):
    """Keys, Gaussian ids and tile ranges of the stable (tile, depth) sort built from given FP32
    decision inputs uvrd [n, 4] = (u, v, r, depth) per Gaussian (r < 0: culled), with the forward
    pass's own rectangle rule, key layout and sort.  Returns (keys uint64 [P], ids uint32 [P],
    ranges int32 [tiles, 2])."""
    a = np.ascontiguousarray(np.asarray(uvrd, np.float32).reshape(-1, 4))
    n = a.shape[0]
    tiles = ((width + tile - 1) // tile) * ((height + tile - 1) // tile)
    L = lib()
    dummy = np.zeros(1, np.uint64)
    P = int(L.or_pairs_from_fp32(n, _ptr(a), width, height, tile, 0, _ptr(dummy), _ptr(dummy), _ptr(dummy)))
    keys = np.zeros(max(P, 1), np.uint64)
    vals = np.zeros(max(P, 1), np.uint32)
    ranges = np.zeros((tiles, 2), np.int32)
    got = int(L.or_pairs_from_fp32(n, _ptr(a), width, height, tile, P, _ptr(keys), _ptr(vals), _ptr(ranges)))
    assert got == P
    return keys[:P], vals[:P], ranges


def sh_basis(degree: int, d):
    d = np.ascontiguousarray(np.asarray(d, np.float64))
    Y = np.zeros(16)
    dY = np.zeros((16, 3))
    lib().or_sh_basis(degree, _ptr(d), _ptr(Y), _ptr(dY))
    k = (degree + 1) ** 2
    return Y[:k], dY[:k]


def ssim(x, y) -> float:
    x = np.ascontiguousarray(np.asarray(x, np.float64))
    y = np.ascontiguousarray(np.asarray(y, np.float64))
    return float(lib().or_ssim_map(_ptr(x), _ptr(y), x.shape[1], x.shape[2], None))


def ssim_map(x, y):
    x = np.ascontiguousarray(np.asarray(x, np.float64))
    y = np.ascontiguousarray(np.asarray(y, np.float64))
    m = np.zeros_like(x)
    lib().or_ssim_map(_ptr(x), _ptr(y), x.shape[1], x.shape[2], _ptr(m))
    return m


def loss_l1_dssim(x, y, lam: float = 0.2, grad: bool = True):
    """Eq. 1 loss and (optionally) its gradient with respect to the rendered image x."""
    x = np.ascontiguousarray(np.asarray(x, np.float64))
    y = np.ascontiguousarray(np.asarray(y, np.float64))
    g = np.zeros_like(x) if grad else None
    L = lib().or_loss_l1_dssim(_ptr(x), _ptr(y), x.shape[1], x.shape[2], float(lam),
                               _ptr(g) if grad else None)
    return (float(L), g) if grad else float(L)
