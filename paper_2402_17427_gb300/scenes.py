"""Seeded synthetic scenes and cameras: the inputs both the CUDA path and the CPU oracle consume.

This module only draws random numbers and builds cameras; it holds none of the rasteriser's
arithmetic (no projection, no covariance, no spherical harmonics, no compositing).  Every array
is float32, the precision the rasteriser's parameters are stored in.

The paper trains on aerial drone captures (Mill-19, UrbanScene3D; Sec. 5.1) that are not
available here, so these generators stand in for their shapes: a blob-mixture volume (1080p
single-cell step), an aerial ground-plus-buildings city split into cells (batched training),
a dense urban volume with facades (memory-scale cell) and a 16-cell merged city (serving).

Conventions (world +y is up, as after the paper's Manhattan-world alignment, Sec. 5.1;
cameras are OpenCV-style: +x right, +y down, +z forward; ``R`` maps world to camera).
Parameters per Gaussian: mean [3], log-scale [3], quaternion [4] in (w, x, y, z) order,
opacity logit [1] and spherical-harmonic coefficients [K, 3] with K = (degree + 1)^2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Value of the degree-0 real spherical harmonic, 1 / (2 sqrt(pi)).  Only used to turn a
# drawn base colour c into the DC coefficient (c - 0.5) / Y00 of the input recipe.
_DC_BASIS = 0.5 / math.sqrt(math.pi)


def sh_coeffs(degree: int) -> int:
    return (degree + 1) ** 2


@dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray          # [3,3] float32, world -> camera rotation
    t: np.ndarray          # [3] float32, camera = R @ world + t
    cam_pos: np.ndarray    # [3] float32, camera centre in world coordinates
    near: float = 0.2

    @property
    def world_to_cam(self) -> np.ndarray:
        """Row-major 3x4 [R | t] as float32."""
        return np.concatenate([self.R, self.t[:, None]], axis=1).astype(np.float32)

    @property
    def num_pixels(self) -> int:
        return self.width * self.height


@dataclass
class Gaussians:
    means: np.ndarray          # [N,3]
    log_scales: np.ndarray     # [N,3]
    quats: np.ndarray          # [N,4] (w,x,y,z)
    opacity_logits: np.ndarray  # [N]
    sh: np.ndarray             # [N,K,3]
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def arrays(self):
        return (self.means, self.log_scales, self.quats, self.opacity_logits, self.sh)

    def subset(self, idx) -> "Gaussians":
        return Gaussians(self.means[idx], self.log_scales[idx], self.quats[idx],
                         self.opacity_logits[idx], self.sh[idx], self.sh_degree)

    @staticmethod
    def concat(parts) -> "Gaussians":
        deg = parts[0].sh_degree
        return Gaussians(*(np.ascontiguousarray(np.concatenate(a, axis=0)) for a in
                           zip(*(p.arrays() for p in parts))), deg)


@dataclass
class Cell:
    gaussians: Gaussians
    aabb: np.ndarray            # [6] float32: xmin, ymin, zmin, xmax, ymax, zmax
    camera: Camera | None = None
    target: np.ndarray | None = None


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def camera_from_forward(eye, forward, width, height, hfov_deg=60.0, up_hint=(0.0, 1.0, 0.0),
                        fx=None, near=0.2) -> Camera:
    """Pinhole camera at ``eye`` looking along ``forward``; principal point at the image centre."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(forward, np.float64)
    f = f / np.linalg.norm(f)
    up = np.asarray(up_hint, np.float64)
    if abs(float(np.dot(f, up))) > 0.999:     # looking straight along the hint: use +z instead
        up = np.array([0.0, 0.0, 1.0])
    x = np.cross(f, up)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f])
    t = -R @ eye
    if fx is None:
        fx = width / (2.0 * math.tan(math.radians(hfov_deg) / 2.0))
    return Camera(width, height, float(np.float32(fx)), float(np.float32(fx)),
                  float(np.float32(width / 2.0)), float(np.float32(height / 2.0)),
                  _f32(R), _f32(t), _f32(eye), near)


def look_at(eye, target, width, height, **kw) -> Camera:
    return camera_from_forward(eye, np.asarray(target, np.float64) - np.asarray(eye, np.float64),
                               width, height, **kw)


def yaw_pitch_forward(yaw, pitch):
    """Unit view direction from yaw (about +y, 0 = +z) and pitch (negative = looking down)."""
    cp = math.cos(pitch)
    return np.array([cp * math.sin(yaw), math.sin(pitch), cp * math.cos(yaw)])


def _random_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _colour_sh(rng, n, degree, higher_std):
    k = sh_coeffs(degree)
    sh = np.empty((n, k, 3), np.float32)
    c = rng.random((n, 3))
    sh[:, 0, :] = (c - 0.5) / _DC_BASIS
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, higher_std, (n, k - 1, 3))
    return sh


def _gaussians(rng, means, log_scale_mu, log_scale_sigma, degree, higher_std=0.2) -> Gaussians:
    n = means.shape[0]
    return Gaussians(
        means=_f32(means),
        log_scales=_f32(rng.normal(log_scale_mu, log_scale_sigma, (n, 3))),
        quats=_f32(_random_quats(rng, n)),
        opacity_logits=_f32(rng.standard_normal(n)),
        sh=_colour_sh(rng, n, degree, higher_std),
        sh_degree=degree,
    )


def random_target(rng, camera: Camera) -> np.ndarray:
    return _f32(rng.random((3, camera.height, camera.width)))


# ---------------------------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------------------------

def small_cell(seed: int = 0):
    """10 000 Gaussians in a 4x4x4 box seen from 6 units away by a 128x128 camera, SH degree 0.

    means ~ U([-2,2]^3), log-scales ~ N(-3, 0.5), random unit quaternions, opacity logits
    ~ N(0,1), base colours c ~ U(0,1) stored as DC coefficients; fx = fy = 128.
    Returns (gaussians, camera, target).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n = 10_000
    means = rng.uniform(-2.0, 2.0, (n, 3))
    g = _gaussians(rng, means, -3.0, 0.5, 0)
    cam = look_at((0.0, 0.0, -6.0), (0.0, 0.0, 0.0), 128, 128, fx=128.0)
    return g, cam, random_target(rng, cam)


def blob_cell_1080p(seed: int = 1000, n: int = 1_000_000, width=1920, height=1080):
    """One cell of 1M Gaussians, SH degree 3, drawn from 64 Gaussian blobs in 100x20x100 m.

    Blob centres ~ U([0,100]x[0,20]x[0,100]) (x, y-up, z), blob std ~ U(2,8) m, means clipped to
    the box; log-scales ~ N(ln 0.08, 0.5); DC colour ~ U(0,1), higher bands ~ N(0, 0.2).
    Camera: 1920x1080, 60 deg horizontal FOV, on a 30 m-radius orbit around (50, ., 50) at 30 m
    altitude, random yaw, pitched down 45 deg.  Returns (gaussians, camera, target).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = np.array([0.0, 0.0, 0.0]), np.array([100.0, 20.0, 100.0])
    centres = rng.uniform(lo, hi, (64, 3))
    stds = rng.uniform(2.0, 8.0, 64)
    which = rng.integers(0, 64, n)
    means = np.clip(centres[which] + rng.standard_normal((n, 3)) * stds[which, None], lo, hi)
    g = _gaussians(rng, means, math.log(0.08), 0.5, 3)
    yaw = rng.uniform(0.0, 2.0 * math.pi)
    eye = (50.0 + 30.0 * math.sin(yaw), 30.0, 50.0 + 30.0 * math.cos(yaw))
    cam = camera_from_forward(eye, yaw_pitch_forward(yaw + math.pi, -math.pi / 4), width, height)
    return g, cam, random_target(rng, cam)


def _heightfield(x, z):
    """Gently rolling ground (metres) used by the aerial city generators."""
    return 2.0 * np.sin(x / 57.0) * np.cos(z / 83.0) + 1.0 * np.sin((x + z) / 31.0)


def _city_points(rng, n, x0, x1, z0, z1, n_boxes, facade_frac=0.7, hmin=10.0, hmax=60.0,
                 foot=(10.0, 40.0), jitter=0.1):
    """Points on axis-aligned building boxes (walls + roof) and on the ground heightfield."""
    bx = rng.uniform(x0, x1, n_boxes)
    bz = rng.uniform(z0, z1, n_boxes)
    bw = rng.uniform(foot[0], foot[1], n_boxes)
    bd = rng.uniform(foot[0], foot[1], n_boxes)
    bh = rng.uniform(hmin, hmax, n_boxes)
    base = _heightfield(bx, bz)
    # areas of the 4 walls and the roof, per box
    areas = np.stack([bw * bh, bw * bh, bd * bh, bd * bh, bw * bd], axis=1)
    n_fac = int(round(n * facade_frac))
    flat = areas.ravel() / areas.sum()
    pick = rng.choice(flat.size, n_fac, p=flat)
    b, face = pick // 5, pick % 5
    s, t = rng.random(n_fac), rng.random(n_fac)
    px = bx[b] + (s - 0.5) * bw[b]
    pz = bz[b] + (s - 0.5) * bd[b]
    py = base[b] + t * bh[b]
    nrm = np.zeros((n_fac, 3))
    # walls facing -z / +z (span x), walls facing -x / +x (span z), roof (+y)
    m0, m1, m2, m3, m4 = (face == i for i in range(5))
    pz[m0] = bz[b[m0]] - 0.5 * bd[b[m0]]; nrm[m0, 2] = -1
    pz[m1] = bz[b[m1]] + 0.5 * bd[b[m1]]; nrm[m1, 2] = 1
    px[m2] = bx[b[m2]] - 0.5 * bw[b[m2]]; nrm[m2, 0] = -1
    px[m3] = bx[b[m3]] + 0.5 * bw[b[m3]]; nrm[m3, 0] = 1
    px[m4] = bx[b[m4]] + (s[m4] - 0.5) * bw[b[m4]]
    pz[m4] = bz[b[m4]] + (t[m4] - 0.5) * bd[b[m4]]
    py[m4] = base[b[m4]] + bh[b[m4]]; nrm[m4, 1] = 1
    fac = np.stack([px, py, pz], 1) + nrm * rng.normal(0.0, jitter, (n_fac, 1))
    n_gnd = n - n_fac
    gx = rng.uniform(x0, x1, n_gnd)
    gz = rng.uniform(z0, z1, n_gnd)
    gnd = np.stack([gx, _heightfield(gx, gz) + rng.normal(0.0, jitter, n_gnd), gz], 1)
    pts = np.concatenate([fac, gnd], 0)
    return pts[rng.permutation(n)]


def _aabb(means) -> np.ndarray:
    return _f32(np.concatenate([means.min(0), means.max(0)]))


CELL_SIZES_8 = (300_000, 500_000, 800_000, 1_200_000, 1_500_000, 2_000_000, 2_500_000, 3_000_000)


def aerial_cells(step: int = 0, seed: int = 2000, sizes=CELL_SIZES_8, width=1152, height=864):
    """Eight cells of uneven size tiling a 1x1 km aerial scene as a 4x2 grid (250x500 m cells).

    Each cell: Gaussians on the ground heightfield plus random building boxes, log-scales ~
    N(ln(0.5 sqrt(area / n)), 0.5), SH degree 3.  One nadir camera per cell at 100 m altitude,
    1152x864, 60 deg FOV, placed on a lawnmower path (tracks 60 m apart) indexed by ``step``.
    Returns a list of Cell with camera and target filled in.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    cells = []
    for k, n in enumerate(sizes):
        ix, iz = k % 4, k // 4
        x0, z0 = 250.0 * ix, 500.0 * iz
        pts = _city_points(rng, n, x0, x0 + 250.0, z0, z0 + 500.0, n_boxes=20)
        area = 250.0 * 500.0
        g = _gaussians(rng, pts, math.log(0.5 * math.sqrt(area / n)), 0.5, 3)
        tracks = [x0 + 35.0 + 60.0 * j for j in range(4)]
        along = [z0 + 25.0 + 50.0 * j for j in range(10)]
        pos = step % (len(tracks) * len(along))
        tj, aj = pos // len(along), pos % len(along)
        if tj % 2:                       # lawnmower: alternate direction on every track
            aj = len(along) - 1 - aj
        ex, ez = tracks[tj], along[aj]
        eye = (ex, float(_heightfield(ex, ez)) + 100.0, ez)
        cam = camera_from_forward(eye, (0.0, -1.0, 0.0), width, height, up_hint=(0.0, 0.0, 1.0))
        cells.append(Cell(g, _aabb(g.means), cam, random_target(rng, cam)))
    return cells


def urban_cell_20m(seed: int = 3000, n: int = 20_000_000, width=1920, height=1080):
    """20M Gaussians in a 500x500x60 m urban volume: 70 % on ~150 building facades, 30 % ground.

    Log-scales ~ N(ln 0.05, 0.5), SH degree 3; one 1920x1080 camera at 80 m altitude pitched
    down 45 deg, random position over the central 300x300 m and random yaw.
    Returns (gaussians, camera, target).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = _city_points(rng, n, 0.0, 500.0, 0.0, 500.0, n_boxes=150)
    g = _gaussians(rng, pts, math.log(0.05), 0.5, 3)
    ex, ez = rng.uniform(100.0, 400.0, 2)
    yaw = rng.uniform(0.0, 2.0 * math.pi)
    cam = camera_from_forward((ex, 80.0, ez), yaw_pitch_forward(yaw, -math.pi / 4), width, height)
    return g, cam, random_target(rng, cam)


def merged_city(seed: int = 4000, total_scale: float = 1.0):
    """16 cells on a 4x4 grid over 1x1 km (250x250 m cells) for serving the merged scene.

    Cell k holds 0.5M * (1 + k/5) Gaussians (20M in total at ``total_scale`` = 1), assigned to
    grid positions in a shuffled order; the generator is the urban one (facades + ground).
    Returns a list of Cell (no cameras: requests bring their own).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = [int(round(500_000 * (1 + k / 5) * total_scale)) for k in range(16)]
    order = rng.permutation(16)
    cells = []
    for k in range(16):
        slot = int(order[k])
        x0, z0 = 250.0 * (slot % 4), 250.0 * (slot // 4)
        n = sizes[k]
        pts = _city_points(rng, n, x0, x0 + 250.0, z0, z0 + 250.0, n_boxes=10)
        g = _gaussians(rng, pts, math.log(0.5 * math.sqrt(250.0 * 250.0 / n)), 0.5, 3)
        cells.append(Cell(g, _aabb(g.means)))
    return cells


RESOLUTIONS = ((1280, 720), (1920, 1080), (3840, 2160))
RESOLUTION_MIX = (0.50, 0.35, 0.15)


@dataclass
class Request:
    arrival_s: float
    camera: Camera
    rid: int = 0
    meta: dict = field(default_factory=dict)


def request_stream(seed: int = 5000, rate_hz: float = 200.0, duration_s: float = 30.0,
                   bounds=(0.0, 1000.0, 0.0, 1000.0)):
    """Poisson arrivals of novel-view requests over the merged city.

    Inter-arrival ~ Exp(rate); resolution mix 50 % 1280x720, 35 % 1920x1080, 15 % 3840x2160;
    camera position uniform in ``bounds`` at 20-150 m altitude, yaw ~ U(0, 2 pi),
    pitch ~ U(-90, -30) deg.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        w, h = RESOLUTIONS[int(rng.choice(3, p=RESOLUTION_MIX))]
        x = rng.uniform(bounds[0], bounds[1])
        z = rng.uniform(bounds[2], bounds[3])
        alt = rng.uniform(20.0, 150.0)
        yaw = rng.uniform(0.0, 2.0 * math.pi)
        pitch = math.radians(rng.uniform(-90.0, -30.0))
        cam = camera_from_forward((x, alt, z), yaw_pitch_forward(yaw, pitch), w, h,
                                  up_hint=(math.sin(yaw), 0.0, math.cos(yaw)) if pitch < -1.55
                                  else (0.0, 1.0, 0.0))
        out.append(Request(t, cam, len(out)))
    return out


def tiny_scene(n=40, width=32, height=32, degree=3, seed=0, box=1.0, dist=4.0,
               log_scale=(-2.5, 0.4), fx=None):
    """A handful of Gaussians in front of a small camera, for brute-force and FD checks."""
    rng = np.random.Generator(np.random.PCG64(seed))
    means = rng.uniform(-box, box, (n, 3))
    g = _gaussians(rng, means, log_scale[0], log_scale[1], degree, higher_std=0.3)
    cam = look_at((0.3, 0.2, -dist), (0.0, 0.0, 0.0), width, height,
                  fx=fx if fx is not None else 1.2 * width)
    return g, cam, random_target(rng, cam)
