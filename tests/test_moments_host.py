"""The adjoint compositing kernel reduces, per (warp, splat), six moments of dpow = alpha dL/dalpha
over the warp's pixels, and the 2D gradient (du, dv, the conic's three entries, the opacity) is
formed from the moments' totals once per Gaussian (grad2d_from_moments in csrc/vg_common.cuh).
This CPU test compiles that map as host code and checks it against the gradient written out per
pixel from the definitions (Sec. 3: alpha = o exp(P), P = -(a dx^2 + c dy^2) / 2 - b dx dy,
dx = x - u, dy = y - v), summed in FP64 over random pixels:
  dL/du = sum g (a dx + b dy),  dL/dv = sum g (b dx + c dy),
  dL/da = -sum g dx^2 / 2,  dL/db = -sum g dx dy,  dL/dc = -sum g dy^2 / 2,  dL/do = sum g / o,
with g = alpha dL/dalpha = dL/dP.  A dropped factor, a sign or the log2 scaling of the stored conic
going wrong fails it."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2402_17427_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")

PROGRAM = r"""
#include <cstdio>
#include "vg_common.cuh"
int main() {
  float m[6], ca, cb, cc, lo, d[6];
  while (std::scanf("%f %f %f %f %f %f %f %f %f %f", &m[0], &m[1], &m[2], &m[3], &m[4], &m[5], &ca, &cb, &cc, &lo) == 10) {
    vg::grad2d_from_moments(m, ca, cb, cc, lo, d);
    std::printf("%.9g %.9g %.9g %.9g %.9g %.9g\n", d[0], d[1], d[2], d[3], d[4], d[5]);
  }
  return 0;
}
"""


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


@pytest.fixture(scope="module")
def host_map(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("moments")
    src, exe = d / "moments.cu", d / "moments"
    src.write_text(PROGRAM)
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O2", "-I" + INCLUDE,
                    "-I" + CSRC, str(src), "-o", str(exe)], check=True, capture_output=True)

    def run(rows):
        text = "\n".join(" ".join("%.9g" % v for v in r) for r in rows) + "\n"
        out = subprocess.run([str(exe)], input=text, capture_output=True, text=True, check=True).stdout
        return np.array([[float(x) for x in line.split()] for line in out.strip().splitlines()])
    return run


def test_moment_map_matches_per_pixel_gradients(host_map):
    rng = np.random.default_rng(7)
    log2e = 1.0 / math.log(2.0)
    rows, want = [], []
    for _ in range(200):
        # a positive-definite conic (a, b, c), an opacity, a centre and a pixel block near it
        L = rng.normal(size=(2, 2)) + 2.0 * np.eye(2)
        cov = L @ L.T * rng.uniform(0.5, 20.0)
        a, b, c = np.linalg.inv(cov)[0, 0], np.linalg.inv(cov)[0, 1], np.linalg.inv(cov)[1, 1]
        o = rng.uniform(0.05, 0.99)
        u, v = rng.uniform(-3, 3, 2)
        xs, ys = np.meshgrid(np.arange(-8, 8), np.arange(-4, 4))
        dx, dy = (xs - u).ravel(), (ys - v).ravel()
        g = rng.normal(size=dx.size)                     # dL/dP at each pixel
        m = [np.sum(g * dx), np.sum(g * dy), np.sum(g * dx * dx), np.sum(g * dx * dy), np.sum(g * dy * dy), np.sum(g)]
        # the splat record stores the conic scaled to log2 units and log2(opacity)
        rows.append(m + [-0.5 * log2e * a, -log2e * b, -0.5 * log2e * c, math.log2(o)])
        want.append([np.sum(g * (a * dx + b * dy)), np.sum(g * (b * dx + c * dy)), -0.5 * np.sum(g * dx * dx),
                     -np.sum(g * dx * dy), -0.5 * np.sum(g * dy * dy), np.sum(g) / o])
    got, want = host_map(rows), np.array(want)
    # FP32 inputs and arithmetic: compare per field against the field's scale
    scale = np.abs(want).max(axis=0)
    err = np.abs(got - want).max(axis=0) / scale
    assert (err < 1e-5).all(), err
