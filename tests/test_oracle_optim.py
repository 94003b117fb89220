"""Pins of the optimiser-step oracle (Adam and adaptive densification; paper Sec. 3, Sec. 5.1)."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import optim as OO


def test_adam_constant_gradient_closed_form():
    # with a constant gradient the bias-corrected moments are exactly g and g^2, so every step
    # moves the parameter by lr * g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-3], np.float32)
    p, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    lr, eps = 0.01, 1e-15
    for t in range(1, 6):
        p, m, v = OO.adam_step(p, g, m, v, lr, t, eps=eps)
        gd = g.astype(np.float64)
        assert np.allclose(p, -t * lr * gd / (np.abs(gd) + eps), rtol=1e-12, atol=1e-15)


def test_accumulate_sums_normalised_norms():
    acc, cnt = OO.accumulate(np.zeros(4), np.zeros(4, np.int64), [1, 3, 1], [3.0, 0.0, -1.0], [0.0, 2.0, 0.0],
                             width=2, height=4)
    # ndc scaling: du * W/2 = du, dv * H/2 = 2 dv
    assert np.allclose(acc, [0, 3 + 1, 0, 4]) and list(cnt) == [0, 2, 0, 1]


def _params(n, rng):
    return {"means": rng.normal(0, 1, (n, 3)).astype(np.float32),
            "log_scales": rng.normal(-3, 0.3, (n, 3)).astype(np.float32),
            "quats": rng.normal(0, 1, (n, 4)).astype(np.float32),
            "opacity_logits": rng.normal(0, 1, n).astype(np.float32),
            "sh": rng.normal(0, 1, (n, 4, 3)).astype(np.float32)}


def test_densify_cases():
    rng = np.random.default_rng(0)
    P = _params(6, rng)
    th = OO.thresholds(2e-4, 0.01, 10.0, 0.005, 1.0)    # clone if max scale <= 0.1; drop if > 1
    P["opacity_logits"][0] = -6.0                         # 0: pruned (opacity < 0.005)
    P["log_scales"][2] = np.log([0.5, 0.2, 0.3])          # 2: split (max scale 0.5 > 0.1)
    P["log_scales"][3] = np.log([0.05, 0.02, 0.03])       # 3: clone
    P["log_scales"][4] = np.log([3.0, 0.2, 0.3])          # 4: split; children at 1.875 > 1: dropped
    P["opacity_logits"][1:] = 1.0
    acc = np.array([1.0, 0.0, 3e-3, 1e-3, 1.0, 1e-4], np.float32)
    cnt = np.array([1, 0, 10, 2, 1, 1])                   # grads 1, 0, 3e-4, 5e-4, 1, 1e-4
    P["log_scales"][5] = np.log([0.05, 0.02, 0.03])       # 5: grad below threshold: kept
    P["log_scales"][1] = np.log([0.05, 0.02, 0.03])       # 1: never seen: kept
    mom = {k: (np.full_like(v, 0.1), np.full_like(v, 0.2)) for k, v in P.items()}
    z = rng.standard_normal((6, 2, 3))
    out, outm, act = OO.densify(P, mom, acc, cnt, z, th)
    assert list(act) == [0, 1, 3, 2, 3, 1]
    # outputs: 1, split children of 2 (two), 3, copy of 3, (4 dropped), 5
    assert len(out["means"]) == 6
    assert np.array_equal(out["means"][0], P["means"][1].astype(np.float64))
    R = Rotation.from_quat(np.roll(P["quats"][2].astype(np.float64), -1)).as_matrix()   # scipy: (x, y, z, w)
    s = np.exp(P["log_scales"][2].astype(np.float64))
    for j in range(2):
        assert np.allclose(out["means"][1 + j], P["means"][2] + R @ (s * z[2, j]), rtol=1e-6, atol=1e-7)
        assert np.allclose(np.exp(out["log_scales"][1 + j]), s / 1.6, rtol=1e-6)
        assert np.all(outm["sh"][0][1 + j] == 0)
    assert np.array_equal(out["sh"][3], out["sh"][4]) and np.array_equal(out["sh"][3], P["sh"][3].astype(np.float64))
    assert np.all(outm["means"][0][3] == np.float32(0.1)) and np.all(outm["means"][0][4] == 0)   # kept; copy fresh
    assert np.array_equal(out["quats"][5], P["quats"][5].astype(np.float64))
