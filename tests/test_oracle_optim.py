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


@pytest.mark.parametrize("betas,eps", [((0.9, 0.999), 1e-15), ((0.8, 0.95), 1e-8)])
def test_adam_matches_torch_optim_adam(betas, eps):
    # an independent implementation (torch.optim.Adam, FP64 on the CPU) over several steps of
    # gradients that change sign and magnitude from step to step, with elements small enough that
    # eps matters next to sqrt(v): swapped betas, eps inside the square root or a missing bias
    # correction each fail this
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    n = 64
    p0 = rng.normal(0.0, 1.0, n)
    scale = np.concatenate([np.full(n // 2, 1e-2), np.full(n // 4, 1e-9), np.full(n - n // 2 - n // 4, 1e-14)])
    lr = 0.003
    pt = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([pt], lr=lr, betas=betas, eps=eps)
    p, m, v = p0.copy(), np.zeros(n), np.zeros(n)
    for t in range(1, 8):
        g = (rng.standard_normal(n) * scale * (1.0 + t)).astype(np.float32)
        opt.zero_grad()
        pt.grad = torch.tensor(g.astype(np.float64))
        opt.step()
        p, m, v = OO.adam_step(p, g, m, v, lr, t, b1=betas[0], b2=betas[1], eps=eps)
        ref = pt.detach().numpy()
        assert np.allclose(p, ref, rtol=1e-12, atol=1e-15 * lr), (t, np.abs(p - ref).max())
        st = opt.state[pt]
        assert np.allclose(m, st["exp_avg"].numpy(), rtol=1e-12, atol=0)
        assert np.allclose(v, st["exp_avg_sq"].numpy(), rtol=1e-12, atol=0)


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
