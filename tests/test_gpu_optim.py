"""GPU parity of the optimiser step (Adam, densification statistics, clone / split / prune;
paper Sec. 3 and Sec. 5.1) against the optimiser oracle."""
import numpy as np
import pytest
import torch

import oracle
from oracle import optim as OO
from paper_2402_17427_gb300 import optim as OP
from paper_2402_17427_gb300 import rasterize as R
from paper_2402_17427_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2402_17427_gb300 import _build
    _build.build()
    oracle.build()
    assert torch.cuda.is_available()


def _rand_params(n, degree, rng):
    k = (degree + 1) ** 2
    return [rng.normal(0, 1, (n, 3)).astype(np.float32), rng.normal(-3, 0.3, (n, 3)).astype(np.float32),
            rng.normal(0, 1, (n, 4)).astype(np.float32), rng.normal(0, 1, n).astype(np.float32),
            rng.normal(0, 1, (n, k, 3)).astype(np.float32)]


@pytest.mark.parametrize("n,degree", [(1001, 3), (37, 0), (258, 2)])
def test_adam_matches_oracle(n, degree):
    rng = np.random.default_rng(n)
    P = _rand_params(n, degree, rng)
    s = OP.AdamSettings()
    params = [torch.from_numpy(a.copy()).cuda() for a in P]
    adam = OP.Adam(params, s)
    ref = [a.astype(np.float64) for a in P]
    rm = [np.zeros_like(a, np.float64) for a in P]
    rv = [np.zeros_like(a, np.float64) for a in P]
    lrs = [s.lr_means, s.lr_log_scales, s.lr_quats, s.lr_opacity]
    lr_sh = np.full(P[4].shape, s.lr_sh_rest)
    lr_sh[:, 0, :] = s.lr_sh_dc           # the degree-0 coefficients have their own rate
    for t in range(1, 4):
        G = [rng.normal(0, 1e-2, a.shape).astype(np.float32) for a in P]
        adam.step(params, [torch.from_numpy(g).cuda() for g in G], degree)
        for k in range(4):
            ref[k], rm[k], rv[k] = OO.adam_step(ref[k], G[k], rm[k], rv[k], lrs[k], t, s.beta1, s.beta2, s.eps)
        ref[4], rm[4], rv[4] = OO.adam_step(ref[4], G[4], rm[4], rv[4], lr_sh, t, s.beta1, s.beta2, s.eps)
    torch.cuda.synchronize()
    for k in range(5):
        assert np.allclose(params[k].cpu().numpy(), ref[k], rtol=1e-5, atol=1e-7), k
        assert np.allclose(adam.m[k].cpu().numpy(), rm[k], rtol=1e-5, atol=1e-9), k
        assert np.allclose(adam.v[k].cpu().numpy(), rv[k], rtol=1e-4, atol=1e-12), k


def test_densification_statistics_match_oracle():
    g, cam, _ = scenes.tiny_scene(n=180, width=48, height=40, degree=2, seed=5)
    rng = np.random.default_rng(6)
    dL = rng.standard_normal((3, cam.height, cam.width)).astype(np.float32)
    ras = R.Rasterizer(R.RasterSettings())
    params = R.to_device(g)
    rgb, T, last = ras.forward(*params, g.sh_degree, cam)
    ras.backward(*params, g.sh_degree, cam, T, last, torch.from_numpy(dL).cuda())
    stats = OP.DensifyStats(g.n, "cuda")
    stats.add_view(ras, g.n, cam)
    stats.add_view(ras, g.n, cam)       # a second view of the same render doubles both
    torch.cuda.synchronize()
    orc = oracle.render(g, cam)
    g2d = orc.backward(dL.astype(np.float64))["g2d"]
    vis = np.nonzero(orc.rec["visible"])[0]
    acc, cnt = OO.accumulate(np.zeros(g.n), np.zeros(g.n, np.int64), np.concatenate([vis, vis]),
                             np.concatenate([g2d[vis, 0]] * 2), np.concatenate([g2d[vis, 1]] * 2), cam.width, cam.height)
    assert np.array_equal(stats.count.cpu().numpy(), cnt)
    keep = ~(orc.rec["grad_amb"] | orc.rec["rect_amb"])
    a = stats.accum.cpu().numpy().astype(np.float64)
    assert np.abs(a - acc)[keep].max() <= 2e-3 * np.abs(acc).max() + 1e-9


@pytest.mark.parametrize("degree", [3, 1])
def test_densify_matches_oracle(degree):
    rng = np.random.default_rng(10 + degree)
    n = 5000
    P = _rand_params(n, degree, rng)
    P[1] = rng.normal(np.log(0.05), 0.8, (n, 3)).astype(np.float32)        # clone / split / too-big mix
    P[3] = rng.normal(0, 3, n).astype(np.float32)                           # some below min opacity
    acc = rng.exponential(3e-4, n).astype(np.float32)
    cnt = rng.integers(0, 4, n).astype(np.int32)
    z = rng.standard_normal((n, 2, 3)).astype(np.float32)
    ds = OP.DensifySettings(scene_extent=10.0)
    params = [torch.from_numpy(a.copy()).cuda() for a in P]
    adam = OP.Adam(params)
    mom = [rng.random(a.shape).astype(np.float32) for a in P]
    adam.m = tuple(torch.from_numpy(a.copy()).cuda() for a in mom)
    adam.v = tuple(torch.from_numpy((2 * a).copy()).cuda() for a in mom)
    stats = OP.DensifyStats(n, "cuda")
    stats.accum.copy_(torch.from_numpy(acc))
    stats.count.copy_(torch.from_numpy(cnt))
    # the kernel's FP32 thresholds come from the FP32-rounded settings it receives
    f = np.float32
    th = OO.thresholds(f(ds.grad_threshold), float(f(ds.percent_dense)), float(f(ds.scene_extent)),
                       float(f(ds.min_opacity)), float(f(ds.max_world_scale_frac * ds.scene_extent)))
    names = OP.PARAM_NAMES
    new = OP.densify_with(params, adam, stats, degree, ds, torch.from_numpy(z).cuda())
    ref, refm, act = OO.densify(dict(zip(names, P)), {k: (mom[i], 2 * mom[i]) for i, k in enumerate(names)},
                                acc, cnt, z.astype(np.float64), th)
    assert set(np.unique(act)) == {0, 1, 2, 3}
    m = int(new[0].shape[0])
    assert m == len(ref["means"])
    assert int(stats.accum.shape[0]) == m and int(stats.count.sum()) == 0
    for i, k in enumerate(names):
        got = new[i].cpu().numpy().astype(np.float64)
        if k == "means":
            assert np.allclose(got, ref[k], rtol=1e-5, atol=1e-6)
        else:
            assert np.array_equal(got, ref[k]), k
        assert np.array_equal(adam.m[i].cpu().numpy().astype(np.float64), refm[k][0]), k
        assert np.array_equal(adam.v[i].cpu().numpy().astype(np.float64), refm[k][1]), k
