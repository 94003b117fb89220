"""Concurrent callers: host threads rendering on streams of their own through the C ABI.

Each forward forks the tile counting to a side stream and joins it back, the backward forks the
zeroing of the culled Gaussians' gradients, and the loss forks its reduction; the events of those
forks are created once per host thread and reused by every call.  Four threads, each with its own
stream, rasteriser and loss object, run forward, loss and backward repeatedly on different scenes
at once.  The image and the loss must equal, bit for bit, the same scene run alone on the default
stream; the gradients, summed by atomics in an order the hardware picks, must agree to FP32
rounding (1e-5 of each array's largest magnitude).
"""
import threading

import numpy as np
import pytest
import torch

from paper_2402_17427_gb300 import rasterize as R
from paper_2402_17427_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2402_17427_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()


def _step(r, loss, params, deg, cam, target):
    rgb, T, last = r.forward(*params, deg, cam)
    L, dL = loss(rgb, target)
    grads = r.backward(*params, deg, cam, T, last, dL)
    return [rgb, L] + [g for g in grads if isinstance(g, torch.Tensor)]


def test_threads_on_own_streams_match_serial_runs():
    cases = [scenes.tiny_scene(n=400 + 150 * k, width=96 + 16 * k, height=80, degree=k % 4, seed=20 + k)
             for k in range(4)]
    cases.append(scenes.small_cell(1))
    dev = [(R.to_device(g), g.sh_degree, cam, torch.from_numpy(np.asarray(t, np.float32)).cuda())
           for g, cam, t in cases]
    # alone, on the default stream
    ref = []
    for params, deg, cam, target in dev:
        out = _step(R.Rasterizer(), R.LossL1DSSIM(0.2), params, deg, cam, target)
        torch.cuda.synchronize()
        ref.append([t.clone() for t in out])
    errors, results = [], {}

    def worker(k):
        try:
            s = torch.cuda.Stream()
            r, loss = R.Rasterizer(), R.LossL1DSSIM(0.2)
            with torch.cuda.stream(s):
                for it in range(6):
                    j = (k + it) % len(dev)
                    params, deg, cam, target = dev[j]
                    out = _step(r, loss, params, deg, cam, target)
                    s.synchronize()
                    results[(k, it)] = (j, [t.clone() for t in out])
        except Exception as e:      # reported to the main thread
            errors.append(repr(e))

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    assert len(results) == 24
    for (k, it), (j, out) in results.items():
        assert len(out) == len(ref[j])
        assert torch.equal(out[0], ref[j][0]) and torch.equal(out[1], ref[j][1]), (k, it, j)
        for a, b in zip(out[2:], ref[j][2:]):
            tol = 1e-5 * float(b.abs().max()) + 1e-30
            assert float((a - b).abs().max()) <= tol, (k, it, j)


def test_appearance_calls_on_concurrent_streams_match_serial_runs():
    """Two host threads evaluate the appearance loss (Eq. 3) with every gradient on streams of their
    own at once: their tensor-core passes allocate tensor memory side by side on the same SMs.  The
    loss and the map must equal the serial runs bit for bit, the gradients to FP32 rounding."""
    from paper_2402_17427_gb300 import appearance as AP
    rng = np.random.default_rng(11)
    cases = []
    for k, (W, H) in enumerate([(640, 360), (512, 384)]):
        img = torch.from_numpy(rng.random((3, H, W), dtype=np.float32)).cuda()
        tgt = torch.from_numpy(rng.random((3, H, W), dtype=np.float32)).cuda()
        cases.append((img, tgt))
    models = [AP.AppearanceModel(2, seed=3), AP.AppearanceModel(2, seed=3)]
    ref = []
    for (img, tgt), m in zip(cases, models):
        out = m.loss(img, tgt, 1, 0.2, want_map=True)
        torch.cuda.synchronize()
        ref.append({k: v.clone() for k, v in out.items()})
    errors, results = [], {}

    def worker(k):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                for it in range(5):
                    out = models[k].loss(cases[k][0], cases[k][1], 1, 0.2, want_map=True)
                    s.synchronize()
                    results[(k, it)] = {n: v.clone() for n, v in out.items()}
        except Exception as e:      # reported to the main thread
            errors.append(repr(e))

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    assert len(results) == 10
    for (k, it), out in results.items():
        assert torch.equal(out["loss"], ref[k]["loss"]) and torch.equal(out["map"], ref[k]["map"]), (k, it)
        for n in ("grad_img", "grad_embedding", "grad_params"):
            tol = 1e-5 * float(ref[k][n].abs().max()) + 1e-30
            assert float((out[n] - ref[k][n]).abs().max()) <= tol, (k, it, n)
