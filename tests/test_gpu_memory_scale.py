"""The differentiable cell at memory scale (pattern 3): 20,000,000 Gaussians on urban facades and
ground, SH degree 3, one 1920x1080 camera, forward and backward through the torch.autograd.Function
(recompute from the stored final transmittance; no per-sample state).

Checks, all against the FP64 oracle on the tiles they concern:
  * the image on every tile that 1,000 randomly chosen visible Gaussians touch (max-abs 1e-4
    outside the pixels inside a decision band);
  * the gradients of those 1,000 Gaussians against tile-local central differences of the oracle's
    forward: per Gaussian, one direction per parameter group (mean, log-scale, quaternion, logit,
    SH), h = 1e-6 max(1, |theta|) per component, only that Gaussian re-projected and only its
    tiles re-composited.  Samples whose perturbation changes any decision are skipped.  Per group
    the directional derivatives hold the gradient tolerance (relative L2 2e-3 against the
    differences) and each is within 2e-3 |fd| + 1e-4 max|fd| of its difference.
The loss is L = sum(w * image) with random weights w, zeroed at the oracle's ambiguous pixels of
the checked tiles (there an FP32 and an FP64 decision may differ), so the backward pass starts
from dL/dimage = w.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2402_17427_gb300 import binding as B
from paper_2402_17427_gb300 import rasterize as R
from paper_2402_17427_gb300 import scenes

from _gpu import conservative_tile_rects, subset_reaching

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N_TARGETS = 1000
GROUPS = ("means", "log_scales", "quats", "logits", "sh")


@pytest.fixture(scope="module")
def urban():
    from paper_2402_17427_gb300 import _build
    _build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    g, cam, _ = scenes.urban_cell_20m()
    T = 16
    tx_n, ty_n = (cam.width + T - 1) // T, (cam.height + T - 1) // T
    rects = conservative_tile_rects(g, cam, T)
    rng = np.random.default_rng(41)
    cand_pool = np.nonzero(rects[0])[0]
    cand = rng.permutation(cand_pool)[:6 * N_TARGETS]
    # oracle renders of the candidates' tiles, a batch at a time, until enough targets are found
    batches, amb = [], np.zeros((cam.height, cam.width), bool)
    found = 0
    for b0 in range(0, len(cand), 500):
        cb = np.sort(cand[b0:b0 + 500])
        mask = np.zeros(tx_n * ty_n, np.uint8)
        for i in cb:
            mask.reshape(ty_n, tx_n)[rects[3][i]:rects[4][i] + 1, rects[1][i]:rects[2][i] + 1] = 1
        sub = subset_reaching(rects, mask, tx_n, ty_n)
        orc = oracle.render(g.subset(sub), cam, oracle.Options(), tile_mask=mask)
        pos = np.searchsorted(sub, cb)
        assert np.array_equal(sub[pos], cb)
        rec = orc.rec
        ok = rec["visible"][pos] & ~rec["grad_amb"][pos] & ~rec["rect_amb"][pos]
        tgt_sub = pos[ok][:N_TARGETS - found]
        found += len(tgt_sub)
        pm = np.repeat(np.repeat(mask.reshape(ty_n, tx_n).astype(bool), T, 0), T, 1)[:cam.height, :cam.width]
        amb |= pm & orc.amb.astype(bool)
        batches.append(dict(sub=sub, orc=orc, mask=mask, pix=pm, targets=tgt_sub))
        if found >= N_TARGETS:
            break
    assert found == N_TARGETS
    # GPU: forward through the autograd Function, L = sum(w * image), backward
    w = rng.standard_normal((3, cam.height, cam.width))
    w[:, amb] = 0.0
    params = [p.requires_grad_(True) for p in R.to_device(g)]
    torch.cuda.reset_peak_memory_stats()
    ras = R.Rasterizer()
    img = R.rasterize(*params, g.sh_degree, cam, ras)
    loss = (img * torch.from_numpy(w.astype(np.float32)).cuda()).sum()
    loss.backward()
    torch.cuda.synchronize()
    cnt = ras.counters.cpu().numpy()
    assert cnt[B.VG_CNT_STATUS] == 0
    out = dict(g=g, cam=cam, w=w, amb=amb, batches=batches, image=img.detach().cpu().numpy(),
               grads={k: p.grad.cpu().numpy() for k, p in zip(GROUPS, params)}, counters=cnt,
               peak=torch.cuda.max_memory_allocated())
    del params, img, loss, ras
    torch.cuda.empty_cache()
    return out


def test_urban_20m_autograd_image_on_checked_tiles(urban):
    cnt = urban["counters"]
    # about 4 % of the 20M Gaussians face this camera; every one of the 20M is projected
    assert 100_000 < cnt[B.VG_CNT_VISIBLE] < cnt[B.VG_CNT_PAIRS]
    checked = 0
    for b in urban["batches"]:
        ok = b["pix"] & ~b["orc"].amb.astype(bool)
        d = np.abs(urban["image"] - b["orc"].image)[:, ok]
        assert d.max() <= 1e-4, d.max()
        checked += int(ok.sum())
    assert checked > 100_000
    # everything of the 20M-Gaussian step fit on the device: parameters, gradients, workspace
    assert urban["peak"] < 40e9


def test_urban_20m_gradients_by_tile_local_central_differences(urban):
    g = urban["g"]
    K = 16
    F = 11 + 3 * K
    spans = {"means": (0, 3), "log_scales": (3, 6), "quats": (6, 10), "logits": (10, 11), "sh": (11, F)}
    G = urban["grads"]
    rng = np.random.default_rng(43)
    fd_all = {k: [] for k in GROUPS}
    an_all = {k: [] for k in GROUPS}
    skipped = 0
    for b in urban["batches"]:
        sub, orc, tg = b["sub"], b["orc"], b["targets"]
        if len(tg) == 0:
            continue
        full = sub[tg]                        # indices in the 20M set
        theta = np.concatenate([g.means[full], g.log_scales[full], g.quats[full], g.opacity_logits[full][:, None],
                                g.sh[full].reshape(len(full), -1)], 1).astype(np.float64)
        grad = np.concatenate([G["means"][full], G["log_scales"][full], G["quats"][full], G["logits"][full][:, None],
                               G["sh"][full].reshape(len(full), -1)], 1).astype(np.float64)
        for name in GROUPS:
            a, e = spans[name]
            dirs = np.zeros((len(tg), F))
            dirs[:, a:e] = rng.choice([-1.0, 1.0], (len(tg), e - a)) * np.maximum(1.0, np.abs(theta[:, a:e]))
            fd, flags = orc.fd_directional(urban["w"], tg, dirs, 1e-6)
            keep = flags == 0
            skipped += int((~keep).sum())
            fd_all[name].append(fd[keep])
            an_all[name].append((grad * dirs).sum(1)[keep])
    assert skipped <= 0.2 * 5 * N_TARGETS, skipped
    for name in GROUPS:
        fd = np.concatenate(fd_all[name])
        an = np.concatenate(an_all[name])
        assert len(fd) >= 0.8 * N_TARGETS, (name, len(fd))
        rel = np.linalg.norm(an - fd) / np.linalg.norm(fd)
        assert rel <= 2e-3, (name, rel)
        bound = 2e-3 * np.abs(fd) + 1e-4 * np.abs(fd).max()
        worst = np.argmax(np.abs(an - fd) - bound)
        assert np.all(np.abs(an - fd) <= bound), (name, fd[worst], an[worst])
