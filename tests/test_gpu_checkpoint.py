"""Resume from a checkpoint on the GPU: a cell trained for a few steps, saved, and loaded into fresh
objects continues exactly as the uninterrupted run does (the same Adam update and densification
statistics, bit for bit, for the same gradients)."""
import pytest
import torch

from paper_2402_17427_gb300 import checkpoint as CK
from paper_2402_17427_gb300 import optim as OP
from paper_2402_17427_gb300 import rasterize as R
from paper_2402_17427_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2402_17427_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()


def test_resume_continues_bit_for_bit(tmp_path):
    g, cam, target = scenes.small_cell(2)
    params = R.to_device(g)
    tgt = torch.from_numpy(target).cuda()
    r, loss = R.Rasterizer(), R.LossL1DSSIM(0.2)
    adam, stats = OP.Adam(params), OP.DensifyStats(g.n, "cuda")

    def grads_of(ps, rast):
        rgb, T, last = rast.forward(*ps, g.sh_degree, cam)
        _, dL = loss(rgb, tgt)
        return rast.backward(*ps, g.sh_degree, cam, T, last, dL)

    for _ in range(3):
        gr = grads_of(params, r)
        stats.add_view(r, g.n, cam)
        adam.step(params, gr, g.sh_degree)
    p = str(tmp_path / "cell.vgckpt")
    CK.save(p, params, g.sh_degree, iteration=3, adam=adam, stats=stats)
    # the next step's gradients, shared by both runs (the adjoint's atomics sum in an order the
    # hardware picks, so each run must not draw its own)
    gr = [t.clone() for t in grads_of(params, r)]
    stats.add_view(r, g.n, cam)
    adam.step(params, gr, g.sh_degree)
    # resumed: fresh objects filled from the file, the same step
    adam2, stats2 = OP.Adam(params), OP.DensifyStats(1, "cuda")
    params2, deg, it, _ = CK.load(p, "cuda", adam=adam2, stats=stats2)
    assert deg == g.sh_degree and it == 3 and adam2.t == 3
    r2 = R.Rasterizer()
    rgb2, T2, last2 = r2.forward(*params2, g.sh_degree, cam)
    _, dL2 = loss(rgb2, tgt)
    r2.backward(*params2, g.sh_degree, cam, T2, last2, dL2)    # this view's 2D mean gradients, for the statistics
    stats2.add_view(r2, g.n, cam)
    adam2.step(params2, gr, g.sh_degree)
    torch.cuda.synchronize()
    for a, b in zip(params, params2):
        assert torch.equal(a, b)
    for a, b in zip(adam.m + adam.v, adam2.m + adam2.v):
        assert torch.equal(a, b)
    assert torch.equal(stats.count, stats2.count)
    assert torch.allclose(stats.accum, stats2.accum, rtol=1e-5, atol=0)
