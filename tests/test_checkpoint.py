"""Checkpoint / resume of a cell's training state (host side, no GPU): exact round trip of every
array and counter, refusal of corrupted, truncated or foreign files, and the atomic replace that
keeps the previous checkpoint when a write fails."""
import os

import numpy as np
import pytest
import torch

from paper_2402_17427_gb300 import checkpoint as CK
from paper_2402_17427_gb300 import optim as OP


def _state(n=257, degree=2, seed=0):
    g = torch.Generator().manual_seed(seed)
    K = (degree + 1) ** 2
    params = (torch.randn(n, 3, generator=g), torch.randn(n, 3, generator=g), torch.randn(n, 4, generator=g),
              torch.randn(n, generator=g), torch.randn(n, K, 3, generator=g))
    adam = OP.Adam(params)
    adam.m = tuple(torch.randn(t.shape, generator=g) for t in params)
    adam.v = tuple(torch.rand(t.shape, generator=g) for t in params)
    adam.t = 1234
    stats = OP.DensifyStats(n, "cpu")
    stats.accum = torch.rand(n, generator=g)
    stats.count = torch.randint(0, 50, (n,), generator=g, dtype=torch.int32)

    class App:      # the two arrays an appearance model carries
        params = torch.randn(255539, generator=g)
        embeddings = torch.randn(7, 64, generator=g)
    return params, degree, adam, stats, App()


def _same(a, b):
    return a.dtype == b.dtype and a.shape == b.shape and torch.equal(a, b)


def test_round_trip_is_exact(tmp_path):
    params, degree, adam, stats, app = _state()
    p = str(tmp_path / "cell3.vgckpt")
    CK.save(p, params, degree, iteration=4321, adam=adam, stats=stats, appearance=app, meta={"cell": 3})
    adam2, stats2 = OP.Adam(params), OP.DensifyStats(1, "cpu")

    class App2:
        params = embeddings = None
    app2 = App2()
    got, deg, it, meta = CK.load(p, "cpu", adam=adam2, stats=stats2, appearance=app2)
    assert deg == degree and it == 4321 and meta == {"cell": 3}
    assert all(_same(a, b) for a, b in zip(got, params))
    assert adam2.t == 1234
    assert all(_same(a, b) for a, b in zip(adam2.m, adam.m)) and all(_same(a, b) for a, b in zip(adam2.v, adam.v))
    assert _same(stats2.accum, stats.accum) and _same(stats2.count, stats.count)
    assert _same(app2.params, app.params) and _same(app2.embeddings, app.embeddings)


def test_params_only_and_missing_parts(tmp_path):
    params, degree, adam, stats, app = _state(n=0, degree=0)     # an empty cell is a valid state
    p = str(tmp_path / "empty.vgckpt")
    CK.save(p, params, degree)
    got, deg, it, _ = CK.load(p, "cpu")
    assert deg == 0 and it == 0 and all(_same(a, b) for a, b in zip(got, params))
    with pytest.raises(CK.CheckpointError):
        CK.load(p, "cpu", adam=OP.Adam(params))
    with pytest.raises(CK.CheckpointError):
        CK.load(p, "cpu", stats=OP.DensifyStats(0, "cpu"))


def test_corruption_truncation_and_foreign_files_are_refused(tmp_path):
    params, degree, adam, stats, app = _state(n=100)
    p = str(tmp_path / "c.vgckpt")
    CK.save(p, params, degree, adam=adam, stats=stats)
    raw = bytearray(open(p, "rb").read())
    meta, arrays = CK.read(p)
    # one flipped bit inside the last array's bytes
    bad = bytearray(raw)
    bad[-5] ^= 0x10
    q = str(tmp_path / "flip.vgckpt")
    open(q, "wb").write(bytes(bad))
    with pytest.raises(CK.CheckpointError, match="checksum"):
        CK.read(q)
    # cut short
    open(q, "wb").write(bytes(raw[:len(raw) // 2]))
    with pytest.raises(CK.CheckpointError):
        CK.read(q)
    # another file format
    open(q, "wb").write(b"\x93NUMPY" + bytes(100))
    with pytest.raises(CK.CheckpointError, match="not a checkpoint"):
        CK.read(q)
    # header bytes damaged
    bad = bytearray(raw)
    bad[20] = 0xFF
    open(q, "wb").write(bytes(bad))
    with pytest.raises(CK.CheckpointError):
        CK.read(q)


def test_failed_write_keeps_the_previous_checkpoint(tmp_path, monkeypatch):
    params, degree, adam, stats, app = _state(n=64)
    p = str(tmp_path / "c.vgckpt")
    CK.save(p, params, degree, iteration=1)
    before = open(p, "rb").read()
    params2 = tuple(t + 1 for t in params)

    def fail(*a, **k):
        raise OSError("disk full")
    monkeypatch.setattr(CK.os, "replace", fail)
    with pytest.raises(OSError):
        CK.save(p, params2, degree, iteration=2)
    monkeypatch.undo()
    assert open(p, "rb").read() == before
    assert os.listdir(tmp_path) == ["c.vgckpt"]          # no temporary file left behind
    _, _, it, _ = CK.load(p, "cpu")
    assert it == 1


def test_arrays_are_aligned_and_checksummed_in_the_header(tmp_path):
    params, degree, adam, stats, app = _state(n=33, degree=3)
    p = str(tmp_path / "c.vgckpt")
    CK.save(p, params, degree, adam=adam)
    meta, arrays = CK.read(p)
    assert meta["n"] == 33 and meta["adam_step"] == 1234
    assert set(arrays) == set(CK.PARAM_NAMES) | {"adam_m/" + k for k in CK.PARAM_NAMES} | \
        {"adam_v/" + k for k in CK.PARAM_NAMES}
    assert arrays["sh"].shape == (33, 16, 3) and arrays["sh"].dtype == np.float32
