"""The multi-rank host path of bench.py on CPU ranks (gloo, world size 2, 127.0.0.1).

Cells are independent, so N GPUs run N replicas with no data-path collective; what the ranks
share is the timing: the job's step time is the slowest rank's, and the job's rate counts the
steps of every rank.  These tests run that reduction on two gloo ranks, and check that the
reference arm does its work on rank 0 only.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, times, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, _ = bench.dist_setup()
        slow = bench.slowest_ms(dist, times[rank], "cpu")
        q.put((got_ws, got_rank, slow, bench.job_rate(ws, slow)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _run_ranks(times):
    import torch.multiprocessing as mp
    ws, port = len(times), _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, times, q)) for r in range(ws)]
    for p in procs:
        p.start()
    try:
        out = sorted(q.get(timeout=180) for _ in range(ws))
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    return out


def test_job_time_is_the_slowest_rank_and_rate_counts_every_rank():
    times = [4.0, 7.5]
    out = _run_ranks(times)
    assert [o[:2] for o in out] == [(2, 0), (2, 1)]          # world size and rank from the env
    for _, _, slow, rate in out:
        assert slow == max(times)                             # every rank agrees on the max
        assert rate == pytest.approx(2 * 1000.0 / max(times))


def test_single_rank_reduction_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_ms(None, 3.25, "cpu") == 3.25
    assert bench.job_rate(1, 4.0) == pytest.approx(250.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    calls = []
    monkeypatch.setattr(bench, "oracle_sampled_step", lambda *a, **k: calls.append(a) or (1.0, 2.0, 1, "x"))
    # a rank other than 0 returns before reading its arguments, the scene or the oracle
    assert bench.run_reference(None, 2, 1) is None
    assert calls == []


def test_cpu_baseline_samplers_run_on_a_tiny_scene():
    """The two oracle timings bench.py reports (the CPU baseline of the main line, on all host
    threads and on one, and the reference arm's sampled step) run for real on a small scene."""
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_2402_17427_gb300 import scenes
    oracle.build()
    g, cam, target = scenes.tiny_scene(n=200, width=64, height=48, degree=2, seed=3)
    t, threads, sample = bench.oracle_step_time(g, cam, target, 0.5)
    assert t > 0 and threads >= 1 and "tiles" in sample
    t1, threads1, _ = bench.oracle_step_time(g, cam, target, 0.5, seed=1, threads=1)
    assert t1 > 0 and threads1 == 1
    took, full, threads2, sample2 = bench.oracle_sampled_step(g, cam, target, 0.5, seed=0)
    assert 0 < took and 0 < full and threads2 >= 1 and "tiles" in sample2
