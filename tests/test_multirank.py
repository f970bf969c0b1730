"""The N > 1 path of bench.py on CPU: two gloo ranks (one per GPU in a real
run) take the max of their times and report the whole-job rate; every rank
solves its own batch (replicas, no collective on the data path); the
reference arm prints from rank 0 only."""

import contextlib
import io
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, local_ms, q):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        m = bench.max_over_ranks(local_ms[rank])
        rate = bench.whole_job_rate(1000, ws, 3, m)
        dist.barrier()
        q.put((rank, ws, r, local, m, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    local_ms = [12.5, 20.0]
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, local_ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, r, local, m, rate in got:
        assert (ws, r, local) == (2, rank, rank)
        assert m == 20.0                          # the slowest rank's time
        assert rate == pytest.approx(2 * 1000 * 3 / 0.020)  # units of both ranks / max time


def test_single_process_needs_no_process_group():
    import bench

    assert not dist.is_initialized()
    assert bench.max_over_ranks(7.0) == 7.0
    assert bench.whole_job_rate(10, 1, 2, 1000.0) == pytest.approx(20.0)


def test_replica_batches_differ_by_rank():
    import bench

    a0, a1 = bench.replica_batch(256, 0), bench.replica_batch(256, 1)
    assert a0.shape == a1.shape == (256, 6)
    assert not np.array_equal(a0, a1)
    assert np.array_equal(a0, bench.replica_batch(256, 0))


def test_reference_arm_prints_from_rank_zero_only(monkeypatch):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), {"n": 1024, "steps": 1, "warmup": 0, "gpus": 2})()
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        bench.run_reference(args)
    assert out.getvalue() == ""
