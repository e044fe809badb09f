"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The bench's rule for N > 1 ranks: every rank times its own replica, the
times are reduced with MAX, and the whole-job value counts the units all
ranks processed over that slowest time.  The reference arm runs on rank 0
only; other ranks exit 0 without work.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench as b
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.5, 20.0, 7.0, 19.5][rank]
        got = b.max_over_ranks(ms, world, "cpu")
        rate = b.job_rate(world, 65536 * 64, 10, got)
        dist.barrier()
        q.put((rank, got, rate))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_max_over_ranks_and_job_rate_gloo(world):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = max([12.5, 20.0, 7.0, 19.5][:world])
    for rank, got, rate in out:
        assert got == slowest
        assert rate == pytest.approx(world * 65536 * 64 * 10 / (slowest * 1e-3) / 1e9)


def test_single_rank_is_identity():
    assert bench.max_over_ranks(3.25, 1, "cpu") == 3.25
    assert bench.job_rate(1, 1000, 4, 2.0) == pytest.approx(1000 * 4 / 2e-3 / 1e9)


def test_reference_arm_other_ranks_exit_without_work(capsys):
    class A:
        steps, warmup, gpus = 2, 1, 2
    assert bench.run_reference(A(), dict(bench.WORKLOADS["fio1"]), 1, 2) == 0
    assert capsys.readouterr().out == ""
