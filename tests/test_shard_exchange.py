"""The sharded apply's exchange on CPU ranks (gloo, world size 2 and 4).

ShardedApply.apply_distributed runs front -> all_to_all_single -> back.  Here
the two kernel halves are replaced by stand-ins that write and check the
workspace layout documented in include/bf_shard.h (per-peer blocks
[peer][slice][a_loc][b_loc]), so the test checks that every switch-level pair
(a, b) written by the shard owning b reaches the shard owning a, at the place
that shard's back half reads it.
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


def _code(a, b, sl):
    return float(a * 10000 + b * 10 + sl)


def _worker(rank, world, port, la, lb, nslice, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from paper_1803_04128_gb300 import api
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A, B = 1 << la, 1 << lb
        blk = nslice * A * B                       # pairs per peer block (one complex per pair here)
        sh = api.ShardedApply.__new__(api.ShardedApply)
        sh.G, sh.m, sh.chunk, sh.rows = world, 1, blk, 1

        def front(s, F_rows, W_send, stream=None):   # pair (a, b): a = d A + a_loc, b = s B + b_loc
            for d in range(world):
                for sl in range(nslice):
                    for al in range(A):
                        for bl in range(B):
                            W_send[d * blk + sl * A * B + al * B + bl] = _code(d * A + al, s * B + bl, sl)

        def back(d, W_recv, G_rows, stream=None):
            bad = 0
            for s in range(world):
                for sl in range(nslice):
                    for al in range(A):
                        for bl in range(B):
                            v = W_recv[s * blk + sl * A * B + al * B + bl]
                            bad += int(v.real.item() != _code(d * A + al, s * B + bl, sl))
            G_rows[0] = bad

        sh.front, sh.back = front, back
        F = torch.zeros(1, dtype=torch.complex64)
        Gr = torch.full((1,), -1.0, dtype=torch.complex64)
        sh.apply_distributed(F, Gr)
        q.put((rank, int(Gr[0].real.item())))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,la,lb,nslice", [(2, 2, 3, 2), (4, 1, 2, 3)])
def test_apply_distributed_routes_every_pair(world, la, lb, nslice):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, la, lb, nslice, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(r, 0) for r in range(world)]
