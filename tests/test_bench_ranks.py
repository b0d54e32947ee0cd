"""The replica bookkeeping of bench.py (barrier, max over ranks, whole-job rate) with two
gloo ranks on the CPU: the path a torchrun --nproc-per-node 2 bench run takes."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks("gloo")
    r.barrier()
    t = r.max(1.0 + rank)                 # rank 1 is the slowest
    rate = r.total_rate(1000, t)
    r.barrier()
    q.put((rank, r.world, t, rate))
    r.close()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(i, 2, port, q)) for i in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, world, t, rate in out:
        assert world == 2
        assert t == 2.0                   # max over ranks
        assert rate == 2 * 1000 / 2.0     # all ranks' units / slowest time


def test_single_rank_defaults():
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE"):
        os.environ.pop(k, None)
    r = bench.Ranks("gloo")
    assert r.world == 1 and r.max(3.5) == 3.5 and r.total_rate(10, 2.0) == 5.0
