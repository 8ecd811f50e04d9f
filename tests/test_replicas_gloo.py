"""The multi-GPU path is replicas only: every rank decomposes its own
problems and the job's time is the slowest rank's.  The host side of that --
the max-over-ranks reduction and the per-rank problem seeds of ``bench.py``
-- runs here as two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 20.0][rank]
    got = bench.max_over_ranks(ms, dist, "cpu")
    seeds = [bench.problem_seed(rank, i) for i in range(1000)]
    q.put((rank, got, seeds))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_draw_disjoint_problems():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        r, got, seeds = q.get(timeout=120)
        res[r] = (got, seeds)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][0] == res[1][0] == 20.0
    assert not set(res[0][1]) & set(res[1][1])
    assert bench.max_over_ranks(7.0, None, "cpu") == 7.0
