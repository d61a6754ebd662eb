"""The multi-rank path of bench.py on CPU with gloo, world size 2: every rank runs its own
replica (there is no collective on the data path); the job's time is the slowest rank's and
its throughput counts every rank's units."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_time = 1.5 + rank          # rank 1 is the slow one
    t = bench.dist_max(local_time, dist)
    value = bench.job_throughput(1000, world, t)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, value))


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, value in out:
        assert t == 2.5                 # the slowest rank's time on every rank
        assert value == pytest.approx(2 * 1000 / 2.5)


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_max(3.0) == 3.0
    assert bench.job_throughput(10, 1, 2.0) == 5.0
