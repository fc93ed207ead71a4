"""The multi-GPU path of bench.py on CPU: replicas on world_size 2 with gloo.

Ranks fix independent problems; the only cross-rank operations are the
barrier and the reduction of the timing (max) and the work (sum)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    dist.barrier()
    # rank r "took" 1 + r seconds and did 100 * (r + 1) site-updates
    t, su = bench.reduce_over_ranks(1.0 + rank, 100.0 * (rank + 1))
    q.put((rank, t, su))
    dist.destroy_process_group()


def test_reduce_over_ranks_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, t, su in out:
        assert t == 2.0  # the slowest rank
        assert su == 300.0  # all ranks' work


def test_reduce_without_process_group():
    import bench

    assert bench.reduce_over_ranks(1.5, 42) == (1.5, 42.0)
