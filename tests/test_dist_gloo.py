"""The multi-GPU harness of bench.py on CPU with two gloo ranks: every rank
evaluates its own walkers (weak scaling, no exchange in the data path); the
timing is the maximum over ranks and the units the sum."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r, w, _ = bench.dist_env()
    bench.dist_init(w)
    # rank r "took" (r + 1) * 10 ms for 100 * (r + 1) units
    ms, units = bench.aggregate(10.0 * (r + 1), 100.0 * (r + 1))
    bench.barrier()
    q.put((r, ms, units))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for r, ms, units in res:
        assert ms == 20.0          # max over ranks
        assert units == 300.0      # sum over ranks


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(12.5, 7.0) == (12.5, 7.0)
