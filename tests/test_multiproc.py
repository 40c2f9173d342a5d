"""The N>1 path of the benchmark on CPU: replicas with a barrier and a
max-over-ranks of the timings (gloo, world size 2), and the whole-job
aggregation of independent replicas."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys

    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, l = bench.dist_env()
    t = bench.reduce_max(10.0 + 5.0 * rank, w)  # rank 1 is the slowest
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, l, t))


def test_replicas_take_the_max_time_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[:3] for o in out] == [(0, 2, 0), (1, 2, 1)]
    assert all(o[3] == 15.0 for o in out)


def test_aggregate_is_all_units_over_the_slowest_rank():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    assert bench.aggregate([100.0, 100.0], [1.0, 2.0]) == 100.0
    assert bench.aggregate([50.0], [0.5]) == 100.0
