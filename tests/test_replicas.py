"""Multi-rank replica logic of bench.py on CPU (gloo, world size 2).

bench.py runs one independent solve stream per GPU under torchrun; the only
cross-rank traffic is the barrier around the timed region and the max of
its duration.  These tests run that bookkeeping as two CPU processes.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    rep = bench.Replicas(world)
    rep.barrier()
    # rank r "timed" 100 + 50 r ms for 5 steps: the job's time is the slowest rank's
    region = rep.max(100.0 + 50.0 * rank)
    value = rep.aggregate(5, region)
    # the reference arm: rank 0 alone runs (here: the others return without work)
    ran = None
    if rank != 0:
        class A:
            pass
        ran = bench.run_reference(A(), rank)
    out.put((rank, region, value, ran))
    torch.distributed.destroy_process_group()


def test_replicas_barrier_and_max_over_ranks_gloo():
    world = 2
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, region, value, ran in res:
        assert region == pytest.approx(150.0)          # max over ranks
        assert value == pytest.approx(world * 5 / 0.150)  # all ranks' steps over the slowest time
        assert ran is None


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    rep = bench.Replicas(1)
    rep.barrier()
    assert rep.max(3.0) == 3.0
    assert rep.aggregate(4, 2000.0) == pytest.approx(2.0)
