"""Host logic of bench.py's multi-GPU line (independent replicas, one
process per GPU): the job's time is the slowest rank's, the value counts
every rank's projections, and every rank projects its own models.  Two
gloo ranks on the CPU stand in for the GPUs."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    local_ms = 100.0 + 25.0 * rank          # rank 1 is the slow one
    total = bench.reduce_max(local_ms, dist, "cpu")
    seeds = [bench.replica_seed(rank, i) for i in range(4)]
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    out[rank] = (total, bench.job_throughput(world, 300, 2, total), gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_all_work():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        total, value, gathered = res[r]
        assert total == 125.0                       # the slowest rank's time on every rank
        assert value == pytest.approx(2 * 300 * 2 / 0.125)
        flat = [s for seeds in gathered for s in seeds]
        assert len(set(flat)) == len(flat)          # no two models share a seed


def test_single_process_passes_values_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(42.0, None, "cpu") == 42.0
    assert bench.job_throughput(1, 500, 10, 500.0) == pytest.approx(10000.0)
