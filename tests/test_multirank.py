"""Host logic of the multi-GPU bench path on CPU ranks (gloo, world size 2).

The single-system Barnes-Hut step does not shard, so several GPUs run
replicas: every rank times its own steps, the job time is the slowest rank's
and the rate counts every rank's particle-steps.  Two CPU processes exercise
exactly the functions bench.py uses for that.
"""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    my_seconds = 2.0 + rank  # rank 1 is the slower replica
    slowest = bench.max_over_ranks(my_seconds, "cpu")
    rate = bench.whole_job_rate(1000, 10, world, slowest)
    out.put((rank, slowest, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_use_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate in res:
        assert slowest == 3.0
        assert rate == pytest.approx(2 * 1000 * 10 / 3.0)


def test_single_process_rate():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(1.5) == 1.5
    assert bench.whole_job_rate(1048576, 60, 1, 0.4) == pytest.approx(1048576 * 60 / 0.4)
