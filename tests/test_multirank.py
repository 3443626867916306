"""Host logic of the multi-GPU paths on CPU ranks (gloo, world size 2).

The single-system Barnes-Hut step does not shard, so several GPUs run
replicas: every rank times its own steps, the job time is the slowest rank's
and the rate counts every rank's particle-steps.  A batch of independent
systems does shard: each rank takes a balanced share of the systems and the
per-system results are gathered once at the end.  Two CPU processes exercise
exactly the functions bench.py uses for both.
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


def _shard_rank(rank, world, port, out):
    import numpy as np
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1212_2934_gb300 import shard

    sizes = np.array([5, 3, 9, 1, 4, 4, 7])
    parts = shard.partition_systems(sizes, world)
    mine = parts[rank]
    # stand-in per-system results: rows that name their system
    vals = np.stack([mine * 10.0, sizes[mine] * 1.0], axis=1) if len(mine) else np.zeros((0, 2))
    full = shard.gather_system_values(vals, mine, len(sizes))
    out.put((rank, [p.tolist() for p in parts], full.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_batch_shards_and_gathers_in_system_order():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 30500 + os.getpid() % 1000
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sizes = [5, 3, 9, 1, 4, 4, 7]
    (_, parts0, full0), (_, parts1, full1) = res
    assert parts0 == parts1  # every rank computes the same split
    assert sorted(parts0[0] + parts0[1]) == list(range(7))
    loads = [sum(sizes[i] for i in p) for p in parts0]
    assert abs(loads[0] - loads[1]) <= max(sizes)
    want = [[10.0 * i, float(sizes[i])] for i in range(7)]
    assert full0 == want and full1 == want


def test_partition_rules():
    import numpy as np

    sys.path.insert(0, ROOT)
    from paper_1212_2934_gb300 import shard

    # longest-processing-time by hand (loads after each step): #2 (9) -> r0 [9, 0];
    # #6 (7) -> r1 [9, 7]; #0 (5) -> r1 [9, 12]; #4 (4) -> r0 [13, 12]; #5 (4) -> r1 [13, 16];
    # #1 (3) -> r0 [16, 16]; #3 (1) -> r0 on the tie [17, 16]
    sizes = np.array([5, 3, 9, 1, 4, 4, 7])
    p = shard.partition_systems(sizes, 2)
    assert [x.tolist() for x in p] == [[1, 2, 3, 4], [0, 5, 6]]
    assert [int(sizes[x].sum()) for x in p] == [17, 16]
    # fewer systems than ranks: empty shares, nothing lost
    p = shard.partition_systems([3, 2], 4)
    assert [x.tolist() for x in p] == [[0], [1], [], []]
    # the bench batch: 256 log-uniform systems over 8 ranks stay within one system of even
    from paper_1212_2934_gb300 import synth

    s = synth.batched_sizes(256)
    loads = [int(s[x].sum()) for x in shard.partition_systems(s, 8)]
    assert max(loads) - min(loads) <= int(s.max())
    assert sum(loads) == int(s.sum())
    with pytest.raises(ValueError):
        shard.partition_systems([3, 0], 2)
    # a rank's slice of the concatenated arrays
    b = {"pos": np.arange(10.0)[:, None] * np.ones(3), "u": np.ones((10, 3)),
         "sizes": np.array([2, 3, 5]), "fields": np.eye(3), "box_lo": np.zeros((3, 3)),
         "box_hi": np.ones((3, 3))}
    sl = shard.rank_slice(b, [0, 2])
    assert sl["pos"][:, 0].tolist() == [0, 1, 5, 6, 7, 8, 9]
    assert sl["sizes"].tolist() == [2, 5] and sl["fields"].tolist() == [[1, 0, 0], [0, 0, 1]]
