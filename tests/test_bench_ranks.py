"""bench.py's multi-rank logic and the request partitioner, on CPU with two gloo ranks.

The device calls are replaced by the oracle (tables) and by fixed per-rank step times;
what runs is the code bench.py runs under torchrun: the interval shard of each rank,
the max over ranks of the step time, the whole-job value computed from it, the sum
of the ranks' composite counts, and the partition of one seeded request list into
per-rank replicas for the batch and serving forms."""
import os
import socket

import pytest

import bench
import oracle
from paper_1111_3297_gb300 import shard, workloads

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_partition_is_disjoint_complete_and_balanced():
    reqs = workloads.batch_requests(500, seed=3)
    costs = [shard.request_cost(j0, nb) for j0, nb in reqs]
    for world in (1, 2, 3, 8):
        parts = [shard.partition_requests(reqs, r, world) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(reqs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs) + 1e-6
        assert all(p == sorted(p) for p in parts)
    with pytest.raises(ValueError):
        shard.partition_requests(reqs, 2, 2)


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = {}
    # interval shards, as bench.main takes them: weak scaling, each rank its own n segments
    l, f0, n, steps = 10, 4321, 5, 7
    fr, nr = shard.shard(l, f0, n, rank, world, "weak")
    local = oracle.popcount(oracle.sieve(l, fr, nr, nthreads=1))
    res["total"] = shard.total_count(local)
    ms = 10.0 + 5.0 * rank  # the stand-in for each rank's measured step time
    res["ms_max"] = bench.max_over_ranks(dist, ms)
    res["value"] = bench.job_value(world, nr << l, steps, res["ms_max"])
    # replicas of the batched form: each rank its share of one request list
    reqs = [(j0, nb) for j0, nb in workloads.batch_requests(40, seed=9) if nb <= 1 << 18]
    mine = shard.partition_requests(reqs, rank, world)
    counts = {i: oracle.popcount(oracle.sieve_range(reqs[i][0], reqs[i][1], nthreads=1)) for i in mine}
    gathered = [None] * world
    dist.all_gather_object(gathered, counts)
    res["batch_total"] = shard.total_count(sum(counts.values()))
    if rank == 0:
        q.put((res, gathered, reqs))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_run_the_bench_rank_logic():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world = 2
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res, gathered, reqs = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    l, f0, n, steps = 10, 4321, 5, 7
    assert res["total"] == oracle.popcount(oracle.sieve(l, f0, world * n))
    assert res["ms_max"] == 15.0
    assert res["value"] == world * (n << l) * steps / 15e-3
    # every request served by exactly one rank, with the oracle's count
    seen = {}
    for part in gathered:
        for i, c in part.items():
            assert i not in seen
            seen[i] = c
    assert sorted(seen) == list(range(len(reqs)))
    assert res["batch_total"] == sum(seen.values())
