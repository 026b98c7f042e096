"""Multi-rank path on CPU: two gloo ranks sieve their shards (with the oracle) and
sum their counts; the union equals the single-rank result."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1111_3297_gb300 import shard

torch = pytest.importorskip("torch")


def test_shards_tile_the_interval():
    l, f, n = 12, 1000, 37
    for world in (1, 2, 3, 8):
        parts = [shard.shard(l, f, n, r, world, "strong") for r in range(world)]
        assert parts[0][0] == f
        for (fa, na), (fb, _) in zip(parts, parts[1:]):
            assert fa + na == fb
        assert sum(nr for _, nr in parts) == n
        weak = [shard.shard(l, f, n, r, world, "weak") for r in range(world)]
        assert weak == [(f + r * n, n) for r in range(world)]
    with pytest.raises(ValueError):
        shard.shard(l, f, n, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, l, f, n, scaling, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    fr, nr = shard.shard(l, f, n, rank, world, scaling)
    w = oracle.sieve(l, fr, nr, nthreads=1)
    total = shard.total_count(oracle.popcount(w))
    tables = [None] * world
    dist.all_gather_object(tables, (fr, w.tobytes()))
    if rank == 0:
        q.put((total, tables))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("scaling", ["weak", "strong"])
def test_two_gloo_ranks_sum_to_the_whole(scaling):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    l, f, n, world = 11, 5000, 6, 2
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, l, f, n, scaling, q)) for r in range(world)]
    for p in procs:
        p.start()
    total, tables = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    n_all = n * world if scaling == "weak" else n
    whole = oracle.sieve(l, f, n_all)
    assert total == oracle.popcount(whole)
    cat = np.concatenate([np.frombuffer(b, dtype=np.uint32) for _, b in sorted(tables)])
    assert np.array_equal(cat, whole)
