"""Batched and served forms on the GPU, bit-exact against stored oracle values and
against the plain per-interval calls."""
import hashlib
import os
import time

import numpy as np
import pytest

from paper_1111_3297_gb300 import sieve as S
from paper_1111_3297_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_3297_gb300 import build
    build.build_library()
    c = S.sieve_init(0, max_v=1 << 62)
    yield c
    c.close()


class _DevArray:
    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<i4", "data": (ptr, False), "version": 3}


def sha(t):
    return hashlib.sha256(t.cpu().numpy().tobytes()).hexdigest()


def golden_batch():
    rows = []
    with open(os.path.join(GOLDEN, "batch_4096_seed0.txt")) as fh:
        for ln in fh:
            if ln.startswith("#") or not ln.strip():
                continue
            i, j0, nb, cnt, h = ln.split()
            rows.append((int(j0), int(nb), int(cnt), h))
    return rows


def layout(reqs, align_words=1):
    out, off = [], 0
    for j0, nb in reqs:
        out.append((j0, nb, off))
        off += (nb // 32 + align_words - 1) // align_words * align_words
    return out, off


def test_batch_4096_every_request_bit_exact(ctx):
    rows = golden_batch()
    reqs = [(j0, nb) for j0, nb, _, _ in rows]
    assert reqs == workloads.batch_requests(4096, seed=0)
    lay, total = layout(reqs)
    arena = torch.empty(total, dtype=torch.int32, device="cuda")
    counts = torch.empty(len(reqs), dtype=torch.int64, device="cuda")
    for _ in range(2):  # direct launches, then the captured graph
        arena.fill_(-1)
        counts.fill_(-1)
        S.sieve_batch(ctx, lay, arena, counts)
        S.sieve_sync(ctx)
        got = counts.cpu().numpy()
        want = np.array([c for _, _, c, _ in rows])
        bad = np.nonzero(got != want)[0]
        assert len(bad) == 0, "requests with wrong counts: %s" % bad[:10]
    for (j0, nb, off), (_, _, _, h) in zip(lay, rows):
        assert sha(arena[off:off + nb // 32]) == h, (j0, nb)


def test_batch_equals_plain_calls_on_unaligned_offsets(ctx):
    reqs = workloads.batch_requests(96, seed=5)
    lay, total = layout(reqs)
    lay = [(j0, nb, off + 1) for j0, nb, off in lay]  # odd word offsets: no 16-byte alignment
    arena = torch.zeros(total + 1, dtype=torch.int32, device="cuda")
    counts = torch.empty(len(reqs), dtype=torch.int64, device="cuda")
    S.sieve_batch(ctx, lay, arena, counts)
    S.sieve_sync(ctx)
    for (j0, nb, off), c in zip(lay, counts.cpu().tolist()):
        plain = torch.empty(nb // 32, dtype=torch.int32, device="cuda")
        S.sieve_segments(ctx, 5, j0 // 32, nb // 32, plain)
        S.sieve_sync(ctx)
        assert torch.equal(plain, arena[off:off + nb // 32]), (j0, nb)
        assert S.sieve_count(ctx, plain, nb) == c


def test_batch_autotune_keeps_bits(ctx):
    reqs = workloads.batch_requests(256, seed=3)
    lay, total = layout(reqs, 4)
    arena = torch.empty(total, dtype=torch.int32, device="cuda")
    counts = torch.empty(len(reqs), dtype=torch.int64, device="cuda")
    S.sieve_batch(ctx, lay, arena, counts)
    S.sieve_sync(ctx)

    def tables():  # the requests' slices only (the padding between them is not output)
        return [sha(arena[o:o + nb // 32]) for _, nb, o in lay]

    ref_counts, ref_sha = counts.clone(), tables()
    t = S.sieve_autotune_batch(ctx, lay, arena, counts)
    assert 16 <= t["tile_log2"] <= 20
    arena.fill_(0)
    counts.fill_(0)
    S.sieve_batch(ctx, lay, arena, counts)
    S.sieve_sync(ctx)
    assert torch.equal(counts, ref_counts) and tables() == ref_sha


def test_serving_results_equal_alone_and_in_the_mix(ctx):
    rng = workloads.SplitMix64(77)
    reqs = [r for r in workloads.batch_requests(400, seed=9) if r[1] <= (1 << 22)][:160]
    srv = S.Server(ctx, mem_cap=4 << 30, max_inflight=4)
    try:
        def table(res):
            return torch.as_tensor(_DevArray(res["dev_bits"], res["nbits"] // 32), device="cuda").clone()

        alone = {}
        for j0, nb in reqs[:24]:  # one at a time: nothing else on the device
            rid = srv.submit(j0, nb)
            got = []
            while not got:
                got = srv.poll(8, timeout_ms=2000)
            assert len(got) == 1 and got[0]["id"] == rid and got[0]["status"] == 0
            alone[(j0, nb)] = (got[0]["composites"], sha(table(got[0])))
            srv.release(rid)
        # the same requests again, inside a stream of others arriving meanwhile
        order = list(range(len(reqs)))
        for i in range(len(order) - 1, 0, -1):
            k = rng.below(i + 1)
            order[i], order[k] = order[k], order[i]
        ids = {}
        for i in order:
            ids[srv.submit(*reqs[i])] = reqs[i]
            if rng.below(4) == 0:
                time.sleep(0.0005)
        results = {}
        deadline = time.time() + 120
        while len(results) < len(ids) and time.time() < deadline:
            for r in srv.poll(256, timeout_ms=100):
                assert r["status"] == 0
                results[r["id"]] = (r["composites"], sha(table(r)))
                srv.release(r["id"])
        assert len(results) == len(ids)
        for rid, key in ids.items():
            if key in alone:
                assert results[rid] == alone[key], key
        # and every served result equals the plain call
        for rid, (j0, nb) in list(ids.items())[:40]:
            plain = torch.empty(nb // 32, dtype=torch.int32, device="cuda")
            S.sieve_segments(ctx, 5, j0 // 32, nb // 32, plain)
            S.sieve_sync(ctx)
            assert results[rid][1] == sha(plain)
    finally:
        srv.close()


def test_server_destroy_returns_when_held_tables_block_the_queue(ctx):
    """A served result that is never released keeps its table in the arena.  A queued
    request that cannot fit beside it must not hold sieve_server_destroy forever: it
    ends with SIEVE_EBUSY and destroy returns."""
    srv = S.Server(ctx, mem_cap=256 << 20, max_inflight=2)  # 256 MiB for tables and buckets
    try:
        nb = 1 << 30  # 128 MiB of table each
        first = srv.submit(1 << 40, nb)
        got, deadline = [], time.time() + 120
        while not got and time.time() < deadline:
            got = srv.poll(8, timeout_ms=500)
        assert len(got) == 1 and got[0]["id"] == first and got[0]["status"] == 0
        srv.submit((1 << 40) + nb, nb)  # does not fit while the first table is held
        time.sleep(0.2)
        assert srv.poll(8) == []
    finally:
        t0 = time.time()
        srv.close()
        assert time.time() - t0 < 60


def test_batch_with_epochs_longer_than_2p32_bits(ctx):
    """Two long requests through the multi-request scatter with epochs of 8192 tiles of
    2^20 bits (2^33 bits): the next hits carried between its groups are 32-bit offsets,
    so there it must recompute first hits per group instead; the tables must equal the
    single-interval path bit for bit and Miller-Rabin on sampled bits."""
    import oracle
    saved = [S.sieve_get_tuning(ctx, k) for k in range(4)]
    try:
        for k in range(4):
            S.sieve_set_tuning(ctx, k, tile_log2=20, presieve_groups=2, coop_max=4096,
                               medium_max=1 << 20, window_tiles=1024, epoch_tiles=8192)
        nb = 1 << 33
        reqs = [(2 ** 46, nb), (3 * 2 ** 47 + (1 << 20), nb)]
        lay, off = layout(reqs, 4)
        arena = torch.empty(off, dtype=torch.int32, device="cuda")
        counts = torch.empty(len(reqs), dtype=torch.int64, device="cuda")
        S.sieve_batch(ctx, lay, arena, counts)
        S.sieve_sync(ctx)
        rng = workloads.SplitMix64(46)
        for (j0, n, o), c in zip(lay, counts.cpu().tolist()):
            plain = torch.empty(n // 32, dtype=torch.int32, device="cuda")
            S.sieve_segments(ctx, 5, j0 // 32, n // 32, plain)
            S.sieve_sync(ctx)
            got = arena[o:o + n // 32]
            assert torch.equal(got, plain), "request at j0=%d differs from the single-interval path" % j0
            assert c == S.sieve_count(ctx, plain, n)
            for _ in range(400):
                j = rng.below(n)
                word = int(got[j // 32].item()) & 0xFFFFFFFF
                assert ((word >> (j % 32)) & 1) == (0 if oracle.is_prime_mr(2 * (j0 + j) + 1) else 1), (j0, j)
            del plain
    finally:
        for k in range(4):
            S.sieve_set_tuning(ctx, k, **saved[k])


def test_server_lane_pool_smaller_than_one_tile_bucket(ctx):
    """Server lanes of a 256 MiB cap shared by 16 hold 2^19 bucket slots per pool.  With
    every prime above the pre-sieve taken as large (medium_max 0), one 2^20-bit tile
    near 2^62 expects about 7.4e5 large-prime hits, more than the pool, so the planner
    clamps its bucket to the pool and the rest goes through the backstop list.  The
    served table must equal the plain call (whose small tiles need no clamp) bit for
    bit, and Miller-Rabin on sampled bits."""
    import oracle
    saved = [S.sieve_get_tuning(ctx, k) for k in range(4)]
    srv = None
    try:
        for k in range(4):
            S.sieve_set_tuning(ctx, k, tile_log2=20, presieve_groups=2, coop_max=4096, medium_max=0,
                               window_tiles=1024, epoch_tiles=4096)
        nb = 1 << 21
        j0 = (1 << 61) - (1 << 22)
        srv = S.Server(ctx, mem_cap=256 << 20, max_inflight=16)
        rid = srv.submit(j0, nb)
        got, deadline = [], time.time() + 120
        while not got and time.time() < deadline:
            got = srv.poll(8, timeout_ms=1000)
        assert len(got) == 1 and got[0]["id"] == rid and got[0]["status"] == 0
        served = torch.as_tensor(_DevArray(got[0]["dev_bits"], nb // 32), device="cuda").clone()
        composites = got[0]["composites"]
        srv.release(rid)
        plain = torch.empty(nb // 32, dtype=torch.int32, device="cuda")
        S.sieve_segments(ctx, 5, j0 // 32, nb // 32, plain)
        S.sieve_sync(ctx)
        assert torch.equal(served, plain)
        assert composites == S.sieve_count(ctx, plain, nb)
        rng = workloads.SplitMix64(62)
        host = served.cpu().numpy().view(np.uint32)
        for _ in range(300):
            j = rng.below(nb)
            bit = (int(host[j // 32]) >> (j % 32)) & 1
            assert bit == (0 if oracle.is_prime_mr(2 * (j0 + j) + 1) else 1), j
    finally:
        if srv is not None:
            srv.close()
        for k in range(4):
            S.sieve_set_tuning(ctx, k, **saved[k])


def test_server_admits_by_table_and_bucket_memory(ctx):
    """Tables and bucket pools share the server's one arena.  A request whose table fits
    but whose table and smallest bucket pools do not is refused at submission; requests
    whose tables and buckets cannot all be resident at once wait, are admitted as
    batches finish and tables are released, and each equals the plain call."""
    cap = 512 << 20
    srv = S.Server(ctx, mem_cap=cap, max_inflight=4)
    try:
        with pytest.raises(S.SieveError):
            srv.submit(1 << 40, (cap - 20000) * 8 // 32 * 32)  # table < arena < table + buckets
        nb = 3 << 28  # 96 MiB of table each: five fill the arena
        f = S.sieve_f_from_midpoint(5, nb // 32 * 8, 1, 15)
        reqs = [((f << 5) + k * nb, nb) for k in range(8)]
        ids = {srv.submit(j0, n): (j0, n) for j0, n in reqs}
        results, deadline = {}, time.time() + 180
        while len(results) < len(ids) and time.time() < deadline:
            for r in srv.poll(8, timeout_ms=200):
                assert r["status"] == 0
                results[r["id"]] = (r["composites"], sha(torch.as_tensor(
                    _DevArray(r["dev_bits"], r["nbits"] // 32), device="cuda")))
                srv.release(r["id"])
        assert len(results) == len(ids)
    finally:
        srv.close()
    for rid, (j0, n) in ids.items():
        plain = torch.empty(n // 32, dtype=torch.int32, device="cuda")
        S.sieve_segments(ctx, 5, j0 // 32, n // 32, plain)
        S.sieve_sync(ctx)
        assert results[rid] == (S.sieve_count(ctx, plain, n), sha(plain)), j0
        del plain
