"""The planner (host code of the C ABI library) checked on the CPU through
sieve_plan_describe, no device needed.

The plan is the work decomposition of Sec. 1.3 (the table cut into segments,
here "tiles" of 2^tile_log2 bits) and Sec. 2.2 (large primes, whose stride
exceeds a segment, routed into per-segment buckets).  These tests check what
any correct decomposition must satisfy.
  * Tiles partition every request exactly.
  * Each tile's outputs land at its own words.
  * Buckets stay inside their epoch's pool, even when one tile would want more.
  * Scatter groups and chunks cover the primes each tile needs: the large primes
    up to isqrt of the request's last number, by Definition "base" and the note
    of Sec. 1.4 that only primes <= sqrt(v) are needed.
"""
import math
import os

import numpy as np
import pytest

from paper_1111_3297_gb300 import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def S():
    import shutil
    from paper_1111_3297_gb300 import build, sieve
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc") \
            and not os.path.exists(build.LIB):
        pytest.skip("no nvcc to build the library")
    build.build_library()
    return sieve


def odd_primes_upto(x):
    s = np.ones(x // 2 + 1, dtype=bool)
    s[0] = False
    for i in range(1, (math.isqrt(x) + 1) // 2 + 1):
        if s[i]:
            p = 2 * i + 1
            s[p * p // 2::p] = False
    p = 2 * np.nonzero(s)[0] + 1
    return p[p <= x].astype(np.uint32)


MAX_V = 10**16
PRIMES = odd_primes_upto(math.isqrt(MAX_V))
PRIMES64 = PRIMES.astype(np.int64)  # searched with int64 keys (no per-call array conversion)


def test_prime_table_of_the_test():
    # pi(10^8) = 5761455 (2 excluded here)
    assert len(PRIMES) == 5761455 - 1
    assert PRIMES[0] == 3 and PRIMES[-1] == 99999989


TUNE = dict(tile_log2=16, presieve_groups=2, coop_max=2048, medium_max=1 << 17, window_tiles=64,
            epoch_tiles=256)


def count_le(x):
    return int(np.searchsorted(PRIMES64, np.int64(x), side="right"))


def check_plan(plan, reqs, tune, pool_entries):
    info, tiles, groups, chunks = plan["info"], plan["tiles"], plan["groups"], plan["chunks"]
    B = 1 << tune["tile_log2"]
    assert info["ntiles"] == len(tiles) == sum(-(-nb // B) for _, nb, _ in reqs)
    assert info["bits"] == sum(nb for _, nb, _ in reqs)
    med_lo = info["med_lo"]
    large_lo = max(med_lo, count_le(tune["medium_max"]))
    assert info["large_lo"] == large_lo
    assert info["coop_hi"] == max(med_lo, count_le(tune["coop_max"]))
    assert med_lo <= info["blk_hi"] <= info["coop_hi"]
    # tiles partition each request, outputs at the request's own words
    by_req = {}
    for t in tiles:
        by_req.setdefault(t["req"], []).append(t)
    assert sorted(by_req) == list(range(len(reqs)))
    for r, (j0, nb, ow) in enumerate(reqs):
        ts = sorted(by_req[r], key=lambda t: t["j0"])
        pos = j0
        for t in ts:
            assert t["j0"] == pos and 0 < t["len"] <= B and t["len"] % 32 == 0
            assert t["out_word"] == ow + (t["j0"] - j0) // 32
            pos += t["len"]
        assert pos == j0 + nb
        vlast = 2 * (j0 + nb - 1) + 1
        plim = math.isqrt(vlast)
        for t in ts:
            assert t["med_hi"] == max(med_lo, count_le(min(tune["medium_max"], plim)))
            needs_large = count_le(plim) > large_lo
            assert (t["bkt_cap"] > 0) == needs_large
            assert (t["group"] != 0xFFFFFFFF) == needs_large
    # epochs: consecutive tiles, at most epoch_tiles each, buckets disjoint inside the pool
    assert info["pool_entries"] <= pool_entries
    ep_tiles = {}
    for i, t in enumerate(tiles):
        ep_tiles.setdefault(t["epoch"], []).append(i)
    assert sorted(ep_tiles) == list(range(info["nepochs"]))
    for e, idx in ep_tiles.items():
        assert idx == list(range(idx[0], idx[0] + len(idx)))
        assert len(idx) <= max(tune["epoch_tiles"], 1) and len(idx) <= info["max_epoch_tiles"]
        spans = sorted((tiles[i]["bkt_off"], tiles[i]["bkt_cap"]) for i in idx if tiles[i]["bkt_cap"])
        end = 0
        for off, cap in spans:
            assert off % 4 == 0 and cap % 4 == 0
            assert off >= end
            end = off + cap
        assert end <= info["pool_entries"]
    # groups: at most window_tiles tiles of one epoch, primes up to the largest plimit
    for gi, g in enumerate(groups):
        assert 0 < g["ntiles"] <= tune["window_tiles"] and g["nunits"] >= 1
        members = range(g["tile0"], g["tile0"] + g["ntiles"])
        assert all(tiles[i]["epoch"] == g["epoch"] for i in members)
        assert all(tiles[i]["group"] == gi for i in members if tiles[i]["bkt_cap"])
        assert g["p_lo"] == large_lo
        need = max(count_le(math.isqrt(2 * (reqs[tiles[i]["req"]][0] + reqs[tiles[i]["req"]][1] - 1) + 1))
                   for i in members)
        assert g["p_hi"] == need
        if g["carry_in"]:
            prev = groups[gi - 1]
            assert prev["carry_out"] and prev["epoch"] == g["epoch"]
            assert (prev["p_lo"], prev["p_hi"]) == (g["p_lo"], g["p_hi"])
    for i, t in enumerate(tiles):
        if t["group"] != 0xFFFFFFFF:
            g = groups[t["group"]]
            assert g["tile0"] <= i < g["tile0"] + g["ntiles"]
    # chunks of an epoch: consecutive, covering every group's primes of that epoch
    for e in range(info["nepochs"]):
        cs = [c for c in chunks if c["epoch"] == e]
        gs = [g for g in groups if g["epoch"] == e]
        if not gs:
            assert not cs
            continue
        lo, hi = min(g["p_lo"] for g in gs), max(g["p_hi"] for g in gs)
        assert cs[0]["p_lo"] == lo and cs[-1]["p_hi"] == hi
        for a, b in zip(cs, cs[1:]):
            assert a["p_hi"] == b["p_lo"]
        for c in cs:
            assert c["p_lo"] < c["p_hi"]
            assert c["p_hi"] == hi or (c["p_hi"] - c["p_lo"]) % 32 == 0


def test_single_interval_plan(S):
    # 2^26 bits around 1e15 (1024 tiles of 2^16 bits)
    f = (10**15 >> 17) - 512
    reqs = [(f << 16, 1 << 26, 0)]
    plan = S.sieve_plan_describe(PRIMES, MAX_V, 152, reqs, TUNE)
    check_plan(plan, reqs, TUNE, 1 << 31)
    info = plan["info"]
    assert info["run_scatter"] == 1
    assert info["nunits"] == info["ngroups"] == 1024 // 64 and info["nepochs"] == 1024 // 256
    # expected large-prime hits: bits x wheel density x sum of 1/p over the large primes
    plim = math.isqrt(2 * (f << 16) + 2 * (1 << 26))
    large = PRIMES[(PRIMES > TUNE["medium_max"]) & (PRIMES <= plim)].astype(np.float64)
    dens = 5760 / 15015 if info["big_wheel"] else 8 / 15
    want = (1 << 26) * dens * float(np.sum(1.0 / large))
    assert abs(info["expected_large_hits"] - want) <= 0.01 * want


def test_plan_is_deterministic(S):
    reqs = [(1 << 40, 3 << 20, 0), (1 << 36, 1 << 20, 3 << 15)]
    a = S.sieve_plan_describe(PRIMES, MAX_V, 152, reqs, TUNE)
    b = S.sieve_plan_describe(PRIMES, MAX_V, 152, reqs, TUNE)
    assert a == b


def test_batch_plan_of_mixed_requests(S):
    # 300 requests of the batch generator's shape (1e6..1e16 here), ragged lengths
    rng = np.random.default_rng(5)
    reqs, off = [], 0
    for _ in range(300):
        mag = 10 ** rng.uniform(6, 15.9)
        nb = int(rng.integers(1, 2048)) * 32
        j0 = (int(mag) // 2) // 32 * 32
        reqs.append((j0, nb, off))
        off += nb // 32
    plan = S.sieve_plan_describe(PRIMES, MAX_V, 152, reqs, TUNE)
    check_plan(plan, reqs, TUNE, 1 << 31)
    assert plan["info"]["run_scatter"] == 0


def test_stored_batch_requests_plan(S):
    reqs = workloads.batch_requests(256, seed=0)
    lay, off = [], 0
    for j0, nb in reqs:
        if 2 * (j0 + nb) > MAX_V:
            continue
        lay.append((j0, nb, off))
        off += (nb // 32 + 3) // 4 * 4
    assert len(lay) > 50
    t = dict(TUNE, tile_log2=18, window_tiles=256, epoch_tiles=1024)
    check_plan(S.sieve_plan_describe(PRIMES, MAX_V, 152, lay, t), lay, t, 1 << 31)


def test_long_request_groups_carry_state(S):
    # one request of 40 groups plus a small one: the batch planner carries each large
    # prime's next hit from a group to the next inside an epoch (<= 2^32 bits)
    reqs = [(1 << 44, 40 * 64 << 16, 0), (1 << 30, 1 << 16, 40 * 64 << 11)]
    plan = S.sieve_plan_describe(PRIMES, MAX_V, 152, reqs, TUNE)
    check_plan(plan, reqs, TUNE, 1 << 31)
    assert plan["info"]["carried_groups"] > 0


def test_bucket_capacity_never_exceeds_a_small_pool(S):
    # a pool smaller than one tile's expected hits: every bucket is clamped to the
    # pool (the rest spills to the backstop list on the device) and buckets of one
    # epoch never overlap or leave the pool
    f = (10**15 >> 17) - 512
    reqs = [(f << 16, 1 << 24, 0)]
    t = dict(TUNE, medium_max=1 << 12)
    full = S.sieve_plan_describe(PRIMES, MAX_V, 152, reqs, t)
    assert max(x["bkt_cap"] for x in full["tiles"]) > 4096
    plan = S.sieve_plan_describe(PRIMES, MAX_V, 152, reqs, t, pool_entries=4096)
    check_plan(plan, reqs, t, 4096)
    assert max(x["bkt_cap"] for x in plan["tiles"]) == 4096
    assert plan["info"]["nepochs"] == len(plan["tiles"])


def test_phase_bounds_follow_the_tuning(S):
    reqs = [(1 << 40, 1 << 22, 0)]
    for t in (TUNE, dict(TUNE, presieve_groups=5, coop_max=1 << 14, medium_max=1 << 20, tile_log2=20,
                         window_tiles=16, epoch_tiles=16)):
        check_plan(S.sieve_plan_describe(PRIMES, MAX_V, 152, reqs, t), reqs, t, 1 << 31)


def test_rejects_bad_arguments(S):
    ok = [(1 << 40, 1 << 20, 0)]
    with pytest.raises(S.SieveError) as e:
        S.sieve_plan_describe(PRIMES[::-1], MAX_V, 152, ok, TUNE, records=False)
    assert e.value.status == 1
    with pytest.raises(S.SieveError):
        S.sieve_plan_describe(np.array([3, 4, 5], dtype=np.uint32), MAX_V, 152, ok, TUNE, records=False)
    with pytest.raises(S.SieveError):
        S.sieve_plan_describe(PRIMES, MAX_V, 152, ok, TUNE, pool_entries=4095, records=False)
    with pytest.raises(S.SieveError):
        S.sieve_plan_describe(PRIMES, MAX_V, 0, ok, TUNE, records=False)
    with pytest.raises(S.SieveError):
        S.sieve_plan_describe(PRIMES, MAX_V, 152, [(1 << 40, 100, 0)], TUNE, records=False)
    with pytest.raises(S.SieveError):
        S.sieve_plan_describe(PRIMES, MAX_V, 152, ok, dict(TUNE, tile_log2=22), records=False)
    with pytest.raises(S.SieveError) as e:
        S.sieve_plan_describe(PRIMES, MAX_V, 152, [(MAX_V, 1 << 20, 0)], TUNE, records=False)
    assert e.value.status == 2
    assert S.sieve_plan_describe(PRIMES, MAX_V, 152, [], TUNE)["info"]["ntiles"] == 0


def test_short_intervals_get_smaller_tiles_without_a_tuning(S):
    # sieve_segments' rule on a fresh context: halve the tile (down to 2^14 bits) while
    # the interval has fewer than 4 tiles per SM
    nsm = 152
    for nbits in (1 << 20, 1 << 26, 1 << 30, 1 << 31):
        info = S.sieve_plan_describe(PRIMES, MAX_V, nsm, [(1 << 40, nbits, 0)], None, records=False)["info"]
        tiles = info["ntiles"]
        bt = (nbits // tiles).bit_length() - 1
        assert nbits == tiles << bt
        assert bt == 14 or tiles >= 4 * nsm
        assert bt == 20 or (nbits >> (bt + 1)) < 4 * nsm


def test_plans_beyond_32_bit_tile_indices_are_refused(S):
    # 2^43 bits in 2^12-bit tiles = 2^31 tiles: refused before anything is allocated
    t = dict(TUNE, tile_log2=12)
    with pytest.raises(S.SieveError) as e:
        S.sieve_plan_describe(PRIMES, MAX_V, 152, [(0, 1 << 43, 0)], t, records=False)
    assert e.value.status == 2


def test_random_plans_keep_the_invariants(S):
    # seeded random batches, tunings and pool sizes: the plan must satisfy every
    # invariant of check_plan whatever the mix
    rng = np.random.default_rng(2024)
    for case in range(40):
        tl = int(rng.integers(12, 21))
        win = int(min(1024, 1 << int(rng.integers(0, 11)), (1 << 30) >> tl))
        t = dict(tile_log2=tl, presieve_groups=int(rng.integers(1, 14)),
                 coop_max=int(1 << int(rng.integers(6, 16))), medium_max=int(1 << int(rng.integers(8, 24))),
                 window_tiles=win, epoch_tiles=int(win * int(rng.integers(1, 9))))
        reqs, off = [], 0
        for _ in range(int(rng.integers(1, 60))):
            mag = 10 ** rng.uniform(2, 15.9)
            nb = int(rng.integers(1, 1 << int(rng.integers(1, 14)))) * 32
            j0 = (int(mag) // 2) // 32 * 32
            reqs.append((j0, nb, off))
            off += nb // 32 + int(rng.integers(0, 3))
        pool = int(1 << int(rng.integers(12, 32)))
        plan = S.sieve_plan_describe(PRIMES, MAX_V, int(rng.integers(1, 200)), reqs, t, pool_entries=pool)
        check_plan(plan, reqs, t, pool)


def test_cluster_tiles_for_one_interval_only(S):
    """Tiles of 2^21 bits (two-CTA clusters) are planned for a single interval; a batch
    of several requests takes 2^20-bit tiles under the same tuning."""
    tune = dict(TUNE, tile_log2=21, window_tiles=512, epoch_tiles=1024)
    j0, nbits = 10**12, (700 << 21) + 96
    one = S.sieve_plan_describe(PRIMES, MAX_V, 152, [(j0, nbits, 0)], tune)
    lens = [t["len"] for t in one["tiles"]]
    assert max(lens) == 1 << 21 and sum(lens) == nbits and lens[-1] == 96
    assert all(g["ntiles"] <= 512 for g in one["groups"])
    two = S.sieve_plan_describe(PRIMES, MAX_V, 152, [(j0, nbits, 0), (j0 + nbits, 1 << 22, nbits // 32)], tune)
    assert max(t["len"] for t in two["tiles"]) == 1 << 20
    with pytest.raises(S.SieveError):
        S.sieve_plan_describe(PRIMES, MAX_V, 152, [(j0, nbits, 0)], dict(tune, window_tiles=1024))  # 2^31-bit units
