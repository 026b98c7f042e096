"""Each large-prime hit is emitted exactly once (Theorem thm:big, Cor. cor:complete,
Sec. 2.3), checked on the device's own counter.

OR is idempotent, so a hit emitted twice leaves the table unchanged: only the count
of bucket entries shows it (and a duplicate would cost scatter time and inflate the
hit count the roofline uses).  With profiling on, the library sums the per-tile
bucket counters after every scatter launch; that sum must equal, exactly, the
oracle's closed-form count of the odd multiples p*c (c coprime to the plan's
wheel modulus) of every large prime p in [max(u, p^2), v-1].  The large primes and
the wheel are those of the plan the call runs, read from sieve_plan_describe.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1111_3297_gb300 import sieve as S
from paper_1111_3297_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_V = 2 * 10**18


class _DevArray:
    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<i4", "data": (ptr, False),
                                         "version": 3}


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_3297_gb300 import build
    build.build_library()
    c = S.sieve_init(0, max_v=MAX_V)
    ptr, cnt, lim = S.sieve_base_info(c)
    primes = torch.as_tensor(_DevArray(ptr, cnt), device="cuda").cpu().numpy().view(np.uint32).copy()
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    yield c, primes, nsm
    c.close()


def tune_class(vlast):
    lg = vlast.bit_length() - 1
    return 0 if lg < 40 else 1 if lg < 50 else 2 if lg < 56 else 3


def interval_tuning(ctx, nsm, vlast, nbits):
    """The tuning sieve_segments takes for one interval: the class tuning, with smaller
    tiles while the interval has fewer than 4 tiles per SM (down to 2^14)."""
    t = S.sieve_get_tuning(ctx, tune_class(vlast))
    while t["tile_log2"] > 14 and (nbits >> t["tile_log2"]) < 4 * nsm:
        t["tile_log2"] -= 1
        if t["coop_max"] > 64:
            t["coop_max"] >>= 1
    return t


def expected_hits(primes, reqs, tuning, nsm):
    plan = S.sieve_plan_describe(primes, MAX_V, nsm, reqs, tuning=tuning, records=False)["info"]
    W = 15015 if plan["big_wheel"] else 15
    lo = plan["large_lo"]
    total = 0
    for j0, nbits, _ in reqs:
        plimit = math.isqrt(2 * (j0 + nbits - 1) + 1)
        hi = int(np.searchsorted(primes, plimit, side="right"))
        if hi > lo:
            total += oracle.large_prime_hits(j0, nbits, primes[lo:hi], W)
    return total, plan


def device_hits(ctx, run):
    S.sieve_profile_enable(ctx, True)
    S.sieve_profile_read(ctx)
    try:
        run()
        prof = S.sieve_profile_read(ctx)
    finally:
        S.sieve_profile_enable(ctx, False)
    S.sieve_sync(ctx)
    return prof["large_hits"]


INTERVALS = [
    # (l, midpoint mantissa, exp10, n, tuning override or None)
    (20, 1, 13, 640, None),                 # 1e13: one scatter group per 1024 tiles
    (16, 1, 17, 1001, None),                # 1e17: ragged last tile of 2^20 bits
    (14, 1 << 60, 0, 300, dict(tile_log2=14, presieve_groups=1, coop_max=256, medium_max=1 << 13,
                               window_tiles=8, epoch_tiles=32)),  # 2^60: 38 groups, 10 epochs
    (15, 3, 11, 777, dict(tile_log2=14, presieve_groups=3, coop_max=512, medium_max=1 << 12,
                          window_tiles=3, epoch_tiles=7)),       # small primes in the buckets
]


@pytest.mark.parametrize("l,mant,exp10,n,tune", INTERVALS)
def test_interval_hits_equal_closed_form(env, l, mant, exp10, n, tune):
    ctx, primes, nsm = env
    f = S.sieve_f_from_midpoint(l, n, mant, exp10)
    j0, nbits = f << l, n << l
    vlast = 2 * (j0 + nbits - 1) + 1
    cls = tune_class(vlast)
    saved = S.sieve_get_tuning(ctx, cls)
    try:
        if tune:
            S.sieve_set_tuning(ctx, cls, **tune)
        t = interval_tuning(ctx, nsm, vlast, nbits)
        want, plan = expected_hits(primes, [(j0, nbits, 0)], t, nsm)
        assert want > 0
        out = torch.empty(nbits // 32, dtype=torch.int32, device="cuda")
        got = device_hits(ctx, lambda: S.sieve_segments(ctx, l, f, n, out))
        assert got == want, (got, want, plan)
        # the table itself against the oracle on its first and last 2^16 bits
        k = min(nbits, 1 << 16) // 32
        host = out.cpu().numpy().view(np.uint32)
        base = oracle.base_for(vlast)
        assert np.array_equal(host[:k], oracle.sieve_range(j0, 32 * k, base=base))
        assert np.array_equal(host[-k:], oracle.sieve_range(j0 + nbits - 32 * k, 32 * k, base=base))
    finally:
        S.sieve_set_tuning(ctx, cls, **saved)


def test_batch_hits_equal_closed_form(env):
    ctx, primes, nsm = env
    reqs = workloads.batch_requests(64, seed=11)
    lay, off = [], 0
    for j0, nb in reqs:
        lay.append((j0, nb, off))
        off += (nb // 32 + 3) // 4 * 4
    vmax = max(2 * (j0 + nb - 1) + 1 for j0, nb in reqs)
    t = S.sieve_get_tuning(ctx, tune_class(vmax))
    want, plan = expected_hits(primes, lay, t, nsm)
    assert want > 0
    arena = torch.empty(off, dtype=torch.int32, device="cuda")
    counts = torch.empty(len(reqs), dtype=torch.int64, device="cuda")
    got = device_hits(ctx, lambda: S.sieve_batch(ctx, lay, arena, counts))
    assert got == want, (got, want, plan)


@pytest.mark.parametrize("l,mant,exp10,n,tune", INTERVALS[:3])
def test_state_writes_follow_the_plan(env, l, mant, exp10, n, tune):
    """The state-word count behind the scatter's byte figure: one 8-byte word written back
    per large prime and scatter group, except in the interval's last group, and in every
    group once the interval is streamed (its successor reads the last group's words)."""
    ctx, primes, nsm = env
    f = S.sieve_f_from_midpoint(l, n, mant, exp10)
    j0, nbits = f << l, n << l
    vlast = 2 * (j0 + nbits - 1) + 1
    cls = tune_class(vlast)
    saved = S.sieve_get_tuning(ctx, cls)
    try:
        if tune:
            S.sieve_set_tuning(ctx, cls, **tune)
        t = interval_tuning(ctx, nsm, vlast, nbits)
        plan = S.sieve_plan_describe(primes, MAX_V, nsm, [(j0, nbits, 0)], tuning=t)
        assert plan["info"]["run_scatter"] == 1
        per_group = [g["p_hi"] - g["p_lo"] for g in plan["groups"]]
        out = torch.empty(nbits // 32, dtype=torch.int32, device="cuda")
        for streamed in (False, True):
            S.sieve_set_streaming(ctx, streamed)
            S.sieve_profile_enable(ctx, True)
            S.sieve_profile_read(ctx)
            S.sieve_segments(ctx, l, f, n, out)
            prof = S.sieve_profile_read(ctx)
            S.sieve_profile_enable(ctx, False)
            S.sieve_sync(ctx)
            assert prof["prime_reads"] == sum(per_group)
            want = sum(per_group) if streamed else sum(per_group[:-1])
            assert prof["state_writes"] == want, (streamed, prof["state_writes"], want, len(per_group))
    finally:
        S.sieve_set_streaming(ctx, False)
        S.sieve_set_tuning(ctx, cls, **saved)
