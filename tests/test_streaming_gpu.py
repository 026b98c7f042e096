"""Streaming (sieve_set_streaming): consecutive single-interval calls continue from each
other's large-prime state (Sec. 2.3-2.4: segments in order, each large prime's next hit
carried along) and give the same bits as separate calls.  Each continued call is checked
bit for bit against the oracle and, with profiling on, its device hit count against the
closed form (a prime continued from a stale or shifted state word would drop or repeat
hits)."""
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
    ptr, cnt, _ = S.sieve_base_info(c)
    primes = torch.as_tensor(_DevArray(ptr, cnt), device="cuda").cpu().numpy().view(np.uint32).copy()
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    yield c, primes, nsm
    S.sieve_set_streaming(c, False)
    c.close()


def tune_class(vlast):
    lg = vlast.bit_length() - 1
    return 0 if lg < 40 else 1 if lg < 50 else 2 if lg < 56 else 3


def expected_hits(ctx, primes, nsm, j0, nbits):
    vlast = 2 * (j0 + nbits - 1) + 1
    t = S.sieve_get_tuning(ctx, tune_class(vlast))
    while t["tile_log2"] > 14 and (nbits >> t["tile_log2"]) < 4 * nsm:
        t["tile_log2"] -= 1
        if t["coop_max"] > 64:
            t["coop_max"] >>= 1
    plan = S.sieve_plan_describe(primes, MAX_V, nsm, [(j0, nbits, 0)], tuning=t, records=False)["info"]
    hi = int(np.searchsorted(primes, math.isqrt(vlast), side="right"))
    W = 15015 if plan["big_wheel"] else 15
    return oracle.large_prime_hits(j0, nbits, primes[plan["large_lo"]:hi], W) if hi > plan["large_lo"] else 0


def run(ctx, l, f, n, prof=False):
    """The table, and with prof (large-prime hits, primes continued from state)."""
    out = torch.empty((n << l) // 32, dtype=torch.int32, device="cuda")
    if prof:
        S.sieve_profile_enable(ctx, True)
        S.sieve_profile_read(ctx)
    S.sieve_segments(ctx, l, f, n, out)
    hits = None
    if prof:
        pr = S.sieve_profile_read(ctx)
        hits = (pr["large_hits"], pr["continued"])
        S.sieve_profile_enable(ctx, False)
    S.sieve_sync(ctx)
    return out.cpu().numpy().view(np.uint32), hits


def check_stream(env, pieces, tune=None):
    """pieces: consecutive (l, n) with the first one's f; every call checked."""
    ctx, primes, nsm = env
    saved = [S.sieve_get_tuning(ctx, k) for k in range(4)]
    try:
        if tune:
            for k in range(4):
                S.sieve_set_tuning(ctx, k, **tune)
        S.sieve_set_streaming(ctx, True)
        J = None
        continued = 0
        for l, n, f0 in pieces:
            f = f0 if J is None else J >> l
            assert J is None or (f << l) == J
            got, (hits, cont) = run(ctx, l, f, n, prof=True)
            want = oracle.sieve(l, f, n)
            assert np.array_equal(got, want), (l, f, n)
            assert hits == expected_hits(ctx, primes, nsm, f << l, n << l), (l, f, n)
            if J is None:
                assert cont == 0
            continued += cont
            J = (f + n) << l
        assert continued > 0  # the later intervals did continue (where plans allowed it)
    finally:
        S.sieve_set_streaming(ctx, False)
        for k in range(4):
            S.sieve_set_tuning(ctx, k, **saved[k])


def test_consecutive_intervals_near_1e17(env):
    f0 = S.sieve_f_from_midpoint(20, 64, 1, 17)
    check_stream(env, [(20, 64, f0), (20, 64, None), (20, 64, None), (20, 64, None)])


def test_consecutive_intervals_with_new_primes_and_other_segment_sizes(env):
    # near 1e11 every interval adds large primes (the root grows by ~200 per 2^27 numbers);
    # primes above 2^14 are large here
    tune = dict(tile_log2=16, presieve_groups=2, coop_max=1024, medium_max=1 << 14, window_tiles=256,
                epoch_tiles=1024)
    f0 = S.sieve_f_from_midpoint(16, 1024, 1, 11) // 16 * 16  # 2^20-aligned: the l=20 piece follows
    check_stream(env, [(16, 1024, f0), (20, 64, None), (18, 300, None), (16, 1000, None)], tune)


def test_consecutive_intervals_many_groups_at_2p60(env):
    tune = dict(tile_log2=14, presieve_groups=1, coop_max=256, medium_max=1 << 13, window_tiles=8, epoch_tiles=32)
    f0 = S.sieve_f_from_midpoint(14, 300, 1 << 60, 0)
    check_stream(env, [(14, 300, f0), (14, 300, None), (14, 77, None)], tune)


def test_other_work_between_intervals_ends_the_continuation(env):
    ctx, primes, nsm = env
    l, n = 20, 64
    f = S.sieve_f_from_midpoint(l, n, 1, 16)
    S.sieve_set_streaming(ctx, True)
    try:
        run(ctx, l, f, n)
        # a batch on the same context overwrites the state words
        reqs = workloads.batch_requests(16, seed=4)
        lay, off = [], 0
        for j0, nb in reqs:
            lay.append((j0, nb, off))
            off += (nb // 32 + 3) // 4 * 4
        arena = torch.empty(off, dtype=torch.int32, device="cuda")
        counts = torch.empty(len(reqs), dtype=torch.int64, device="cuda")
        S.sieve_batch(ctx, lay, arena, counts)
        got, (hits, cont) = run(ctx, l, f + n, n, prof=True)
        assert np.array_equal(got, oracle.sieve(l, f + n, n))
        assert hits == expected_hits(ctx, primes, nsm, (f + n) << l, n << l)
        assert cont == 0  # the batch ended the continuation
        # and an interval elsewhere, then the continuation of that one
        got, _ = run(ctx, l, f + 10 * n, n)
        got, (hits, cont) = run(ctx, l, f + 11 * n, n, prof=True)
        assert np.array_equal(got, oracle.sieve(l, f + 11 * n, n))
        assert cont > 0 and hits == expected_hits(ctx, primes, nsm, (f + 11 * n) << l, n << l)
    finally:
        S.sieve_set_streaming(ctx, False)


def test_host_output_and_count_only_continue_too(env):
    ctx, _, _ = env
    l, n = 20, 48
    f = S.sieve_f_from_midpoint(l, n, 3, 15)
    S.sieve_set_streaming(ctx, True)
    try:
        host = torch.empty((n << l) // 32, dtype=torch.int32).pin_memory()
        S.sieve_segments_host(ctx, l, f, n, host)
        assert np.array_equal(host.numpy().view(np.uint32), oracle.sieve(l, f, n))
        S.sieve_segments_host(ctx, l, f + n, n, host)
        assert np.array_equal(host.numpy().view(np.uint32), oracle.sieve(l, f + n, n))
        pr = torch.empty(n, dtype=torch.int64, device="cuda")
        tw = torch.empty(n, dtype=torch.int64, device="cuda")
        S.sieve_count_segments(ctx, l, f + 2 * n, n, pr, tw)
        S.sieve_sync(ctx)
        want_p, want_t = oracle.segment_counts(oracle.sieve(l, f + 2 * n, n), (f + 2 * n) << l, n << l, l)
        assert np.array_equal(pr.cpu().numpy(), want_p) and np.array_equal(tw.cpu().numpy(), want_t)
    finally:
        S.sieve_set_streaming(ctx, False)
