"""Parity of the CUDA path (through the C ABI) with the CPU oracle, bit for bit.

Small cases are compared with the oracle computed here; the full-size
configurations with stored values written by tests/golden/make_golden.py from the
oracle (SHA-256 of whole tables, per-segment composite counts) and with
deterministic Miller-Rabin on sampled bits.  Integer work: the bar is exact.
"""
import hashlib
import os

import numpy as np
import pytest

import oracle
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


def run_plain(ctx, l, f, n):
    out = torch.empty((n << l) // 32, dtype=torch.int32, device="cuda")
    S.sieve_segments(ctx, l, f, n, out)
    S.sieve_sync(ctx)
    return out


def host_words(t):
    return t.cpu().numpy().view(np.uint32)


def sha(words):
    return hashlib.sha256(np.ascontiguousarray(words, dtype="<u4").tobytes()).hexdigest()


def first_diff(a, b):
    d = np.nonzero(a != b)[0]
    if len(d) == 0:
        return None
    w = int(d[0])
    return "word %d: got %08x want %08x (%d words differ)" % (w, a[w], b[w], len(d))


# ---------------------------------------------------------------------------
class _DevArray:
    """Wraps a device pointer for torch.as_tensor (CUDA array interface, zero copy)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<i4", "data": (ptr, False),
                                         "version": 3}


def test_base_primes_equal_oracle_base():
    c = S.sieve_init(0, max_v=10**16)
    try:
        ptr, cnt, lim = S.sieve_base_info(c)
        assert lim == 10**8
        got = torch.as_tensor(_DevArray(ptr, cnt), device="cuda").cpu().numpy().view(np.uint32)
        want = oracle.Base(10**8).primes
        assert cnt == len(want)
        assert np.array_equal(got, want)
    finally:
        c.close()


def test_base_count_at_2p31_equals_published_pi(ctx):
    _, cnt, lim = S.sieve_base_info(ctx)
    assert lim == 2**31
    assert cnt + 1 == 105097565  # pi(2^31), OEIS A007053


def test_config1_full_table(ctx):
    got = host_words(run_plain(ctx, 15, 0, 1024))
    want = oracle.sieve(15, 0, 1024)
    assert first_diff(got, want) is None, first_diff(got, want)


@pytest.mark.parametrize("l", [5, 6, 7, 9, 12, 16])
@pytest.mark.parametrize("f", [0, 1, 3, 17, 1000, (1 << 20) + 3])
@pytest.mark.parametrize("n", [1, 2, 7])
def test_tiny_grid(ctx, l, f, n):
    got = host_words(run_plain(ctx, l, f, n))
    want = oracle.sieve(l, f, n)
    assert first_diff(got, want) is None, first_diff(got, want)


# tunings that push work through every path: tiny tiles (many ragged tails),
# large primes through the buckets at low magnitude, all or few pre-sieve groups
TUNINGS = [
    dict(tile_log2=12, presieve_groups=1, coop_max=64, medium_max=1 << 10, window_tiles=64, epoch_tiles=256),
    dict(tile_log2=14, presieve_groups=3, coop_max=1 << 9, medium_max=1 << 12, window_tiles=1024, epoch_tiles=1024),
    dict(tile_log2=16, presieve_groups=13, coop_max=1 << 8, medium_max=1 << 16, window_tiles=512, epoch_tiles=2048),
    dict(tile_log2=18, presieve_groups=6, coop_max=1 << 12, medium_max=1 << 14, window_tiles=16, epoch_tiles=32),
    dict(tile_log2=20, presieve_groups=9, coop_max=1 << 13, medium_max=1 << 21, window_tiles=1024, epoch_tiles=4096),
]


@pytest.mark.parametrize("tune", TUNINGS)
@pytest.mark.parametrize("j0,nbits", [(0, 3 << 20), (10**12 // 2 + 96, (5 << 18) + 224),
                                      (10**15 // 2, 1 << 21), (2**59 + 4096, (1 << 19) + 32)])
def test_tunings_and_ragged_ranges(ctx, tune, j0, nbits):
    saved = [S.sieve_get_tuning(ctx, k) for k in range(4)]
    try:
        for k in range(4):
            S.sieve_set_tuning(ctx, k, **tune)
        out = torch.empty(nbits // 32, dtype=torch.int32, device="cuda")
        # a range given as l=5 segments: f = j0/32, n = nbits/32
        S.sieve_segments(ctx, 5, j0 // 32, nbits // 32, out)
        S.sieve_sync(ctx)
        got = host_words(out)
        want = oracle.sieve_range(j0, nbits)
        assert first_diff(got, want) is None, first_diff(got, want)
    finally:
        for k in range(4):
            S.sieve_set_tuning(ctx, k, **saved[k])


# Cluster tiles of 2^21 bits (two CTAs, distributed shared memory).  Intervals of at
# least 4 tiles per SM keep the tuning's tile size (shorter ones get smaller tiles).
CLUSTER_TUNINGS = [
    dict(tile_log2=21, presieve_groups=2, coop_max=4096, medium_max=1 << 21, window_tiles=512, epoch_tiles=2048),
    dict(tile_log2=21, presieve_groups=4, coop_max=2048, medium_max=1 << 14, window_tiles=64, epoch_tiles=300),
]


def with_tuning(ctx, tune, fn):
    saved = [S.sieve_get_tuning(ctx, k) for k in range(4)]
    try:
        for k in range(4):
            S.sieve_set_tuning(ctx, k, **tune)
        return fn()
    finally:
        for k in range(4):
            S.sieve_set_tuning(ctx, k, **saved[k])


@pytest.mark.parametrize("tune", CLUSTER_TUNINGS)
@pytest.mark.parametrize("j0,nbits", [(10**13 // 2 + 96, (1300 << 20) + 224), (10**17 // 2, (1 << 31) + (3 << 19) + 64)])
def test_cluster_tiles_ragged_ranges(ctx, tune, j0, nbits):
    def run():
        out = torch.empty(nbits // 32, dtype=torch.int32, device="cuda")
        S.sieve_segments(ctx, 5, j0 // 32, nbits // 32, out)
        S.sieve_sync(ctx)
        return host_words(out)
    got = with_tuning(ctx, tune, run)
    want = oracle.sieve_range(j0, nbits)
    assert first_diff(got, want) is None, first_diff(got, want)


def test_config2_cluster_tiles_against_stored_values(ctx):
    """The 1e15 configuration with 2^21-bit cluster tiles: table hash and segment counts,
    the host-output path, and the count mode (which runs 2^20-bit tiles) under the
    same tuning."""
    l, n = 20, 8192
    with open(os.path.join(GOLDEN, "c2_segments.txt")) as fh:
        lines = fh.read().splitlines()
    want_sha = lines[1].split()[2]
    want_counts = np.array([int(x.split()[1]) for x in lines[3:]], dtype=np.int64)

    def run():
        out = torch.empty((n << l) // 32, dtype=torch.int32, device="cuda")
        S.sieve_segments_midpoint(ctx, l, 1, 15, n, out)
        S.sieve_sync(ctx)
        words = host_words(out)
        del out
        f = S.sieve_f_from_midpoint(l, n, 1, 15)
        host = torch.empty((n << l) // 32, dtype=torch.int32).pin_memory()
        S.sieve_segments_host(ctx, l, f, n, host)
        pr = torch.empty(n, dtype=torch.int64, device="cuda")
        S.sieve_count_segments(ctx, l, f, n, pr)
        S.sieve_sync(ctx)
        return words, host.numpy().view(np.uint32), pr.cpu().numpy()
    words, hwords, primes = with_tuning(ctx, CLUSTER_TUNINGS[0], run)
    seg_counts = np.unpackbits(words.view(np.uint8)).reshape(n, -1).sum(axis=1)
    assert np.array_equal(seg_counts, want_counts)
    assert sha(words) == want_sha
    assert sha(hwords) == want_sha
    assert np.array_equal(primes, (1 << l) - want_counts)


def test_config3_cluster_tiles_against_stored_hash(ctx):
    l, n = 20, 32768
    f = oracle.f_from_midpoint(l, n, 1 << 60, 0)
    with open(os.path.join(GOLDEN, "c3_segments.txt")) as fh:
        want_sha = fh.read().splitlines()[1].split()[2]
    tune = dict(CLUSTER_TUNINGS[0], medium_max=1 << 20)

    def run():
        out = torch.empty((n << l) // 32, dtype=torch.int32, device="cuda")
        S.sieve_segments(ctx, l, f, n, out)
        S.sieve_sync(ctx)
        w = host_words(out)
        del out
        torch.cuda.empty_cache()
        return w
    assert sha(with_tuning(ctx, tune, run)) == want_sha


def test_config2_full_table_hash_and_segment_counts(ctx):
    l, n = 20, 8192
    f = oracle.f_from_midpoint(l, n, 1, 15)
    out = torch.empty((n << l) // 32, dtype=torch.int32, device="cuda")
    S.sieve_segments_midpoint(ctx, l, 1, 15, n, out)
    S.sieve_sync(ctx)
    with open(os.path.join(GOLDEN, "c2_segments.txt")) as fh:
        lines = fh.read().splitlines()
    assert ("f=%d" % f) in lines[0]
    want_sha = lines[1].split()[2]
    want_counts = np.array([int(x.split()[1]) for x in lines[3:]], dtype=np.int64)
    words = host_words(out)
    seg_counts = np.unpackbits(words.view(np.uint8)).reshape(n, -1).sum(axis=1)
    bad = np.nonzero(seg_counts != want_counts)[0]
    assert len(bad) == 0, "segments with wrong counts: %s" % bad[:10]
    assert sha(words) == want_sha
    assert S.sieve_count(ctx, out, n << l) == int(want_counts.sum())


def test_config3_whole_table_segments_and_miller_rabin(ctx):
    """The 2^60 configuration (l=20, n=32768) whole: SHA-256 of all 2^35 bits and every
    segment's composite count against the oracle's stored values, the 24 stored
    sampled segments, and 10^5 Miller-Rabin samples, half on 1 bits (composite) and
    half on 0 bits (prime), drawn at seeded random positions."""
    l, n = 20, 32768
    f = oracle.f_from_midpoint(l, n, 1 << 60, 0)
    assert f == 2**39 - 16384
    out = torch.empty((n << l) // 32, dtype=torch.int32, device="cuda")
    S.sieve_segments(ctx, l, f, n, out)
    S.sieve_sync(ctx)
    words = host_words(out)
    del out
    torch.cuda.empty_cache()
    with open(os.path.join(GOLDEN, "c3_segments.txt")) as fh:
        lines = fh.read().splitlines()
    assert ("f=%d" % f) in lines[0]
    want_sha = lines[1].split()[2]
    want_counts = np.array([int(x.split()[1]) for x in lines[3:]], dtype=np.int64)
    assert len(want_counts) == n
    seg_words = (1 << l) // 32
    seg = words.reshape(n, seg_words)
    got_counts = np.array([oracle.popcount(seg[t]) for t in range(n)], dtype=np.int64)
    bad = np.nonzero(got_counts != want_counts)[0]
    assert len(bad) == 0, "segments with wrong counts: %s" % bad[:10]
    assert sha(words) == want_sha
    with open(os.path.join(GOLDEN, "c3_samples.txt")) as fh:
        rows = [ln.split() for ln in fh if not ln.startswith("#")]
    for t, cnt, h in rows:
        assert oracle.popcount(seg[int(t)]) == int(cnt), "segment %s" % t
        assert sha(seg[int(t)]) == h, "segment %s" % t
    # Miller-Rabin, stratified: 5e4 bits that are 1 and 5e4 that are 0
    J0 = f << l
    rng = np.random.default_rng(0xC3)
    pos = rng.integers(0, n << l, size=3_000_000, dtype=np.int64)
    bits = (words[pos >> 5] >> (pos & 31).astype(np.uint32)) & 1
    ones, zeros = pos[bits == 1][:50_000], pos[bits == 0][:50_000]
    assert len(ones) == 50_000 and len(zeros) == 50_000
    for j in ones.tolist():
        assert not oracle.is_prime_mr(2 * (J0 + j) + 1), j
    for j in zeros.tolist():
        assert oracle.is_prime_mr(2 * (J0 + j) + 1), j


def test_count_matches_numpy(ctx):
    out = run_plain(ctx, 16, 12345, 77)
    w = host_words(out)
    assert S.sieve_count(ctx, out, 77 << 16) == int(np.unpackbits(w.view(np.uint8)).sum())
    assert S.sieve_count(ctx, out[1:], (77 << 16) - 32 * 5) == \
        int(np.unpackbits(w[1:-4].view(np.uint8)).sum())


def test_midpoint_entry_matches_oracle_reading(ctx):
    for (l, n, mant, e) in [(20, 16, 1, 12), (18, 40, 5, 13), (15, 3, 2, 18), (10, 5, 1, 3)]:
        f = S.sieve_f_from_midpoint(l, n, mant, e)
        assert f == oracle.f_from_midpoint(l, n, mant, e)
        out = torch.empty((n << l) // 32, dtype=torch.int32, device="cuda")
        S.sieve_segments_midpoint(ctx, l, mant, e, n, out)
        S.sieve_sync(ctx)
        assert np.array_equal(host_words(out), oracle.sieve(l, f, n))


def test_host_output_path_equals_device_path(ctx):
    l, f, n = 20, 2**30, 2500  # 2.4 Gbit: two windows of the host path
    dev = run_plain(ctx, l, f, n)
    host = torch.empty((n << l) // 32, dtype=torch.int32).pin_memory()
    S.sieve_segments_host(ctx, l, f, n, host)
    assert torch.equal(host, dev.cpu())


def test_graph_replay_is_identical(ctx):
    l, f, n = 19, 10**9, 300
    outs = []
    out = torch.empty((n << l) // 32, dtype=torch.int32, device="cuda")
    for _ in range(3):  # first direct, second captured, third replayed
        out.fill_(-1)
        S.sieve_segments(ctx, l, f, n, out)
        S.sieve_sync(ctx)
        outs.append(host_words(out).copy())
    want = oracle.sieve(l, f, n)
    for o in outs:
        assert np.array_equal(o, want)


def test_calls_on_two_streams_share_the_scratch_safely(ctx):
    """Two intervals issued back to back on two streams with no wait between them, three
    times (direct, captured, replayed).  Every plan of a context shares its bucket pools
    and counters, so each table must still equal the one computed alone."""
    saved = [S.sieve_get_tuning(ctx, k) for k in range(4)]
    try:
        for k in range(4):  # eight epochs of 128 tiles per interval: both pools reused often
            S.sieve_set_tuning(ctx, k, tile_log2=20, presieve_groups=2, coop_max=4096,
                               medium_max=1 << 19, window_tiles=128, epoch_tiles=128)
        l, n = 20, 1024
        fs = ((10**15 >> 21) - 512, (10**16 >> 21) - 512)
        want = []
        for f in fs:
            w = torch.empty((n << l) // 32, dtype=torch.int32, device="cuda")
            S.sieve_segments(ctx, l, f, n, w)
            S.sieve_sync(ctx)
            want.append(w)
        streams = (torch.cuda.Stream(), torch.cuda.Stream())
        outs = [torch.empty_like(w) for w in want]
        for _ in range(3):
            for o in outs:
                o.fill_(-1)
            torch.cuda.synchronize()
            for f, o, st in zip(fs, outs, streams):
                S.sieve_segments(ctx, l, f, n, o, stream=st)
            for st in streams:
                S.sieve_sync(ctx, st)
            for o, w in zip(outs, want):
                assert torch.equal(o, w)
    finally:
        for k in range(4):
            S.sieve_set_tuning(ctx, k, **saved[k])


def test_argument_errors(ctx):
    out = torch.empty(1 << 10, dtype=torch.int32, device="cuda")
    with pytest.raises(S.SieveError) as e:
        S.sieve_segments(ctx, 4, 0, 1, out)
    assert e.value.status == 1
    with pytest.raises(S.SieveError) as e:
        S.sieve_segments(ctx, 10, 0, 0, out)
    assert e.value.status == 1
    with pytest.raises(S.SieveError) as e:  # numbers beyond 2^64
        S.sieve_segments(ctx, 20, 1 << 43, 1, torch.empty(1 << 15, dtype=torch.int32, device="cuda"))
    assert e.value.status == 2
    with pytest.raises(ValueError):  # a table larger than the buffer never reaches the library
        S.sieve_segments(ctx, 20, 0, 1, out)
    with pytest.raises(S.SieveError) as e:  # sqrt beyond the context's base (2^31)
        S.sieve_segments(ctx, 5, (1 << 58) - 1, 1, out)
    assert e.value.status == 2
    with pytest.raises(S.SieveError) as e:  # batch request not word aligned
        S.sieve_batch(ctx, [(16, 64, 0)], out, torch.zeros(1, dtype=torch.int64, device="cuda"))
    assert e.value.status == 1


def test_top_of_range_against_miller_rabin():
    c = S.sieve_init(0, max_v=(1 << 64) - 1)
    try:
        _, cnt, lim = S.sieve_base_info(c)
        assert lim == 2**32 - 1 and cnt + 1 == 203280221  # pi(2^32), OEIS A007053
        nbits = 1 << 13
        j0 = (1 << 63) - nbits  # the last number is 2^64 - 1
        out = torch.empty(nbits // 32, dtype=torch.int32, device="cuda")
        S.sieve_segments(c, 5, j0 // 32, nbits // 32, out)
        S.sieve_sync(c)
        w = host_words(out)
        for j in range(nbits):
            bit = (int(w[j // 32]) >> (j % 32)) & 1
            assert bit == (0 if oracle.is_prime_mr(2 * (j0 + j) + 1) else 1), j
    finally:
        c.close()


def test_segments_larger_than_a_tile_equal_small_segments(ctx):
    """The table depends only on the numbers, not on l (Sec. 1.3): two segments of
    l = 30 (each 1024 on-chip tiles) equal 2048 segments of l = 20 over the same
    numbers, bit for bit, and Miller-Rabin on sampled bits."""
    f30 = 9311  # numbers around 2^42 * 2 ~ 1.8e13
    big = run_plain(ctx, 30, f30, 2)
    small = run_plain(ctx, 20, f30 << 10, 2048)
    assert torch.equal(big, small)
    rng = workloads.SplitMix64(30)
    J0 = f30 << 30
    for _ in range(500):
        j = rng.below(2 << 30)
        bit = (int(big[j // 32].item()) >> (j % 32)) & 1
        assert bit == (0 if oracle.is_prime_mr(2 * (J0 + j) + 1) else 1), j


def test_host_output_small_and_repeated(ctx):
    """Host output for tables of one word to one tile, twice each: the second call
    reuses the cached plan and must write the new host buffer."""
    for (l, f, n) in [(5, 3, 1), (5, 3, 7), (12, 1000, 3), (20, 2 ** 30, 1)]:
        want = oracle.sieve(l, f, n)
        for _ in range(2):
            host = torch.full(((n << l) // 32,), -1, dtype=torch.int32).pin_memory()
            S.sieve_segments_host(ctx, l, f, n, host)
            got = host.numpy().view(np.uint32)
            assert first_diff(got, want) is None, (l, f, n, first_diff(got, want))
