"""Seeded random intervals and tunings against the oracle, bit for bit: segment sizes
l = 5..20, magnitudes 1 .. 1e17, lengths from one word to 2^22 bits, and every tuning
parameter drawn from its valid range (tiles 2^12..2^20, 1..13 pre-sieve groups,
medium / large thresholds, scatter groups and epochs)."""
import pytest

import oracle
from paper_1111_3297_gb300 import sieve as S
from paper_1111_3297_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_3297_gb300 import build
    build.build_library()
    c = S.sieve_init(0, max_v=2 * 10**17 + (1 << 30))
    yield c
    c.close()


def draw(seed):
    r = workloads.SplitMix64(0x5EED + seed)
    l = 5 + r.below(16)
    mag = 10 ** (r.below(18))
    n = 1 + r.below(max(1, (1 << 22) >> l))
    f = (mag // (2 << l)) + r.below(1 << 10)
    tl = 12 + r.below(9)
    tune = dict(tile_log2=tl, presieve_groups=1 + r.below(13), coop_max=1 << (6 + r.below(8)),
                medium_max=1 << (8 + r.below(14)), window_tiles=1 << r.below(11), epoch_tiles=0)
    while (tune["window_tiles"] << tl) > (1 << 30):
        tune["window_tiles"] >>= 1
    tune["epoch_tiles"] = tune["window_tiles"] * (1 + r.below(8))
    return l, f, n, tune


@pytest.mark.parametrize("seed", range(40))
def test_random_interval_and_tuning(ctx, seed):
    l, f, n, tune = draw(seed)
    saved = [S.sieve_get_tuning(ctx, k) for k in range(4)]
    try:
        for k in range(4):
            S.sieve_set_tuning(ctx, k, **tune)
        out = torch.empty((n << l) // 32, dtype=torch.int32, device="cuda")
        S.sieve_segments(ctx, l, f, n, out)
        S.sieve_sync(ctx)
        got = out.cpu().numpy().view("uint32")
    finally:
        for k in range(4):
            S.sieve_set_tuning(ctx, k, **saved[k])
    want = oracle.sieve(l, f, n)
    assert (got == want).all(), (l, f, n, tune)


def draw_batch(seed):
    r = workloads.SplitMix64(0xBA7C + seed)
    reqs, off = [], 0
    for _ in range(8 + r.below(40)):
        nb = 32 * (1 + r.below(1 << (4 + r.below(12))))
        mag = 10 ** r.below(18)
        j0 = 32 * ((mag // 64) + r.below(1 << 12))
        reqs.append((j0, nb, off))
        off += (nb // 32 + 3) // 4 * 4 + 4 * r.below(3)
    return reqs, off, draw(1000 + seed)[3]


@pytest.mark.parametrize("seed", range(12))
def test_random_batch_and_tuning(ctx, seed):
    reqs, words, tune = draw_batch(seed)
    saved = [S.sieve_get_tuning(ctx, k) for k in range(4)]
    try:
        for k in range(4):
            S.sieve_set_tuning(ctx, k, **tune)
        arena = torch.zeros(words, dtype=torch.int32, device="cuda")
        counts = torch.empty(len(reqs), dtype=torch.int64, device="cuda")
        S.sieve_batch(ctx, reqs, arena, counts)
        S.sieve_sync(ctx)
        host = arena.cpu().numpy().view("uint32")
        got_c = counts.cpu().tolist()
    finally:
        for k in range(4):
            S.sieve_set_tuning(ctx, k, **saved[k])
    for (j0, nb, o), c in zip(reqs, got_c):
        want = oracle.sieve_range(j0, nb)
        assert (host[o:o + nb // 32] == want).all(), (j0, nb, tune)
        assert c == oracle.popcount(want), (j0, nb)


@pytest.mark.parametrize("seed", range(12))
def test_random_count_segments(ctx, seed):
    r = workloads.SplitMix64(0xC0DE + seed)
    l = 12 + r.below(9)
    n = 1 + r.below(max(1, (1 << 22) >> l))
    f = (10 ** r.below(18)) // (2 << l) + r.below(1 << 8)
    tune = draw(2000 + seed)[3]
    saved = [S.sieve_get_tuning(ctx, k) for k in range(4)]
    try:
        for k in range(4):
            S.sieve_set_tuning(ctx, k, **tune)
        pr = torch.empty(n, dtype=torch.int64, device="cuda")
        tw = torch.empty(n, dtype=torch.int64, device="cuda")
        S.sieve_count_segments(ctx, l, f, n, pr, tw)
        S.sieve_sync(ctx)
    finally:
        for k in range(4):
            S.sieve_set_tuning(ctx, k, **saved[k])
    want_p, want_t = oracle.segment_counts(oracle.sieve(l, f, n), f << l, n << l, l)
    assert (pr.cpu().numpy() == want_p).all() and (tw.cpu().numpy() == want_t).all(), (l, f, n, tune)


@pytest.mark.parametrize("seed", range(8))
def test_random_goldbach(ctx, seed):
    r = workloads.SplitMix64(0x601D + seed)
    p_max = 3 + r.below(3000)
    count = 1 + r.below(1 << 15)
    win = 5 + r.below(12)
    mag = 10 ** (3 + r.below(15))
    n_lo = max(4, mag - mag % 2 + 2 * r.below(1 << 20))
    # a table of 2^12-bit segments from below N - p_max (or from 1) to past the largest N - 3
    l = 12
    lo_j = max(0, (n_lo - p_max - 1) // 2)
    f = lo_j >> l
    if n_lo <= p_max + 3:
        f = 0
    hi_j = (n_lo + 2 * count) // 2
    n = (hi_j >> l) + 1 - f
    out = torch.empty((n << l) // 32, dtype=torch.int32, device="cuda")
    S.sieve_segments(ctx, l, f, n, out)
    nwin = ((count - 1) >> win) + 1
    w = torch.empty(2 * nwin, dtype=torch.int64, device="cuda")
    S.sieve_goldbach(ctx, out, f << l, n << l, n_lo, count, p_max, win, w)
    S.sieve_sync(ctx)
    got = S.goldbach_windows(w.cpu().tolist(), n_lo, win)
    want = oracle.goldbach_windows(n_lo, oracle.goldbach_min_p(n_lo, count, p_max), win)
    assert got == want, (n_lo, count, p_max, win)
