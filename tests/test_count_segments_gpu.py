"""The count-only consumer (sieve_count_segments) against the oracle: per-segment prime
counts and twin-pair counts of an interval, computed inside the segment kernel without
writing the table.  Integer results: compared exactly, segment by segment."""
import os

import numpy as np
import pytest

import oracle
from paper_1111_3297_gb300 import sieve as S

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


def device_counts(ctx, l, f, n, twins=True):
    pr = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    tw = torch.full((n,), -1, dtype=torch.int64, device="cuda") if twins else None
    S.sieve_count_segments(ctx, l, f, n, pr, tw)
    S.sieve_sync(ctx)
    return pr.cpu().numpy(), (tw.cpu().numpy() if twins else None)


def oracle_counts(l, f, n):
    w = oracle.sieve(l, f, n)
    return oracle.segment_counts(w, f << l, n << l, l)


def test_config1_counts(ctx):
    l, f, n = 15, 0, 1024
    pr, tw = device_counts(ctx, l, f, n)
    want_p, want_t = oracle_counts(l, f, n)
    assert np.array_equal(pr, want_p)
    assert np.array_equal(tw, want_t)
    # pi(2^26) - 1 (2 is not in the table) and the pairs below 2^26
    assert int(pr.sum()) == 3957809 - 1


GRID = [(12, 0, 3), (12, 1, 700), (13, 5000, 333), (16, 10**6, 77), (20, 10**6, 50),
        (14, 2**40, 300), (12, 2**44 + 7, 257), (20, 2**36, 64), (18, 2**42 + 3, 33)]


@pytest.mark.parametrize("l,f,n", GRID)
def test_grid_counts(ctx, l, f, n):
    pr, tw = device_counts(ctx, l, f, n)
    want_p, want_t = oracle_counts(l, f, n)
    assert np.array_equal(pr, want_p), np.nonzero(pr != want_p)[0][:5]
    assert np.array_equal(tw, want_t), np.nonzero(tw != want_t)[0][:5]


TUNINGS = [
    dict(tile_log2=12, presieve_groups=1, coop_max=64, medium_max=1 << 11, window_tiles=4, epoch_tiles=9),
    dict(tile_log2=14, presieve_groups=6, coop_max=256, medium_max=1 << 13, window_tiles=16, epoch_tiles=40),
    dict(tile_log2=20, presieve_groups=13, coop_max=4096, medium_max=1 << 20, window_tiles=1024, epoch_tiles=4096),
]


@pytest.mark.parametrize("tune", TUNINGS)
@pytest.mark.parametrize("l,f,n", [(12, 3, 1000), (15, 2**33 + 5, 90), (13, 0, 129)])
def test_tunings_counts(ctx, tune, l, f, n):
    saved = [S.sieve_get_tuning(ctx, k) for k in range(4)]
    try:
        for k in range(4):
            S.sieve_set_tuning(ctx, k, **tune)
        pr, tw = device_counts(ctx, l, f, n)
    finally:
        for k in range(4):
            S.sieve_set_tuning(ctx, k, **saved[k])
    want_p, want_t = oracle_counts(l, f, n)
    assert np.array_equal(pr, want_p)
    assert np.array_equal(tw, want_t)


def test_counts_equal_the_table_path_and_replay(ctx):
    l, mant, e, n = 20, 1, 16, 256
    f = S.sieve_f_from_midpoint(l, n, mant, e)
    out = torch.empty((n << l) // 32, dtype=torch.int32, device="cuda")
    S.sieve_segments(ctx, l, f, n, out)
    S.sieve_sync(ctx)
    words = out.cpu().numpy().view(np.uint32).reshape(n, -1)
    comp = np.array([oracle.popcount(words[t]) for t in range(n)])
    for rep in range(3):  # the second call captures a graph, the third replays it
        pr, tw = device_counts(ctx, l, f, n)
        assert np.array_equal(pr, (1 << l) - comp), rep
    want_p, want_t = oracle.segment_counts(words.reshape(-1), f << l, n << l, l)
    assert np.array_equal(tw, want_t)
    pr2, _ = device_counts(ctx, l, f, n, twins=False)
    assert np.array_equal(pr2, pr)


def test_config2_counts_against_stored_values(ctx):
    l, n = 20, 8192
    f = oracle.f_from_midpoint(l, n, 1, 15)
    with open(os.path.join(GOLDEN, "c2_counts.txt")) as fh:
        lines = fh.read().splitlines()
    assert ("f=%d" % f) in lines[0]
    rows = np.array([[int(x) for x in ln.split()] for ln in lines[2:]], dtype=np.int64)
    pr, tw = device_counts(ctx, l, f, n)
    assert np.array_equal(pr, rows[:, 1])
    assert np.array_equal(tw, rows[:, 2])
    with open(os.path.join(GOLDEN, "c2_segments.txt")) as fh:
        comp = np.array([int(x.split()[1]) for x in fh.read().splitlines()[3:]], dtype=np.int64)
    assert np.array_equal(pr, (1 << l) - comp)


def test_count_argument_errors(ctx):
    pr = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(S.SieveError):
        S.sieve_count_segments(ctx, 11, 0, 8, pr)  # segments below 4096 bits
    with pytest.raises(ValueError):
        S.sieve_count_segments(ctx, 12, 0, 9, pr)  # output shorter than n
