"""The Goldbach consumer (sieve_goldbach) against the oracle: per window of even
numbers, the largest minimal partition prime p, the first N attaining it, and the
numbers with no p <= p_max.  Integer results: compared exactly."""
import numpy as np
import pytest

import oracle
from paper_1111_3297_gb300 import sieve as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_3297_gb300 import build
    build.build_library()
    c = S.sieve_init(0, max_v=1 << 62)
    yield c
    c.close()


def table(ctx, l, f, n):
    out = torch.empty((n << l) // 32, dtype=torch.int32, device="cuda")
    S.sieve_segments(ctx, l, f, n, out)
    S.sieve_sync(ctx)
    return out


def device_windows(ctx, out, j0, nbits, n_lo, count, p_max, win_log2):
    nwin = ((count - 1) >> win_log2) + 1
    w = torch.full((2 * nwin,), -1, dtype=torch.int64, device="cuda")
    S.sieve_goldbach(ctx, out, j0, nbits, n_lo, count, p_max, win_log2, w)
    S.sieve_sync(ctx)
    return S.goldbach_windows(w.cpu().tolist(), n_lo, win_log2)


def test_small_numbers_from_the_table_at_one(ctx):
    # odd numbers 1 .. 2^23 - 1; even N from 4: N = 4 has no odd-prime partition
    l, f, n = 16, 0, 64
    out = table(ctx, l, f, n)
    n_lo, count, p_max = 4, (1 << 22) - 8, 4000
    got = device_windows(ctx, out, 0, n << l, n_lo, count, p_max, 12)
    want = oracle.goldbach_windows(n_lo, oracle.goldbach_min_p(n_lo, count, p_max), 12)
    assert got == want
    assert got[0][2] == 1  # N = 4
    assert max(g[0] for g in got) >= 601  # the record at 1077422 lies in the range


@pytest.mark.parametrize("mid,count,p_max,win_log2", [(10**12, 1 << 17, 2000, 10), (10**15, 1 << 16, 5000, 16),
                                                      (10**18, 1 << 17, 3000, 13), (2**61, 70001, 8000, 5)])
def test_windows_at_large_magnitude(ctx, mid, count, p_max, win_log2):
    n_lo = mid - mid % 2
    # a table from below N - p_max to above the largest N - 3, in 2^16-bit segments
    l = 16
    lo_j = (n_lo - p_max - 1) // 2
    hi_j = (n_lo + 2 * count) // 2
    f = lo_j >> l
    n = ((hi_j >> l) + 1) - f
    out = table(ctx, l, f, n)
    got = device_windows(ctx, out, f << l, n << l, n_lo, count, p_max, win_log2)
    want = oracle.goldbach_windows(n_lo, oracle.goldbach_min_p(n_lo, count, p_max), win_log2)
    assert got == want


def test_small_p_max_reports_failures(ctx):
    l, f, n = 16, 0, 16
    out = table(ctx, l, f, n)
    n_lo, count, p_max = 1000, 100000, 13
    got = device_windows(ctx, out, 0, n << l, n_lo, count, p_max, 14)
    want = oracle.goldbach_windows(n_lo, oracle.goldbach_min_p(n_lo, count, p_max), 14)
    assert got == want
    assert sum(g[2] for g in got) > 0


def test_goldbach_argument_errors(ctx):
    out = table(ctx, 12, 0, 4)
    w = torch.zeros(64, dtype=torch.int64, device="cuda")
    with pytest.raises(S.SieveError):
        S.sieve_goldbach(ctx, out, 0, 4 << 12, 5, 16, 100, 5, w)       # odd n_lo
    with pytest.raises(S.SieveError):
        S.sieve_goldbach(ctx, out, 0, 4 << 12, 4, 16, 100, 4, w)       # windows below 32 numbers
    with pytest.raises(S.SieveError):
        S.sieve_goldbach(ctx, out, 0, 4 << 12, 4, (1 << 14) + 2, 100, 12, w)  # N - 3 beyond the table
    with pytest.raises(S.SieveError):
        S.sieve_goldbach(ctx, out, 64, 4 << 12, 100, 16, 101, 5, w)    # N - p_max below the table


@pytest.mark.parametrize("n_lo,count,win", [(4, 1, 5), (6, 3, 32), (1000, 33, 5), (4, 1 << 20, 32)])
def test_goldbach_edge_ranges(ctx, n_lo, count, win):
    # tables from 1: one number, a window wider than the range, a block straddling two
    # windows of 32, a 2^32-number window over 2^20 numbers
    l, f = 12, 0
    n = ((n_lo + 2 * count) // 2 >> l) + 1
    out = table(ctx, l, f, n)
    got = device_windows(ctx, out, 0, n << l, n_lo, count, 997, win)
    want = oracle.goldbach_windows(n_lo, oracle.goldbach_min_p(n_lo, count, 997), win)
    assert got == want
