"""Pins of the oracle's Goldbach search (oracle.goldbach_min_p, goldbach_windows):
the published record minimal partitions below 1.1e6, and trial division on small N."""
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_records_below_1p1e6_equal_published():
    want = []
    with open(os.path.join(GOLDEN, "goldbach_records.txt")) as fh:
        for ln in fh:
            if not ln.startswith("#") and ln.strip():
                want.append(tuple(int(x) for x in ln.split()))
    m = oracle.goldbach_min_p(4, (1_100_000 - 4) // 2, 1000)
    got, best = [], 0
    for i, p in enumerate(m.tolist()):
        if p > best:
            best = p
            got.append((4 + 2 * i, p))
    assert got == want
    assert m[0] == 0  # 4 = 2 + 2 has no odd-prime partition
    assert (m[1:] > 0).all()


def is_prime_trial(m):
    return m > 1 and not oracle.is_composite_trial(m)


def test_min_p_equals_trial_division():
    n_lo, count = 4, 1500
    m = oracle.goldbach_min_p(n_lo, count, 200)
    for i in range(count):
        N = n_lo + 2 * i
        want = 0
        for p in range(3, min(200, N - 3) + 1, 2):
            if is_prime_trial(p) and is_prime_trial(N - p):
                want = p
                break
        assert m[i] == want, N


def test_p_max_bounds_the_search_and_windows_decode():
    n_lo = 10**12
    m = oracle.goldbach_min_p(n_lo, 4096, 50)
    big = oracle.goldbach_min_p(n_lo, 4096, 10**5)
    assert ((m == big) | ((m == 0) & (big > 50))).all()
    w = oracle.goldbach_windows(n_lo, big, 10)
    assert len(w) == 4
    for k, (mx, N, fail) in enumerate(w):
        part = big[k * 1024:(k + 1) * 1024]
        assert mx == part.max() and fail == 0
        assert N == n_lo + 2 * (k * 1024 + int(np.nonzero(part == mx)[0][0]))
