"""Pins of oracle.segment_counts (per-segment primes and twin pairs of a table):
published pi(10^k) and twin-pair counts below 10^k, brute force by trial division
on small intervals, and sums over segments equal to counts over the whole."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for ln in fh:
            if ln.startswith("#") or not ln.strip():
                continue
            x, v = ln.split()
            rows.append((int(x), int(v)))
    return rows


def counts_below(x, l):
    """Counts over the odd numbers below x (x even): bits j < x/2, l-bit segments."""
    nbits = x // 2
    words = oracle.sieve_range(0, (nbits + 31) // 32 * 32)
    return oracle.segment_counts(words, 0, nbits, l)


@pytest.mark.parametrize("x,pairs", read_table("twin_table.txt"))
def test_twin_pairs_below_powers_of_ten(x, pairs):
    pr, tw = counts_below(x, 12)
    assert int(tw.sum()) == pairs


@pytest.mark.parametrize("x,pi", [r for r in read_table("pi_table.txt") if r[0] % 10 == 0])
def test_primes_below_powers_of_ten(x, pi):
    pr, tw = counts_below(x, 12)
    assert int(pr.sum()) == pi - 1  # the table holds the odd numbers: 2 is not in it


def is_prime_trial(m):
    return m > 1 and not oracle.is_composite_trial(m)


@pytest.mark.parametrize("J0,nbits,l", [(0, 4096, 6), (0, 1000, 3), (12352, 3000, 7), (10**6, 2048, 5),
                                        (10**9, 4096, 10), (2**31 - 96, 640, 4)])
def test_segment_counts_equal_trial_division(J0, nbits, l):
    words = oracle.sieve_range(J0, (nbits + 31) // 32 * 32)
    pr, tw = oracle.segment_counts(words, J0, nbits, l)
    want_p = np.zeros_like(pr)
    want_t = np.zeros_like(tw)
    isp = [is_prime_trial(2 * (J0 + j) + 1) for j in range(nbits)]
    for j in range(nbits):
        if isp[j]:
            want_p[j >> l] += 1
            if j + 1 < nbits and isp[j + 1]:
                want_t[j >> l] += 1
    assert np.array_equal(pr, want_p)
    assert np.array_equal(tw, want_t)


def test_segments_sum_to_the_whole_and_split_by_lower_member():
    J0, nbits = 777760, 1 << 14
    words = oracle.sieve_range(J0, nbits)
    whole_p, whole_t = oracle.segment_counts(words, J0, nbits, 20)
    for l in (5, 8, 13):
        pr, tw = oracle.segment_counts(words, J0, nbits, l)
        assert pr.sum() == whole_p[0] and tw.sum() == whole_t[0]
    # a pair straddling two segments belongs to the segment of its lower member:
    # 3, 5 (bits 1, 2) with 1-bit segments lands in segment 1 (bit 1)
    w = oracle.sieve_range(0, 32)
    pr, tw = oracle.segment_counts(w, 0, 8, 0)
    assert list(pr) == [0, 1, 1, 1, 0, 1, 1, 0]  # 1 is not prime; 3, 5, 7, 11, 13
    assert list(tw) == [0, 1, 1, 0, 0, 1, 0, 0]  # (3,5) (5,7) (11,13); (1,3) is not a pair
