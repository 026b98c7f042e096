"""Pins of oracle.large_prime_hits (the hit count that Theorem thm:big and
Cor. cor:complete, Sec. 2.3, imply: every odd multiple from max(u, p^2) on, struck
once) against brute-force enumeration of multiples on tiny intervals."""
import math

import numpy as np
import pytest

import oracle


def brute(j0, nbits, primes, W):
    n = 0
    for J in range(j0, j0 + nbits):
        m = 2 * J + 1
        for p in primes:
            if m % p == 0 and m >= p * p and math.gcd(m // p, W) == 1:
                n += 1
    return n


@pytest.mark.parametrize("W", [1, 15, 15015])
@pytest.mark.parametrize("j0,nbits", [(0, 700), (31, 1000), (5000, 2048), (123456, 3000), (10**7, 1500)])
def test_hits_closed_form_equals_enumeration(W, j0, nbits):
    primes = [int(p) for p in oracle.Base(5000).primes if p >= 3]
    sel = [p for p in primes if p >= (17 if W == 15015 else 7)]
    assert oracle.large_prime_hits(j0, nbits, sel, W) == brute(j0, nbits, sel, W)


def test_hits_without_wheel_are_the_marks_of_the_table():
    # with W = 1 and every base prime, the hits are the (p, m) pairs with p | m, m >= p^2:
    # on an interval above sqrt, each composite m is hit once per distinct prime factor
    # p <= sqrt(m); so the hits are at least the composite count and at most 9 per number
    j0, nbits = 10**6, 4096
    base = oracle.base_for(2 * (j0 + nbits) - 1)
    h = oracle.large_prime_hits(j0, nbits, base.primes, 1)
    comp = oracle.popcount(oracle.sieve_range(j0, nbits, base=base))
    assert comp <= h <= 9 * comp
    # exact: sum over composites of their distinct prime factors up to their root
    want = 0
    for J in range(j0, j0 + nbits):
        m = 2 * J + 1
        want += sum(1 for p in base.primes if m % p == 0 and p * p <= m)
    assert h == want


def test_hits_density_of_the_big_wheel():
    # an interval of p*W bits starting at the multiple p*c covers the odd multipliers
    # c, c+2, ..., c+2W-2: one whole period, of which phi(15015) = 5760 are coprime
    p, W = 100003, 15015
    c = 2 * W * 50 + 1
    j0 = (p * c - 1) // 2
    assert oracle.large_prime_hits(j0, p * W, [p], W) == 5760
    assert oracle.large_prime_hits(j0, p * W, [p], 15) == W * 8 // 15
    assert oracle.large_prime_hits(j0, p * W, [p], 1) == W
