"""Pins for the CPU oracle: each test checks it against something other than itself.

* brute force (trial division, an independent primality routine) on tiny inputs;
* published prime counts pi(x) (tests/golden/pi_table.txt);
* deterministic Miller-Rabin, itself pinned by trial division and by numbers of
  known primality (tests/golden/known_primality.txt);
* Lemma lem:q (Sec. 2.1) in the paper's parity form against brute force and the
  congruence form;
* invariants: p itself never marked, 1 never marked, concatenation of tables,
  independence of the segment size.
"""
import math
import os
import random

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def bits_of(words, nbits):
    return np.unpackbits(words.view(np.uint8), bitorder="little")[:nbits]


def test_isqrt_matches_exact_integer_root():
    rnd = random.Random(1)
    vals = [0, 1, 2, 3, 4, 15, 16, 17, 2**32 - 1, 2**32, 2**62, 2**64 - 1]
    vals += [rnd.getrandbits(64) for _ in range(2000)]
    vals += [k * k - 1 for k in (3, 2**20, 2**31 + 11, 2**32 - 1)]
    for v in vals:
        assert oracle.isqrt(v) == math.isqrt(v), v


def read_pi_table():
    out = []
    with open(os.path.join(GOLDEN, "pi_table.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            x, pi = line.split()
            out.append((int(x), int(pi)))
    return out


@pytest.mark.parametrize("x,pi", read_pi_table())
def test_base_primes_count_matches_published_pi(x, pi):
    # the base holds the odd primes <= x; pi(x) also counts 2
    assert 1 + len(oracle.Base(x).primes) == pi


def test_base_primes_are_exactly_the_trial_division_primes():
    b = oracle.Base(20000).primes.tolist()
    want = [m for m in range(3, 20001, 2) if not oracle.is_composite_trial(m)]
    assert b == want


def test_mr_agrees_with_trial_division_on_small_numbers():
    for m in range(0, 200001):
        comp = oracle.is_composite_trial(m)
        prime = oracle.is_prime_mr(m)
        # 0 and 1 are neither prime nor composite
        if m < 2:
            assert not prime and not comp
        else:
            assert prime == (not comp), m


def test_mr_on_numbers_of_known_primality():
    with open(os.path.join(GOLDEN, "known_primality.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            v = int(parts[1])
            if parts[0] == "prime":
                assert oracle.is_prime_mr(v), v
            else:
                prod = 1
                for x in parts[2:]:
                    prod *= int(x)
                assert prod == v  # the factorisation really is one
                assert not oracle.is_prime_mr(v), v


def _bruteforce_table(l, f, n):
    return np.array([1 if oracle.is_composite_trial(2 * ((f << l) + j) + 1) else 0
                     for j in range(n << l)], dtype=np.uint8)


@pytest.mark.parametrize("l", [5, 6, 7, 8, 10])
@pytest.mark.parametrize("f", [0, 1, 2, 3, 5, 13, 34, 64])
@pytest.mark.parametrize("n", [1, 2, 3, 8])
def test_table_equals_trial_division_on_tiny_grid(l, f, n):
    got = bits_of(oracle.sieve(l, f, n), n << l)
    assert np.array_equal(got, _bruteforce_table(l, f, n))


def test_config1_first_65536_bits_by_trial_division():
    w = oracle.sieve(15, 0, 1024)
    got = bits_of(w[:2048], 65536)
    assert np.array_equal(got, _bruteforce_table(16, 0, 1))


def test_config1_count_equals_published_pi():
    # odd numbers 1..2^26-1 are 2^25 bits; the primes among them are pi(2^26)-1
    # (no 2) and 1 is not composite, so composites = 2^25 - pi(2^26)
    w = oracle.sieve(15, 0, 1024)
    assert oracle.popcount(w) == 2**25 - 3957809


@pytest.mark.parametrize("j0", [10**12 // 2, 10**15 // 2, 10**16 // 2 + 12345 * 32,
                                (2**60) // 2 - 4096])
def test_table_equals_miller_rabin_far_from_zero(j0):
    j0 = j0 // 32 * 32
    nbits = 8192
    w = oracle.sieve_range(j0, nbits, seg_bits=2048)
    got = bits_of(w, nbits)
    want = np.array([0 if oracle.is_prime_mr(2 * (j0 + j) + 1) else 1 for j in range(nbits)],
                    dtype=np.uint8)
    assert np.array_equal(got, want)


def test_lemma_q_parity_form():
    rnd = random.Random(7)
    primes = oracle.Base(1 << 20).primes
    for _ in range(3000):
        p = int(primes[rnd.randrange(len(primes))])
        l = rnd.randrange(5, 31)
        f = rnd.getrandbits(rnd.choice([1, 8, 20, 33]))
        q = oracle.lemma_q(p, f, l)
        assert 0 <= q < p
        assert (2 * ((f << l) + q) + 1) % p == 0
        # congruence form: q = (p-1)/2 - f*2^l (mod p)
        assert q == ((p - 1) // 2 - (f << l)) % p
    # brute force: the smallest q >= 0 with p | 2(f 2^l + q) + 1
    for p in (3, 5, 7, 11, 13, 101):
        for l in (5, 6, 9):
            for f in range(0, 40):
                q = next(q for q in range(p) if (2 * ((f << l) + q) + 1) % p == 0)
                assert oracle.lemma_q(p, f, l) == q


def test_primes_and_one_are_never_marked():
    w = oracle.sieve(10, 0, 64)  # odd numbers below 2^17
    bits = bits_of(w, 64 << 10)
    assert bits[0] == 0  # the number 1
    for p in oracle.Base((64 << 11) - 1).primes:
        assert bits[(int(p) - 1) // 2] == 0
    # an interval that contains base primes of its own square root
    l, f, n = 12, 3, 4
    w = oracle.sieve(l, f, n)
    bits = bits_of(w, n << l)
    for j in range(n << l):
        m = 2 * ((f << l) + j) + 1
        if oracle.is_prime_mr(m):
            assert bits[j] == 0


def test_concatenation_and_segment_size_independence():
    l, f, n, n1 = 11, 1000, 12, 5
    whole = oracle.sieve(l, f, n)
    a = oracle.sieve(l, f, n1)
    b = oracle.sieve(l, f + n1, n - n1)
    assert np.array_equal(whole, np.concatenate([a, b]))
    # the same numbers with another segment size give the same bits
    j0, nbits = f << l, n << l
    for seg in (32, 96, 4096, 1 << 16):
        assert np.array_equal(whole, oracle.sieve_range(j0, nbits, seg_bits=seg))
    assert np.array_equal(oracle.sieve(10, 4, 8), oracle.sieve(12, 1, 2))


def test_f_from_midpoint_reading():
    # midpoint 2^60, l=20, n=32768: f = 2^39 - 16384
    assert oracle.f_from_midpoint(20, 32768, 1 << 60, 0) == 2**39 - 16384
    assert oracle.f_from_midpoint(20, 8192, 1, 15) == 10**15 // 2**21 - 4096
    assert oracle.f_from_midpoint(15, 1024, 1, 3) == 0
    for (l, n, mant, e) in [(20, 1024, 1, 12), (20, 1024, 2, 18), (16, 7, 5, 13)]:
        f = oracle.f_from_midpoint(l, n, mant, e)
        M = mant * 10**e
        mid = (f + n / 2) * 2 ** (l + 1)
        assert abs(mid - M) <= 2 ** (l + 1)
