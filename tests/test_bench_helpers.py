"""The roofline figures of bench.py rest on closed-form mark counts; these tests pin
them against brute force (no GPU)."""
import importlib.util
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def brute_marks(J0, N, primes):
    """Odd multiples m = p*c of each prime with c coprime to 15 and m >= p^2 whose
    index (m-1)/2 lies in [J0, J0+N) (the marks of Sec. 1.4 and the wheel of Sec. 3.2.1)."""
    total = 0
    lo, hi = 2 * J0 + 1, 2 * (J0 + N) - 1
    for p in primes:
        c = max(p, -(-lo // p))
        if c % 2 == 0:
            c += 1
        while p * c <= hi:
            if c % 3 and c % 5:
                total += 1
            c += 2
    return total


def test_wheel_marks_equals_brute_force():
    b = _bench()
    primes = [int(p) for p in b.base_primes_upto(3000) if p >= 17]
    for J0, N in [(0, 1 << 14), (12345, 1 << 13), (10 ** 6, 1 << 15), (10 ** 9 + 7, 1 << 14), (2 ** 40, 5000)]:
        assert b.wheel_marks(J0, N, np.array(primes)) == brute_marks(J0, N, primes), (J0, N)


def test_medium_marks_takes_primes_between_presieve_and_medium_max():
    b = _bench()
    tune = {"presieve_groups": 2, "medium_max": 1000}
    J0, N = 5 * 10 ** 5, 1 << 14
    primes = [int(p) for p in b.base_primes_upto(1000) if 23 < p <= 1000]
    assert b.medium_marks(J0, N, tune) == brute_marks(J0, N, primes)


def test_base_primes_upto_counts():
    b = _bench()
    # pi(10^k) - 1 odd primes (2 is not in the odd-only base)
    for x, pi in [(10, 4), (100, 25), (1000, 168), (10 ** 5, 9592)]:
        assert len(b.base_primes_upto(x)) == pi - 1
