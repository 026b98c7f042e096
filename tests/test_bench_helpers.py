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


def test_step_roofline_is_the_slower_of_bytes_and_marks():
    # B_alg = N/8 + 16 H_large + 4 V bytes at the copy bandwidth, against H marks at the
    # shared-memory atomic rate; the fraction is the roofline time over the step time
    b = _bench()
    N, h_large, visits, marks = 8 * 10**9, 10**8, 5 * 10**7, 4 * 10**9
    bytes_alg = N / 8 + 16 * h_large + 4 * visits  # 2.8e9 B
    r = b.step_roofline(N, marks, h_large, visits, 2e-3, 7000.0, 3.5e12)
    assert r["bytes_alg"] == bytes_alg
    t_hbm, t_atom = bytes_alg / 7e12, marks / 3.5e12  # 0.4 ms, 1.143 ms
    assert r["bound"] == "smem_atomic"
    assert abs(r["t_roof_ms"] - t_atom * 1e3) < 1e-12
    assert abs(r["frac"] - t_atom / 2e-3) < 1e-12
    r = b.step_roofline(N, marks / 100, h_large, visits, 2e-3, 7000.0, 3.5e12)
    assert r["bound"] == "hbm" and abs(r["frac"] - t_hbm / 2e-3) < 1e-12
