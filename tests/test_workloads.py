"""The seeded input generators are deterministic and produce valid requests."""
import os

from paper_1111_3297_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_reference_outputs():
    # first outputs for seed 0, from the generator's published definition
    # (Steele, Lea & Flood 2014; also the seeding generator of xoshiro)
    r = workloads.SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_batch_requests_deterministic_and_word_aligned():
    a = workloads.batch_requests(4096, seed=0)
    b = workloads.batch_requests(4096, seed=0)
    assert a == b
    assert a != workloads.batch_requests(4096, seed=1)
    for j0, nbits in a:
        assert j0 % 32 == 0 and nbits % 32 == 0 and nbits >= 32
        assert 2**15 - 32 <= nbits <= 2**27
        assert 2 * (j0 + nbits) + 1 < 2 * 10**18 + 2**28


def test_stored_batch_requests_match_generator():
    path = os.path.join(GOLDEN, "batch_4096_seed0.txt")
    if not os.path.exists(path):
        import pytest
        pytest.skip("golden batch file not generated")
    stored = []
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            stored.append((int(parts[1]), int(parts[2])))
    assert stored == workloads.batch_requests(4096, seed=0)


def test_poisson_arrivals_rate():
    t = workloads.poisson_arrivals(20000, 2000.0, seed=0)
    assert all(b > a for a, b in zip(t, t[1:]))
    rate = len(t) / t[-1]
    assert 1900 < rate < 2100
