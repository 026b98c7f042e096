"""Seeded synthetic workloads shared by the tests, the benchmark and the oracle side.

This module holds none of the sieve's arithmetic: it only draws random numbers
and turns them into interval requests (absolute bit index j0 and bit count
nbits, both multiples of 32) and arrival times.  Both the CUDA path and the
oracle consume what it produces.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written out here so that a seed
gives the same stream on every machine and numpy version.
"""
import math

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64: state += golden gamma; output = mix(state)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def below(self, n: int) -> int:
        """Uniform integer in [0, n) (n <= 2^64), by rejection."""
        if n <= 0:
            raise ValueError("n must be positive")
        lim = (1 << 64) - ((1 << 64) % n)
        while True:
            x = self.next_u64()
            if x < lim:
                return x % n


# The paper-style interval configurations: segment size exponent l, number of
# segments n, and the interval's midpoint as mantissa * 10^exp10 (or a power of
# two, given as mant=2^k, exp10=0).
PLAIN_CONFIGS = {
    # odd numbers in [1, 2^26]: l=15, f=0, n=1024
    "c1_l15_f0_n1024": dict(l=15, f=0, n=1024),
    # 2^34 consecutive numbers around 1e15: l=20, n=8192
    "c2_l20_n8192_mid1e15": dict(l=20, n=8192, mant=1, exp10=15),
    # 2^36 consecutive numbers around 2^60: l=20, n=32768
    "c3_l20_n32768_mid2p60": dict(l=20, n=32768, mant=1 << 60, exp10=0),
}


def batch_requests(count: int = 4096, seed: int = 0,
                   len_lo: float = 2.0 ** 16, len_hi: float = 2.0 ** 28,
                   mid_lo: float = 1e6, mid_hi: float = 1e18):
    """Interval requests with lengths (in numbers) log-uniform in [len_lo, len_hi]
    and midpoints log-uniform in [mid_lo, mid_hi].

    Each request becomes (j0, nbits): nbits = floor(L/2) rounded down to a
    multiple of 32 (odd numbers only), j0 = max(0, floor(M/2) - nbits/2)
    rounded down to a multiple of 32.  Returns a list of (j0, nbits) tuples.
    """
    rng = SplitMix64(0x5EED0000 + seed)
    la, lb = math.log(len_lo), math.log(len_hi)
    ma, mb = math.log(mid_lo), math.log(mid_hi)
    out = []
    for _ in range(count):
        L = math.exp(la + (lb - la) * rng.uniform())
        M = math.exp(ma + (mb - ma) * rng.uniform())
        nbits = (int(L) // 2) // 32 * 32
        nbits = max(nbits, 32)
        j0 = max(0, int(M) // 2 - nbits // 2) // 32 * 32
        out.append((j0, nbits))
    return out


def poisson_arrivals(count: int, rate_per_s: float, seed: int = 0):
    """Arrival times (seconds from 0) of a Poisson process with the given rate."""
    rng = SplitMix64(0xA7712000 + seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += -math.log(1.0 - rng.uniform()) / rate_per_s
        out.append(t)
    return out
