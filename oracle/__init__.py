"""Python access to the CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does: it has no
CPU fallback and fails when its CUDA library is missing.

The oracle computes the sieve table of Jarai & Vatai (Definition "Sieve table,
Segments", Sec. 1.3): bit j stands for the odd number 2(J0 + j) + 1 and is 1
exactly when that number is composite.  See ``sieve_oracle.c`` for the passage
each routine follows.
"""
import ctypes
import os

import numpy as np

from .build import build_oracle

_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        lib.oracle_isqrt.restype = _u64
        lib.oracle_isqrt.argtypes = [_u64]
        lib.oracle_base_primes.restype = _u64
        lib.oracle_base_primes.argtypes = [_u64, ctypes.c_void_p, _u64]
        lib.oracle_sieve_range.restype = ctypes.c_int
        lib.oracle_sieve_range.argtypes = [_u64, _u64, _u64, ctypes.c_void_p, _u64, _u64,
                                           ctypes.c_void_p, ctypes.c_int]
        lib.oracle_sieve.restype = ctypes.c_int
        lib.oracle_sieve.argtypes = [_u32, _u64, _u64, ctypes.c_void_p, _u64, _u64,
                                     ctypes.c_void_p, ctypes.c_int]
        lib.oracle_lemma_q.restype = _u64
        lib.oracle_lemma_q.argtypes = [_u64, _u64, _u32]
        lib.oracle_f_from_midpoint.restype = ctypes.c_int
        lib.oracle_f_from_midpoint.argtypes = [_u32, _u64, _u64, _u32, ctypes.POINTER(_u64)]
        lib.oracle_popcount.restype = _u64
        lib.oracle_popcount.argtypes = [ctypes.c_void_p, _u64]
        lib.oracle_is_composite_trial.restype = ctypes.c_int
        lib.oracle_is_composite_trial.argtypes = [_u64]
        lib.oracle_is_prime_mr.restype = ctypes.c_int
        lib.oracle_is_prime_mr.argtypes = [_u64]
        lib.oracle_goldbach_min_p.restype = ctypes.c_int
        lib.oracle_goldbach_min_p.argtypes = [_u64, _u64, ctypes.c_void_p, _u64, _u32, ctypes.c_void_p]
        lib.oracle_segment_counts.restype = ctypes.c_int
        lib.oracle_segment_counts.argtypes = [ctypes.c_void_p, _u64, _u64, _u32, ctypes.c_void_p,
                                              ctypes.c_void_p]
        _lib = lib
    return _lib


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def isqrt(x: int) -> int:
    return int(_load().oracle_isqrt(x))


class Base:
    """The base P of Sec. 1.4: odd primes 3 <= p <= limit (ascending, uint32)."""

    def __init__(self, limit: int):
        lib = _load()
        limit = min(int(limit), 0xFFFFFFFF)
        cnt = lib.oracle_base_primes(limit, None, 0)
        if cnt == 2**64 - 1:
            raise MemoryError("oracle base primes")
        arr = np.zeros(max(int(cnt), 1), dtype=np.uint32)
        got = lib.oracle_base_primes(limit, arr.ctypes.data, cnt)
        if got != cnt:
            raise MemoryError("oracle base primes")
        self.limit = limit
        self.primes = arr[:cnt]


_base_cache = {}


def base_for(max_number: int) -> Base:
    """A base covering every number up to max_number (cached by limit)."""
    need = isqrt(max_number)
    for lim, b in _base_cache.items():
        if lim >= need:
            return b
    b = Base(need)
    _base_cache.clear()
    _base_cache[need] = b
    return b


def sieve_range(j0: int, nbits: int, seg_bits: int = 1 << 20, base: Base = None,
                nthreads: int = None) -> np.ndarray:
    """Table words (uint32, LSB-first) for absolute bit indices j0 .. j0+nbits-1."""
    if nbits == 0:
        return np.zeros(0, dtype=np.uint32)
    if base is None:
        base = base_for(2 * (j0 + nbits - 1) + 1)
    out = np.zeros(nbits // 32, dtype=np.uint32)
    rc = _load().oracle_sieve_range(j0, nbits, seg_bits, base.primes.ctypes.data,
                                    len(base.primes), base.limit, out.ctypes.data,
                                    nthreads or default_threads())
    if rc != 0:
        raise ValueError("oracle_sieve_range failed with code %d" % rc)
    return out


def sieve(l: int, f: int, n: int, base: Base = None, nthreads: int = None) -> np.ndarray:
    """The paper's table for (l, f, n): n*2^l bits, segments of 2^l bits."""
    nbits = n << l
    if base is None:
        base = base_for(2 * ((f << l) + nbits - 1) + 1)
    out = np.zeros(nbits // 32, dtype=np.uint32)
    rc = _load().oracle_sieve(l, f, n, base.primes.ctypes.data, len(base.primes),
                              base.limit, out.ctypes.data, nthreads or default_threads())
    if rc != 0:
        raise ValueError("oracle_sieve failed with code %d" % rc)
    return out


def lemma_q(p: int, f: int, l: int) -> int:
    return int(_load().oracle_lemma_q(p, f, l))


def f_from_midpoint(l: int, n: int, mant: int, exp10: int) -> int:
    out = _u64(0)
    rc = _load().oracle_f_from_midpoint(l, n, mant, exp10, ctypes.byref(out))
    if rc != 0:
        raise ValueError("oracle_f_from_midpoint failed with code %d" % rc)
    return int(out.value)


def popcount(words: np.ndarray) -> int:
    words = np.ascontiguousarray(words, dtype=np.uint32)
    return int(_load().oracle_popcount(words.ctypes.data, len(words)))


def is_composite_trial(m: int) -> bool:
    return bool(_load().oracle_is_composite_trial(m))


def is_prime_mr(m: int) -> bool:
    return bool(_load().oracle_is_prime_mr(m))


def segment_counts(words: np.ndarray, J0: int, nbits: int, l: int):
    """(primes, twins) per segment of 2^l bits of a table whose bit j stands for
    2(J0 + j) + 1: the primes (0 bits, the number 1 excluded) and the twin pairs
    (m, m + 2) both prime with m + 2 inside the first nbits bits, by the segment of m
    (oracle_segment_counts)."""
    words = np.ascontiguousarray(words, dtype=np.uint32)
    assert 32 * len(words) >= nbits
    nseg = (nbits + (1 << l) - 1) >> l
    pr = np.zeros(max(nseg, 1), dtype=np.uint64)
    tw = np.zeros(max(nseg, 1), dtype=np.uint64)
    rc = _load().oracle_segment_counts(words.ctypes.data, J0, nbits, l, pr.ctypes.data, tw.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_segment_counts failed with code %d" % rc)
    return pr[:nseg].astype(np.int64), tw[:nseg].astype(np.int64)


def goldbach_min_p(n_lo: int, count: int, p_max: int) -> np.ndarray:
    """For each even N = n_lo + 2i (i < count) the smallest odd prime p <= p_max with
    N - p prime (Miller-Rabin on N - p), 0 if none (oracle_goldbach_min_p)."""
    primes = Base(max(3, p_max)).primes
    out = np.zeros(max(int(count), 1), dtype=np.uint32)
    rc = _load().oracle_goldbach_min_p(n_lo, count, primes.ctypes.data, len(primes), p_max, out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_goldbach_min_p failed with code %d" % rc)
    return out[:count]


def goldbach_windows(n_lo: int, min_p: np.ndarray, win_log2: int):
    """Per window of 2^win_log2 consecutive even numbers: (largest minimal p, the first N
    attaining it, or None when no N of the window has a p; numbers with no p)."""
    out = []
    w = 1 << win_log2
    for k in range(0, len(min_p), w):
        part = np.asarray(min_p[k:k + w], dtype=np.int64)
        fail = int((part == 0).sum())
        mx = int(part.max())
        if mx == 0:
            out.append((0, None, fail))
        else:
            out.append((mx, int(n_lo) + 2 * (k + int(np.argmax(part == mx))), fail))
    return out


def get_bit(words: np.ndarray, j: int) -> int:
    return int((int(words[j >> 5]) >> (j & 31)) & 1)


def _coprime_prefix(W: int) -> np.ndarray:
    """pre[x] = number of odd c in [1, x] with gcd(c, W) = 1, for 0 <= x < 2W (W odd)."""
    c = np.arange(2 * W, dtype=np.int64)
    ok = (c % 2 == 1) & (np.gcd(c, W) == 1)
    return np.cumsum(ok)


def large_prime_hits(j0: int, nbits: int, primes, W: int = 1) -> int:
    """Hits that striking with the primes `primes` emits on the bits j0 .. j0+nbits-1:
    for each p, the odd multiples m = p*c in [max(2*j0+1, p^2), 2*(j0+nbits)-1] (Sec. 1.4:
    from the first multiple in the interval, but never below p^2), keeping only the
    multipliers c coprime to W (the wheel, Sec. 3.2.1; W = 1 keeps all).  By Theorem
    thm:big and Cor. cor:complete (Sec. 2.3) every such multiple lands in exactly one
    segment's bucket, so a method that emits each hit once emits exactly this many.
    Closed form per prime (numpy, int64: numbers below 2^62)."""
    p = np.asarray(primes, dtype=np.int64)
    if len(p) == 0 or nbits == 0:
        return 0
    lo_num = 2 * int(j0) + 1
    hi_num = 2 * (int(j0) + int(nbits)) - 1
    assert hi_num < (1 << 62)
    start = np.maximum(lo_num, p * p)
    c1 = (start + p - 1) // p            # smallest multiplier with p*c >= start
    c1 = c1 + (1 - c1 % 2)               # ... made odd
    c2 = hi_num // p
    c2 = c2 - (1 - c2 % 2)               # largest odd multiplier with p*c <= hi_num
    ok = c1 <= c2
    if W == 1:
        cnt = (c2 - c1) // 2 + 1
        return int(cnt[ok].sum())
    pre = _coprime_prefix(W)
    per = int(pre[-1])                   # phi(W) odd residues per period 2W

    def F(x):                            # odd c in [1, x] coprime to W, x >= 0
        return (x // (2 * W)) * per + pre[x % (2 * W)]
    cnt = F(c2) - F(np.maximum(c1 - 1, 0))
    return int(cnt[ok].sum())
