"""Write the stored expected values used by the full-size parity tests.

Calls only the CPU oracle (``oracle/``) and the seeded input generators; no value
here comes from the CUDA path.  Run from the repository root:

    python tests/golden/make_golden.py [c2] [c2counts] [c3] [c3full] [batch]

Outputs (text, one record per line):
  c2_segments.txt     l=20, n=8192, midpoint 1e15: per-segment composite counts,
                      plus the SHA-256 of the whole packed table.
  c3_samples.txt      l=20, n=32768, midpoint 2^60: 24 seeded segments, each with its
                      composite count and SHA-256.
  c2_counts.txt       the l=20, n=8192, 1e15 table's per-segment prime and twin-pair
                      counts (oracle.segment_counts).
  c3_segments.txt     the same table whole: per-segment composite counts and the
                      SHA-256 of all 2^35 bits (computed 512 segments at a time).
  batch_4096_seed0.txt  the 4096 seeded batch requests (j0, nbits) with each one's
                      composite count and SHA-256.
Tables are hashed as little-endian uint32 words (bit j = word j/32, bit j%32).
"""
import hashlib
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1111_3297_gb300 import workloads  # noqa: E402


def sha(words):
    return hashlib.sha256(np.ascontiguousarray(words, dtype="<u4").tobytes()).hexdigest()


def make_c2():
    l, n = 20, 8192
    f = oracle.f_from_midpoint(l, n, 1, 15)
    t0 = time.time()
    w = oracle.sieve(l, f, n)
    seg_words = (1 << l) // 32
    counts = [oracle.popcount(w[t * seg_words:(t + 1) * seg_words]) for t in range(n)]
    with open(os.path.join(HERE, "c2_segments.txt"), "w") as fh:
        fh.write("# l=20 n=8192 midpoint=1e15 f=%d (written by tests/golden/make_golden.py "
                 "from the CPU oracle, %.0f s)\n" % (f, time.time() - t0))
        fh.write("# sha256 %s\n" % sha(w))
        fh.write("# total %d\n" % sum(counts))
        for t, c in enumerate(counts):
            fh.write("%d %d\n" % (t, c))


def make_c2_counts():
    l, n = 20, 8192
    f = oracle.f_from_midpoint(l, n, 1, 15)
    t0 = time.time()
    w = oracle.sieve(l, f, n)
    pr, tw = oracle.segment_counts(w, f << l, n << l, l)
    with open(os.path.join(HERE, "c2_counts.txt"), "w") as fh:
        fh.write("# l=20 n=8192 midpoint=1e15 f=%d: segment t, primes, twin pairs with the lower "
                 "member in t (tests/golden/make_golden.py, CPU oracle, %.0f s)\n" % (f, time.time() - t0))
        fh.write("# total %d %d\n" % (int(pr.sum()), int(tw.sum())))
        for t in range(n):
            fh.write("%d %d %d\n" % (t, pr[t], tw[t]))


def make_c3(nsamples=24):
    l, n = 20, 32768
    f = oracle.f_from_midpoint(l, n, 1 << 60, 0)
    rng = workloads.SplitMix64(0xC3)
    segs = sorted({0, n - 1} | {rng.below(n) for _ in range(nsamples - 2)})
    base = oracle.base_for(2 * ((f + n) << l) - 1)
    t0 = time.time()
    with open(os.path.join(HERE, "c3_samples.txt"), "w") as fh:
        fh.write("# l=20 n=32768 midpoint=2^60 f=%d: sampled segments t, composite count, "
                 "sha256 (tests/golden/make_golden.py, CPU oracle)\n" % f)
        for t in segs:
            w = oracle.sieve(l, f + t, 1, base=base)
            fh.write("%d %d %s\n" % (t, oracle.popcount(w), sha(w)))
            fh.flush()
    print("c3 %.0f s" % (time.time() - t0))


def make_c3_full(chunk=512):
    l, n = 20, 32768
    f = oracle.f_from_midpoint(l, n, 1 << 60, 0)
    base = oracle.base_for(2 * ((f + n) << l) - 1)
    seg_words = (1 << l) // 32
    h = hashlib.sha256()
    counts = []
    t0 = time.time()
    for t0seg in range(0, n, chunk):
        w = oracle.sieve(l, f + t0seg, chunk, base=base)
        h.update(np.ascontiguousarray(w, dtype="<u4").tobytes())
        counts += [oracle.popcount(w[k * seg_words:(k + 1) * seg_words]) for k in range(chunk)]
        print("c3full %d/%d segments, %.0f s" % (t0seg + chunk, n, time.time() - t0), flush=True)
    with open(os.path.join(HERE, "c3_segments.txt"), "w") as fh:
        fh.write("# l=20 n=32768 midpoint=2^60 f=%d (written by tests/golden/make_golden.py "
                 "from the CPU oracle, %.0f s)\n" % (f, time.time() - t0))
        fh.write("# sha256 %s\n" % h.hexdigest())
        fh.write("# total %d\n" % sum(counts))
        for t, c in enumerate(counts):
            fh.write("%d %d\n" % (t, c))


_base = None


def _batch_one(args):
    global _base
    idx, j0, nbits, lim = args
    if _base is None or _base.limit < oracle.isqrt(2 * (j0 + nbits) - 1):
        _base = oracle.Base(lim)
    w = oracle.sieve_range(j0, nbits, seg_bits=nbits, base=_base, nthreads=1)
    return idx, oracle.popcount(w), sha(w)


def make_batch(seed=0, count=4096):
    reqs = workloads.batch_requests(count, seed=seed)
    lim = max(oracle.isqrt(2 * (j0 + nb) - 1) for j0, nb in reqs)
    t0 = time.time()
    jobs = [(i, j0, nb, lim) for i, (j0, nb) in enumerate(reqs)]
    res = [None] * count
    with mp.get_context("fork").Pool(os.cpu_count()) as pool:
        for idx, c, h in pool.imap_unordered(_batch_one, jobs, chunksize=4):
            res[idx] = (c, h)
    with open(os.path.join(HERE, "batch_%d_seed%d.txt" % (count, seed)), "w") as fh:
        fh.write("# %d seeded batch requests (paper_1111_3297_gb300.workloads.batch_requests, "
                 "seed %d): index j0 nbits composite_count sha256 "
                 "(tests/golden/make_golden.py, CPU oracle, %.0f s)\n" % (count, seed,
                                                                          time.time() - t0))
        for i, (j0, nb) in enumerate(reqs):
            fh.write("%d %d %d %d %s\n" % (i, j0, nb, res[i][0], res[i][1]))


if __name__ == "__main__":
    which = sys.argv[1:] or ["c2", "c3", "batch"]
    for w in which:
        t = time.time()
        {"c2": make_c2, "c2counts": make_c2_counts, "c3": make_c3, "c3full": make_c3_full, "batch": make_batch}[w]()
        print(w, "done in %.0f s" % (time.time() - t), flush=True)
