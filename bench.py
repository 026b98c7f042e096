"""Benchmark: odd numbers sieved per second on GB300, with roofline and CPU baseline.

Default workload (one GPU): l=20, n=8192 segments (2^34 consecutive numbers,
2^33 odd ones) with the midpoint at 10^15, the paper's (l, f, n) interface.
--workload c3 runs l=20, n=32768 around 2^60 (the large-prime-dominated case).
Beside the workload, the batched-vs-plain measurement runs 4096 seeded requests of
uneven length and magnitude (--batch-requests), then serving and a midpoint sweep.
Under torchrun each rank sieves its own interval of the same size (the next n
segments): weak scaling, no collective on the data path.

Prints one JSON line.  `value` is device-timed throughput (CUDA events on the
launching stream, outputs resident in HBM); `e2e` is the same metric through the
C ABI with the table delivered to pinned host memory.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "c2": dict(name="l20_n8192_mid1e15", l=20, n=8192, mant=1, exp10=15),
    "c3": dict(name="l20_n32768_mid2p60", l=20, n=32768, mant=1 << 60, exp10=0),
    "c1": dict(name="l15_f0_n1024", l=15, n=1024, f=0),
    # one point of the paper's Table 1 sweep: 2^30 odd numbers around 10^18 (profiling case)
    "m1e18": dict(name="l20_n1024_mid1e18", l=20, n=1024, mant=1, exp10=18),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "m1e18"])
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tuning", default="", help="JSON tuning to use as is (no autotune), e.g. for profiling")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--segments", type=int, default=0, help="override n (small profiling cases)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-vs-plain measurement")
    ap.add_argument("--batch-requests", type=int, default=4096,
                    help="requests in the batched-vs-plain measurement (fewer for profiling cases)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-seconds", type=float, default=20.0)
    ap.add_argument("--serve-sweep-seconds", type=float, default=1.5,
                    help="arrival time per rate of the saturating serving sweep (0: no sweep)")
    ap.add_argument("--no-c3", action="store_true", help="skip the 2^60 sub-record of the default run")
    ap.add_argument("--fresh-steps", type=int, default=4, help="fresh-interval steps (0: none)")
    ap.add_argument("--no-consumers", action="store_true", help="skip the count-only and Goldbach legs")
    ap.add_argument("--no-sweep", action="store_true", help="skip the 1e12..1e18 midpoint sweep")
    ap.add_argument("--clocks-csv", default="",
                    help="where to keep the nvidia-smi samples of the timed region (default: a temp file)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device, path=""):
        self.device = device
        self.proc = None
        self.path = path or os.path.join(tempfile.gettempdir(), "clocks_bench_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# exact algorithmic counts for the roofline
# ---------------------------------------------------------------------------
def wheel_marks(J0, N, primes):
    """Marks the device executes for these primes on [J0, J0+N): odd multiples
    m = p*c, c coprime to 15, m >= p^2 (Sec. 1.4, Sec. 3.2.1); closed form per prime."""
    import numpy as np
    p = np.asarray(primes, dtype=np.int64)
    if len(p) == 0:
        return 0
    half = (p - 1) // 2
    first = J0 + ((half - J0) % p)
    jsq = (p * p - 1) // 2
    J1 = np.maximum(first, jsq)
    Jend = J0 + N - 1
    Jlast = Jend - ((Jend - half) % p)
    ok = J1 <= Jlast
    c1 = (2 * J1 + 1) // p
    c2 = (2 * Jlast + 1) // p
    # T[r] = residues in {1, 7, 11, 13, 17, 19, 23, 29} (odd, coprime to 15) that are <= r
    T = np.cumsum(np.isin(np.arange(30), [1, 7, 11, 13, 17, 19, 23, 29]))

    def F(x):  # odd c <= x, coprime to 15
        q, r = np.divmod(x, 30)
        return 8 * q + T[r]

    cnt = F(c2) - F(c1 - 1)
    return int(cnt[ok].sum())


PRESIEVE_MAX = [13, 23, 31, 41, 47, 59, 67, 73, 83, 97, 103, 109, 127]  # largest prime of groups 1..13


def medium_marks(J0, N, tune, primes=None):
    """Wheel-reduced marks of the primes the tile kernel strikes on [J0, J0+N): above
    the pre-sieve's primes, up to medium_max and isqrt of the last number.  primes:
    odd primes up to at least that bound (computed here when None)."""
    import math
    plimit = math.isqrt(2 * (J0 + N) - 1)
    top = min(plimit, tune["medium_max"])
    if primes is None:
        primes = base_primes_upto(top)
    import numpy as np
    a = np.searchsorted(primes, PRESIEVE_MAX[tune["presieve_groups"] - 1], side="right")
    b = np.searchsorted(primes, top, side="right")
    return wheel_marks(J0, N, primes[a:b])


def _marks_chunk(args):
    reqs, tune = args
    primes = base_primes_upto(tune["medium_max"])
    return sum(medium_marks(j0, nb, tune, primes) for j0, nb in reqs)


def batch_medium_marks(reqs, tune, world=1):
    """Sum of medium_marks over many requests (j0, nbits), spread over this rank's share
    of the host cores by a spawn-started process pool (never forked: the parent holds
    a CUDA context); computed in this process if the pool fails or takes over 120 s."""
    import multiprocessing as mp
    k = max(1, min(16, (os.cpu_count() or 1) // max(1, world)))
    chunks = [(reqs[i::k], tune) for i in range(k)]
    if k > 1:
        pool = None
        try:
            pool = mp.get_context("spawn").Pool(k)
            return sum(pool.map_async(_marks_chunk, chunks).get(timeout=120))
        except Exception:
            pass
        finally:
            if pool is not None:
                pool.terminate()
                pool.join()
    return sum(_marks_chunk(c) for c in chunks)


def step_roofline(N, marks, h_large, visits, t_step, hbm_peak, r_atom):
    """T_roof = max(B_alg / BW_HBM, H / R_atom), B_alg = N/8 + 16 H_large + 4 V, against
    the measured step time."""
    b_alg = N / 8 + 16 * h_large + 4 * visits
    t_roof = max(b_alg / (hbm_peak * 1e9), marks / r_atom)
    return {"t_roof_ms": t_roof * 1e3, "t_step_ms": t_step * 1e3, "frac": t_roof / t_step,
            "bytes_alg": b_alg, "marks": marks,
            "bound": "hbm" if b_alg / (hbm_peak * 1e9) >= marks / r_atom else "smem_atomic"}


def base_primes_upto(x):
    """Odd primes <= x (index i stands for 2i+1)."""
    import numpy as np
    x = int(x)
    if x < 3:
        return np.zeros(0, dtype=np.int64)
    s = np.ones((x - 1) // 2 + 1, dtype=bool)
    s[0] = False
    for i in range(1, (int(x ** 0.5) + 1) // 2 + 1):
        if s[i]:
            p = 2 * i + 1
            s[(p * p) // 2::p] = False
    return 2 * np.nonzero(s)[0] + 1


# ---------------------------------------------------------------------------
def run_reference(args, rank, world, wl):
    """The oracle (CPU) on a bounded sample of the workload, timed on the host cores."""
    if rank != 0:
        return
    import oracle
    l, n = wl["l"], wl["n"]
    f = wl.get("f")
    if f is None:
        f = oracle.f_from_midpoint(l, n, wl["mant"], wl["exp10"])
    sample = 64 if args.workload != "c1" else n
    base = oracle.base_for(2 * ((f + n) << l) - 1)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.sieve(l, f, min(sample, 8), base=base, nthreads=cores)
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.sieve(l, f + (k * sample) % max(1, n - sample + 1), sample, base=base, nthreads=cores)
    dt = time.perf_counter() - t0
    val = args.steps * (sample << l) / dt
    print(json.dumps({
        "impl": "reference", "metric": "odd numbers sieved/s", "value": val,
        "unit": "odd numbers/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": wl["name"], "l": l, "f": f, "n": n},
        "cpu_baseline": {"value": val, "unit": "odd numbers/s", "cores": cores, "kind": "oracle",
                         "sample": "%d of %d segments (2^%d bits each) per step, all host cores" % (sample, n, l)},
        "e2e": {"value": val, "unit": "odd numbers/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def cpu_baseline(wl, f):
    import oracle
    l, n = wl["l"], wl["n"]
    cores = os.cpu_count() or 1
    sample = min(n, 1024 if l <= 16 else 256)
    base = oracle.base_for(2 * ((f + n) << l) - 1)
    t0 = time.perf_counter()
    oracle.sieve(l, f, sample, base=base, nthreads=cores)
    dt = time.perf_counter() - t0
    # one core on a proportionally smaller sample (the same segments' start)
    sample1 = max(1, sample // cores)
    t0 = time.perf_counter()
    oracle.sieve(l, f, sample1, base=base, nthreads=1)
    dt1 = time.perf_counter() - t0
    return {"value": (sample << l) / dt, "unit": "odd numbers/s", "cores": cores, "kind": "oracle",
            "sample": "first %d of %d segments (2^%d bits each), %.2f s on %d threads"
                      % (sample, n, l, dt, cores),
            "single_core": {"value": (sample1 << l) / dt1, "unit": "odd numbers/s", "cores": 1,
                            "sample": "first %d segments, %.2f s on 1 thread" % (sample1, dt1)}}


KERNEL_SOURCES = ("kernels.cu", "sieve_internal.cuh")  # everything compiled into the kernels


def kernel_code_hash(csrc):
    """SHA-256 (16 hex digits) of the kernels' CUDA sources with comments and blank
    lines removed: the key under which profiles/traffic.json stores counters of that
    code."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        src = re.sub(r"/\*.*?\*/", "", open(os.path.join(csrc, name)).read(), flags=re.S)
        lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in src.split("\n")]
        h.update("\n".join(ln for ln in lines if ln.strip()).encode())
    return h.hexdigest()[:16]


def measure_sweep(S, ctx, hbm_peak, r_atom):
    """The paper's Table 1 workload (Sec. 5): one interval of 2^30 bits (l = 20,
    n = 1024) with its midpoint at 10^e, e = 12..18, each timed alone (CUDA events,
    5 calls after 3 warm-up calls, class tunings of the context) with its step
    roofline."""
    import torch
    l, n = 20, 1024
    N = n << l
    out = torch.empty(N // 32, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    points = []
    for e in range(12, 19):
        f = S.sieve_f_from_midpoint(l, n, 1, e)
        J0 = f << l
        for _ in range(3):
            S.sieve_segments(ctx, l, f, n, out)
        S.sieve_sync(ctx)
        S.sieve_profile_enable(ctx, True)
        S.sieve_profile_read(ctx)
        reps = 5
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            S.sieve_segments(ctx, l, f, n, out)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = S.sieve_profile_read(ctx)
        S.sieve_profile_enable(ctx, False)
        t = e0.elapsed_time(e1) * 1e-3 / reps
        vlast = 2 * (J0 + N - 1) + 1
        tune = S.sieve_get_tuning(ctx, 0 if vlast < 2**40 else 1 if vlast < 2**50 else 2 if vlast < 2**56 else 3)
        h_large = prof["large_hits"] / reps
        roof = step_roofline(N, medium_marks(J0, N, tune) + h_large, h_large, prof["prime_reads"] / reps, t,
                             hbm_peak, r_atom)
        points.append({"midpoint": "1e%d" % e, "f": f, "ms": t * 1e3, "value": N / t,
                       "step_roofline_frac": roof["frac"], "bound": roof["bound"]})
    del out
    return {"l": l, "n": n, "bits": N, "unit": "odd numbers/s", "points": points}


def max_over_ranks(pg, x):
    """Largest x over the ranks of the default process group (x itself without one):
    the step time of a multi-rank run is the slowest rank's."""
    if not pg:
        return x
    import torch
    dev = "cuda" if pg.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_value(world, N, steps, ms_max):
    """Whole-job throughput: the odd numbers all ranks sieved over the slowest rank's time."""
    return world * N * steps / (ms_max * 1e-3)


def load_traffic(key, N, h_large, n_tile, n_scatter):
    """DRAM bytes per launch from the committed ncu capture of the same kernels on a
    smaller slice of the same workload, scaled by the kernel's units per launch; None
    when the kernels' code (kernels.cu, sieve_internal.cuh) changed since the capture."""
    traffic = {"k_tile": None, "k_scatter": None}
    try:
        tj = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        ksha = kernel_code_hash(os.path.join(ROOT, "paper_1111_3297_gb300", "csrc"))
        if key and tj.get("kernel_code_sha256_16") == ksha and key in tj:
            tt, ts = tj[key]["k_tile"], tj[key]["k_scatter"]
            if n_tile:
                traffic["k_tile"] = tt["dram_bytes"] / tt["units"] * (N / n_tile)
            if n_scatter:
                traffic["k_scatter"] = ts["dram_bytes"] / ts["units"] * (h_large / n_scatter)
    except Exception:
        pass
    return traffic


def measure_interval(S, ctx, l, f, n, steps, warmup, tune, hbm_peak, hbm_src, r_atom, traffic_key,
                     pg=None, clocks_path=""):
    """One interval (l, f, n) sieved `steps` times into the same device table after
    `warmup` untimed calls, CUDA events on the launching stream around the whole
    timed region, nvidia-smi clocks sampled during it.  Returns the device-timed
    figures with the per-kernel split, the dominant kernel's roofline and the step
    roofline (the slower of the algorithmic HBM bytes at the copy bandwidth and the marks at
    the shared-atomic rate, over the step time), and keeps the table in ["out"]."""
    import torch
    N = n << l
    J0 = f << l
    stream = torch.cuda.current_stream()
    out = torch.empty(N // 32, dtype=torch.int32, device="cuda")
    for _ in range(max(3, warmup)):
        S.sieve_segments(ctx, l, f, n, out)
    S.sieve_sync(ctx)

    # ---- timed region: K steps, per-kernel CUDA events inside the library ----
    S.sieve_profile_enable(ctx, True)
    S.sieve_profile_read(ctx)  # reset
    clocks = Clocks(torch.cuda.current_device(), clocks_path)
    clocks.start()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        S.sieve_segments(ctx, l, f, n, out)
    ev1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    prof = S.sieve_profile_read(ctx)
    S.sieve_profile_enable(ctx, False)
    S.sieve_sync(ctx)
    # one more step (not timed) with the scatter and tile launches on one stream: each
    # kernel's own time, whose shares compare with the ncu launch list and which picks
    # the dominant kernel (inside the timed region the two overlap and share the SMs)
    S.sieve_profile_enable(ctx, True, serial=True)
    S.sieve_profile_read(ctx)
    S.sieve_segments(ctx, l, f, n, out)
    prof_serial = S.sieve_profile_read(ctx)
    S.sieve_profile_enable(ctx, False)
    S.sieve_sync(ctx)
    ms_max = max_over_ranks(pg, ms)

    h_medium = medium_marks(J0, N, tune)  # per step
    h_large = prof["large_hits"] / steps
    visits = prof["prime_reads"] / steps
    state_writes = prof["state_writes"] / steps
    t_tile = prof["ms"][S.K_TILE] / steps * 1e-3
    t_scatter = prof["ms"][S.K_SCATTER] / steps * 1e-3
    n_tile = prof["launches"][S.K_TILE] / steps
    n_scatter = prof["launches"][S.K_SCATTER] / steps
    marks = h_medium + h_large
    # tile: table written once, each bucket entry read once; scatter (one interval):
    # each bucket entry written once; per prime and scatter group the prime (4 B) and an
    # 8-byte word read (its Barrett constant in the first group, else its state word);
    # the 8-byte state words the library counted as written back
    tile_bytes = N / 8 + 4 * h_large
    scatter_bytes = 4 * h_large + 12 * visits + 8 * state_writes
    kernels = {
        "k_tile": {"ms_per_step": t_tile * 1e3, "launches_per_step": n_tile,
                   "marks": marks, "atomics_per_s": marks / t_tile if t_tile else None,
                   "hbm_bytes": tile_bytes, "hbm_gbs": tile_bytes / t_tile / 1e9 if t_tile else None},
        "k_scatter": {"ms_per_step": t_scatter * 1e3, "launches_per_step": n_scatter,
                      "hits": h_large, "visits": visits, "state_writes": state_writes, "hbm_bytes": scatter_bytes,
                      "hbm_gbs": scatter_bytes / t_scatter / 1e9 if t_scatter else None},
    }
    traffic = load_traffic(traffic_key, N, h_large, n_tile, n_scatter)
    st_tile, st_scatter = prof_serial["ms"][S.K_TILE], prof_serial["ms"][S.K_SCATTER]
    kernels["serialised_step"] = {
        "k_tile_ms": st_tile, "k_scatter_ms": st_scatter,
        "k_tile_share": st_tile / (st_tile + st_scatter) if st_tile + st_scatter else None,
        "k_scatter_share": st_scatter / (st_tile + st_scatter) if st_tile + st_scatter else None}
    if st_tile >= st_scatter:
        ach = marks / t_tile / 1e9
        roof = {"kernel": "k_tile", "bound": "smem_atomic", "achieved": ach, "peak": r_atom / 1e9,
                "unit": "Gatomic/s", "frac": ach / (r_atom / 1e9), "traffic": traffic["k_tile"],
                "peak_source": "measured in this run (conflict-free shared atomicOr stream, "
                               "bound by the atomic unit)",
                "hbm_achieved_gbs": tile_bytes / t_tile / 1e9, "hbm_peak_gbs": hbm_peak,
                "hbm_frac": tile_bytes / t_tile / 1e9 / hbm_peak}
    else:
        ach = scatter_bytes / t_scatter / 1e9
        roof = {"kernel": "k_scatter", "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "traffic": traffic["k_scatter"],
                "peak_source": hbm_src + " (MEASURED_PEAKS.json hbm_gbs)"}
    step_roof = step_roofline(N, marks, h_large, visits, ms_max * 1e-3 / steps, hbm_peak, r_atom)
    # beside the step roofline's byte count (16 B per hit: the paper's (p, q) pair written and
    # read), the bytes this design moves: 4-byte bucket entries written and read
    b_impl = N / 8 + 8 * h_large + 12 * visits + 8 * state_writes
    step_roof["bytes_impl"] = b_impl
    step_roof["t_hbm_impl_ms"] = b_impl / (hbm_peak * 1e9) * 1e3
    return {"N": N, "ms": ms_max, "steps": steps, "value_local": N * steps / (ms * 1e-3),
            "ms_max": ms_max, "roofline": roof, "step_roofline": step_roof, "kernels": kernels,
            # kernels of the library inside the timed region: each tile and scatter launch,
            # plus the per-tile hit sum (k_sum_u32) that profiling runs after each scatter
            "clocks": clk, "launches": int(sum(prof["launches"]) + prof["launches"][S.K_SCATTER]), "out": out}


def measure_fresh(S, ctx, l, f, n, steps, host=False):
    """Throughput over fresh intervals: step k sieves (l, f + (k+1) n, n), so every
    step builds its plan (tiles, scatter groups, chunks), uploads its descriptors and
    runs it uncaptured -- the first-call cost of a new interval.  Device figure: CUDA
    events around all steps (host planning stalls the stream, so it is inside);
    host=True: the table goes to pinned host memory (sieve_segments_host) and the
    figure is wall-clock time."""
    import torch
    N = n << l
    if host:
        buf = torch.empty(N // 32, dtype=torch.int32).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(steps):
            S.sieve_segments_host(ctx, l, f + (k + 1) * n, n, buf)
        dt = time.perf_counter() - t0
        del buf
        return {"value": N * steps / dt, "ms_per_step": dt / steps * 1e3, "steps": steps}
    stream = torch.cuda.current_stream()
    out = torch.empty(N // 32, dtype=torch.int32, device="cuda")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for k in range(steps):
        S.sieve_segments(ctx, l, f + (k + 1) * n, n, out)
    ev1.record(stream)
    torch.cuda.synchronize()
    S.sieve_sync(ctx)
    ms = ev0.elapsed_time(ev1)
    del out
    return {"value": N * steps / (ms * 1e-3), "ms_per_step": ms / steps, "steps": steps}


def measure_consumers(S, ctx, l, f, n, steps):
    """The consumers fused with the table (Sec. 5 uses of the sieve), each timed with CUDA
    events after 3 warm-up calls:
      count: per-segment prime and twin-pair counts of the workload interval without
             writing its table (sieve_count_segments), odd numbers/s;
      goldbach: the smallest-partition search for 2^30 consecutive even numbers around
             10^18 on their table (sieve_segments of the odd numbers from N - p_max to
             N - 3, then sieve_goldbach), even numbers/s for the search alone and with
             the table's sieving."""
    import torch
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pr = torch.empty(n, dtype=torch.int64, device="cuda")
    tw = torch.empty(n, dtype=torch.int64, device="cuda")
    for _ in range(3):
        S.sieve_count_segments(ctx, l, f, n, pr, tw)
    S.sieve_sync(ctx)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        S.sieve_count_segments(ctx, l, f, n, pr, tw)
    ev1.record(stream)
    torch.cuda.synchronize()
    S.sieve_sync(ctx)
    t_count = ev0.elapsed_time(ev1) * 1e-3 / steps
    count = {"value": (n << l) / t_count, "unit": "odd numbers/s", "ms_per_step": t_count * 1e3,
             "primes": int(pr.sum().item()), "twin_pairs": int(tw.sum().item())}
    del pr, tw

    # Goldbach around 1e18: N = n_lo + 2i, i < 2^30; table from N_lo - p_max up
    lg, cnt, p_max, win = 20, 1 << 30, 1 << 15, 20
    n_lo = 10**18
    lo_j = (n_lo - p_max - 1) // 2
    hi_j = (n_lo + 2 * cnt) // 2
    gf = lo_j >> lg
    gn = (hi_j >> lg) + 1 - gf
    tab = torch.empty((gn << lg) // 32, dtype=torch.int32, device="cuda")
    nwin = ((cnt - 1) >> win) + 1
    wins = torch.empty(2 * nwin, dtype=torch.int64, device="cuda")
    for _ in range(3):
        S.sieve_segments(ctx, lg, gf, gn, tab)
        S.sieve_goldbach(ctx, tab, gf << lg, gn << lg, n_lo, cnt, p_max, win, wins)
    S.sieve_sync(ctx)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        S.sieve_goldbach(ctx, tab, gf << lg, gn << lg, n_lo, cnt, p_max, win, wins)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_gb = ev0.elapsed_time(ev1) * 1e-3 / steps
    ev0.record(stream)
    for _ in range(steps):
        S.sieve_segments(ctx, lg, gf, gn, tab)
        S.sieve_goldbach(ctx, tab, gf << lg, gn << lg, n_lo, cnt, p_max, win, wins)
    ev1.record(stream)
    torch.cuda.synchronize()
    S.sieve_sync(ctx)
    t_both = ev0.elapsed_time(ev1) * 1e-3 / steps
    dec = S.goldbach_windows(wins.cpu().tolist(), n_lo, win)
    top = max(dec, key=lambda x: (x[0], -(x[1] or 0)))
    gold = {"value": cnt / t_gb, "unit": "even numbers/s", "ms_per_step": t_gb * 1e3,
            "with_sieve": cnt / t_both, "with_sieve_ms": t_both * 1e3, "n_lo": n_lo, "count": cnt,
            "p_max": p_max, "max_min_p": top[0], "at": top[1], "failures": sum(x[2] for x in dec)}
    del tab, wins
    torch.cuda.empty_cache()
    return {"count": count, "goldbach": gold}


def measure_stream(S, ctx, hbm_peak, r_atom, k=8):
    """A long range sieved as k consecutive intervals of 2^30 bits (l = 20, n = 1024), the
    paper's segment-after-segment mode, at 1e15 and 1e18: with streaming on, each interval
    continues from the previous one's large-prime state (no first hits for them); off,
    every interval computes them.  Plans are built in an untimed first pass; then the k
    intervals are timed with CUDA events (the first of them starts a new chain), with the
    step roofline of the streamed form."""
    import torch
    l, n = 20, 1024
    N = n << l
    out = torch.empty(N // 32, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    res = {}
    for e in (15, 18):
        f0 = S.sieve_f_from_midpoint(l, n, 1, e)
        row = {}
        for mode in ("off", "on"):
            S.sieve_set_streaming(ctx, mode == "on")
            for j in range(k):
                S.sieve_segments(ctx, l, f0 + j * n, n, out)
            S.sieve_sync(ctx)
            S.sieve_profile_enable(ctx, mode == "on")
            S.sieve_profile_read(ctx)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for j in range(k):
                S.sieve_segments(ctx, l, f0 + j * n, n, out)
            e1.record(stream)
            torch.cuda.synchronize()
            prof = S.sieve_profile_read(ctx)
            S.sieve_profile_enable(ctx, False)
            S.sieve_sync(ctx)
            t = e0.elapsed_time(e1) * 1e-3 / k
            row[mode] = {"ms": t * 1e3, "value": N / t}
            if mode == "on":
                J0 = f0 << l
                tune = S.sieve_get_tuning(ctx, 1 if e == 15 else 3)
                h_large = prof["large_hits"] / k
                roof = step_roofline(N, medium_marks(J0, N, tune) + h_large, h_large, prof["prime_reads"] / k, t,
                                     hbm_peak, r_atom)
                row["on"]["step_roofline_frac"] = roof["frac"]
                row["on"]["continued_primes_per_interval"] = prof["continued"] / k
        S.sieve_set_streaming(ctx, False)
        res["1e%d" % e] = row
    del out
    return {"l": l, "n": n, "intervals": k, "unit": "odd numbers/s", "points": res}


def measure_batch(S, ctx, args, rank, world, hbm_peak, r_atom):
    """args.batch_requests (4096) seeded requests of uneven length (2^16..2^28 numbers) and magnitude
    (1e6..1e18): the batched form (one graph-replayed launch sequence) against the
    plain form (one sieve_segments call per request), same outputs (every request's
    count compared), same GPU, with the batched form's step roofline.  Under torchrun
    each rank takes its share of one seeded request list (shard.partition_requests)."""
    import numpy as np
    import torch
    from paper_1111_3297_gb300 import shard, workloads
    allreqs = workloads.batch_requests(args.batch_requests, seed=0)
    mine = shard.partition_requests(allreqs, rank, world)
    reqs = [allreqs[i] for i in mine]
    lay, off = [], 0
    for j0, nb in reqs:
        lay.append((j0, nb, off))
        off += (nb // 32 + 3) // 4 * 4
    bits = sum(nb for _, nb in reqs)
    arena = torch.empty(off, dtype=torch.int32, device="cuda")
    counts = torch.empty(len(reqs), dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    tuned = S.sieve_autotune_batch(ctx, lay, arena, counts) if not args.no_autotune else None
    t_tune = time.perf_counter() - t0
    for _ in range(3):
        S.sieve_batch(ctx, lay, arena, counts)
    S.sieve_sync(ctx)
    ksteps = max(2, min(args.steps, 5))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(ksteps):
        S.sieve_batch(ctx, lay, arena, counts)
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) * 1e-3 / ksteps
    ref = counts.cpu().clone()
    # one more (untimed) call with profiling on: exact large-prime hits and visits
    S.sieve_profile_enable(ctx, True)
    S.sieve_profile_read(ctx)
    S.sieve_batch(ctx, lay, arena, counts)
    prof = S.sieve_profile_read(ctx)
    S.sieve_profile_enable(ctx, False)
    S.sieve_sync(ctx)
    # plain: one call per request into the same arena slots
    for j0, nb, o in lay:
        S.sieve_segments(ctx, 5, j0 // 32, nb // 32, arena[o:o + nb // 32])
    S.sieve_sync(ctx)
    torch.cuda.synchronize()
    e0.record(stream)
    for j0, nb, o in lay:
        S.sieve_segments(ctx, 5, j0 // 32, nb // 32, arena[o:o + nb // 32])
    e1.record(stream)
    torch.cuda.synchronize()
    t_plain = e0.elapsed_time(e1) * 1e-3
    same = all(S.sieve_count(ctx, arena[o:o + nb // 32], nb) == int(c)
               for (j0, nb, o), c in zip(lay, ref.tolist()))
    # roofline of the batched form: per request its wheel-reduced medium marks, plus the
    # large-prime hits and (prime, unit) first-hit visits the library counted
    vmax = max(2 * (j0 + nb - 1) + 1 for j0, nb in reqs)
    tune = tuned or S.sieve_get_tuning(ctx, 0 if vmax < 2**40 else 1 if vmax < 2**50 else 2 if vmax < 2**56 else 3)
    h_med = batch_medium_marks(reqs, {"medium_max": tune["medium_max"], "presieve_groups": tune["presieve_groups"]},
                               world)
    h_large, visits = prof["large_hits"], prof["prime_reads"]
    roof = step_roofline(bits, h_med + h_large, h_large, visits, t_batch, hbm_peak, r_atom)
    roof["first_hit_visits_per_s"] = visits / t_batch
    roof["note"] = ("the multi-request scatter is bound by its (prime, unit) first-hit visits: "
                    "Barrett reduction and wheel start per visit, issue-bound (see DESIGN)")
    del arena, counts
    torch.cuda.empty_cache()
    return {"requests": len(reqs), "requests_all_ranks": len(allreqs), "odd_numbers": bits,
            "batched": bits / t_batch, "plain": bits / t_plain,
            "unit": "odd numbers/s", "speedup": t_plain / t_batch, "batched_ms": t_batch * 1e3,
            "plain_ms": t_plain * 1e3, "same_counts_all": same, "tuning": tuned,
            "autotune_s": t_tune, "roofline": roof}


def serve_at(S, ctx, rate, count, rank, seed=0):
    """Seeded Poisson arrivals at `rate` requests/s of `count` requests drawn as in the
    batch, admission capped by 64 GB of device memory; latency (submit -> done) and
    sustained odd numbers/s, and the requests in the system (submitted, not yet done)."""
    from paper_1111_3297_gb300 import workloads
    reqs = workloads.batch_requests(count, seed=100 + seed + rank)
    arrivals = workloads.poisson_arrivals(count, rate, seed=seed + rank)
    srv = S.Server(ctx, mem_cap=64 << 30, max_inflight=4)
    lat, done_bits, first, last = [], 0, None, 0.0
    depth_max, depth_sum, depth_n = 0, 0, 0
    try:
        i = 0
        t_start = srv.now()
        pending = 0
        while i < count or pending:
            now = srv.now() - t_start
            while i < count and arrivals[i] <= now:
                srv.submit(*reqs[i])
                pending += 1
                i += 1
            depth_max = max(depth_max, pending)
            depth_sum += pending
            depth_n += 1
            for r in srv.poll(1024, timeout_ms=0 if i < count else 50):
                if r["status"] != 0:
                    raise RuntimeError("served request failed with status %d" % r["status"])
                lat.append(r["t_done"] - r["t_submit"])
                done_bits += r["nbits"]
                first = r["t_submit"] if first is None else min(first, r["t_submit"])
                last = max(last, r["t_done"])
                srv.release(r["id"])
                pending -= 1
            if i < count:
                nxt = arrivals[i] - (srv.now() - t_start)
                if nxt > 0.0002:
                    time.sleep(min(nxt, 0.001))
    finally:
        srv.close()
    lat.sort()
    q = lambda x: lat[min(len(lat) - 1, int(x * len(lat)))]  # noqa: E731
    return {"requests": count, "rate_per_s": rate, "p50_ms": q(0.50) * 1e3, "p99_ms": q(0.99) * 1e3,
            "max_ms": lat[-1] * 1e3, "sustained": done_bits / (last - first), "unit": "odd numbers/s",
            "offered": sum(nb for _, nb in reqs) / arrivals[-1], "in_system_max": depth_max,
            "in_system_mean": depth_sum / max(1, depth_n), "mem_cap_gb": 64, "lanes": 4}


def measure_serving(S, ctx, args, rank):
    """The serving configuration (2000 requests/s for args.serve_seconds), then a
    saturating sweep of arrival rates up to past the server's capacity, each rate for
    a few seconds of arrivals."""
    main = serve_at(S, ctx, 2000.0, int(2000.0 * args.serve_seconds), rank)
    sweep = []
    if args.serve_sweep_seconds > 0:
        for rate in (2000.0, 8000.0, 20000.0, 50000.0, 120000.0):
            r = serve_at(S, ctx, rate, int(rate * args.serve_sweep_seconds), rank, seed=7)
            sweep.append({k: r[k] for k in ("rate_per_s", "requests", "p50_ms", "p99_ms", "sustained", "offered",
                                            "in_system_max", "in_system_mean")})
    main["sweep"] = sweep
    return main


def main():
    args = parse()
    rank, world, local = dist_env()
    wl = WORKLOADS.get(args.workload)
    if args.impl == "reference":
        if world > 1 and rank != 0:
            return
        run_reference(args, rank, world, wl)
        return

    import torch
    from paper_1111_3297_gb300 import build
    build.build_library()
    from paper_1111_3297_gb300 import sieve as S

    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist

    from paper_1111_3297_gb300 import shard
    l, n = wl["l"], wl["n"]
    if args.segments:
        n = args.segments
    f0 = wl.get("f")
    if f0 is None:
        f0 = S.sieve_f_from_midpoint(l, n, wl["mant"], wl["exp10"])
    f, _ = shard.shard(l, f0, n, rank, world, "weak")  # each rank its own n segments
    N = n << l
    vmax = 2 * ((f0 + world * n) << l)
    c3_on = args.workload == "c2" and not args.no_c3 and not args.segments
    # the batch and serving legs draw requests up to ~1e18, the Goldbach leg works just
    # above 1e18, the 2^60 sub-record sieves up to 2^60 + 2^35
    wide = not (args.no_batch and args.no_serve and args.no_sweep and args.no_consumers) or c3_on
    # the fresh-interval legs sieve the next 2 * fresh_steps intervals after this rank's
    vmax_fresh = 2 * ((f0 + world * n + 2 * (args.fresh_steps + 1) * n) << l)
    ctx = S.sieve_init(local, max_v=max(vmax_fresh, 2 * 10**18 + (1 << 31)) if wide else vmax_fresh)

    tuned = None
    if args.tuning:
        tuned = json.loads(args.tuning)
        for k in range(4):
            S.sieve_set_tuning(ctx, k, **tuned)
    elif not args.no_autotune:
        tuned = S.sieve_autotune(ctx, l, f, n)
    r_atom = S.sieve_probe_smem_atomics(local)
    dsmem = {}
    for c in (2, 4, 8):
        own, ctas = S.sieve_probe_dsmem_atomics(local, c, peer=False)
        peer, _ = S.sieve_probe_dsmem_atomics(local, c, peer=True)
        dsmem["cluster%d" % c] = {"own_slice_per_s": own, "peer_slice_per_s": peer, "ctas": ctas}
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    cls = 0 if vmax < 2**40 else 1 if vmax < 2**50 else 2 if vmax < 2**56 else 3
    tune = tuned or S.sieve_get_tuning(ctx, cls)

    m = measure_interval(S, ctx, l, f, n, args.steps, args.warmup, tune, hbm_peak, hbm_src, r_atom,
                         {"c2": "l20_n1024_mid1e15", "c3": "l20_n4096_mid2p60", "m1e18": "l20_n1024_mid1e18"}.get(args.workload), pg,
                         args.clocks_csv)
    out = m.pop("out")
    ms_max = m["ms_max"]
    value = job_value(world, N, args.steps, ms_max)
    composites = shard.total_count(S.sieve_count(ctx, out, N))
    del out
    torch.cuda.empty_cache()

    # ---- end to end: the table delivered to pinned host memory ----
    e2e = None
    if not args.no_e2e:
        host = torch.empty(N // 32, dtype=torch.int32).pin_memory()
        S.sieve_segments_host(ctx, l, f, n, host)  # warm (plans, staging)
        if pg:
            pg.barrier()
        t0 = time.perf_counter()
        ksteps = max(1, min(args.steps, 5))
        for _ in range(ksteps):
            S.sieve_segments_host(ctx, l, f, n, host)
        dt = max_over_ranks(pg, time.perf_counter() - t0)
        # inputs are the call's three scalars (l, f, n); the plan's descriptors were
        # uploaded by the warm-up call and stay cached with its graph
        e2e = {"value": world * N * ksteps / dt, "unit": "odd numbers/s", "h2d_bytes_per_step": 24,
               "d2h_bytes_per_step": N // 8, "steps": ksteps,
               "inputs": "three 8-byte scalars (l, f, n) passed by value; plan descriptors cached"}
        del host

    # ---- fresh intervals: plan building, descriptor upload inside every step ----
    fresh = None
    if args.fresh_steps > 0 and rank == 0:
        fresh = {"device": measure_fresh(S, ctx, l, f, n, args.fresh_steps),
                 "e2e": measure_fresh(S, ctx, l, f + args.fresh_steps * n, n, args.fresh_steps, host=True),
                 "note": "step k sieves (l, f + (k+1) n, n): every step a new interval, its plan built, "
                         "uploaded and run uncaptured"}

    # ---- the 2^60 configuration (l = 20, n = 32768) as a sub-record ----
    c3 = None
    if c3_on and rank == 0:
        w3 = WORKLOADS["c3"]
        f3 = S.sieve_f_from_midpoint(w3["l"], w3["n"], w3["mant"], w3["exp10"])
        t3 = S.sieve_get_tuning(ctx, 3)
        k3 = min(args.steps, 5)
        m3 = measure_interval(S, ctx, w3["l"], f3, w3["n"], k3, 3, t3, hbm_peak, hbm_src, r_atom,
                              "l20_n4096_mid2p60")
        out3 = m3.pop("out")
        m3["composites"] = S.sieve_count(ctx, out3, m3["N"])
        del out3
        torch.cuda.empty_cache()
        c3 = {"config": {"workload": w3["name"], "l": w3["l"], "f": f3, "n": w3["n"], "tuning": t3,
                         "l2": "table 4096 MiB + buckets, larger than L2"},
              "value": m3["value_local"], "unit": "odd numbers/s", "ms_per_step": m3["ms"] / k3,
              "steps": k3, "warmup": 3, **{k: m3[k] for k in ("roofline", "step_roofline", "kernels",
                                                             "clocks", "composites")}}

    consumers = None
    if rank == 0 and not args.no_consumers:
        consumers = measure_consumers(S, ctx, l, f, n, max(2, min(args.steps, 5)))

    sweep = None
    streamed = None
    if rank == 0 and not args.no_sweep:
        sweep = measure_sweep(S, ctx, hbm_peak, r_atom)
        streamed = measure_stream(S, ctx, hbm_peak, r_atom)

    base_line = None
    if rank == 0 and not args.no_cpu_baseline:
        base_line = cpu_baseline(dict(wl, n=n), f0)
    batch = None
    if not args.no_batch:
        batch = measure_batch(S, ctx, args, rank, world, hbm_peak, r_atom)
    serving = None
    if not args.no_serve:
        serving = measure_serving(S, ctx, args, rank)

    if rank == 0:
        print(json.dumps({
            "metric": "odd numbers sieved/s", "value": value, "unit": "odd numbers/s",
            "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": wl["name"], "l": l, "f": f0, "n": n, "parallelism": "interval shards x%d" % world,
                       "l2": "working set larger than L2 (table %d MiB + buckets)" % (N // 8 // 2**20),
                       "tuning": tune},
            "gpu_launches": m["launches"],
            "roofline": m["roofline"], "step_roofline": m["step_roofline"], "kernels": m["kernels"],
            "cpu_baseline": base_line, "e2e": e2e, "fresh": fresh, "clocks": m["clocks"],
            "c3": c3, "consumers": consumers, "streaming": streamed, "batch": batch, "serving": serving, "sweep": sweep,
            "composites": composites, "smem_atomic_peak_per_s": r_atom, "dsmem_probe": dsmem,
        }), flush=True)
    ctx.close()
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
