"""Python binding of libgbsieve.so (include/gbsieve.h): argument marshalling only.

Every function has the C name and forwards to the C ABI; all sieving runs in
the library's CUDA kernels.  Device buffers are torch CUDA tensors (int32 words,
bit j = bit j%32 of word j//32), streams are torch.cuda.Stream objects (default:
the current stream).  There is no CPU fallback: if the library is missing or
fails to load, every call raises.
"""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_PKG, "libgbsieve.so")
_lib = None

_u32, _u64, _i32, _vp, _dbl = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p, ctypes.c_double

STATUS = {0: "SIEVE_OK", 1: "SIEVE_EINVAL", 2: "SIEVE_ERANGE", 3: "SIEVE_ENOMEM", 4: "SIEVE_ECUDA",
          5: "SIEVE_ETIMEOUT", 6: "SIEVE_EBUSY", 7: "SIEVE_EOVERFLOW"}

K_TILE, K_SCATTER, K_COUNT, K_RESET, K_COPY = 0, 1, 2, 3, 4


class SieveError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = "%s: %s (%s)" % (where, STATUS.get(status, status), lib().sieve_strerror(status).decode())
        if status == 4:  # SIEVE_ECUDA: name the failed runtime call
            msg += ": " + lib().sieve_last_cuda_error().decode(errors="replace")
        super().__init__(msg)


class Tuning(ctypes.Structure):
    _fields_ = [("tile_log2", _u32), ("presieve_groups", _u32), ("coop_max", _u32),
                ("medium_max", _u32), ("window_tiles", _u32), ("epoch_tiles", _u32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Req(ctypes.Structure):
    _fields_ = [("j0", _u64), ("nbits", _u64), ("out_word_off", _u64)]


class Profile(ctypes.Structure):
    _fields_ = [("launches", _u64 * 8), ("ms", _dbl * 8), ("tiles", _u64), ("bits", _u64),
                ("large_hits", _u64), ("medium_marks", _u64), ("prime_reads", _u64), ("continued", _u64),
                ("state_writes", _u64)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("ntiles", _u64), ("ngroups", _u64), ("nepochs", _u64), ("nchunks", _u64), ("nunits", _u64),
                ("bits", _u64), ("pool_entries", _u64), ("carry_entries", _u64), ("max_epoch_tiles", _u32),
                ("big_wheel", _u32), ("run_scatter", _u32), ("carried_groups", _u32), ("med_lo", _u32),
                ("blk_hi", _u32), ("coop_hi", _u32), ("large_lo", _u32), ("expected_large_hits", _dbl)]


class PlanTile(ctypes.Structure):
    _fields_ = [("j0", _u64), ("out_word", _u64), ("bkt_off", _u64), ("len", _u32), ("req", _u32),
                ("epoch", _u32), ("group", _u32), ("bkt_cap", _u32), ("med_hi", _u32)]


class PlanGroup(ctypes.Structure):
    _fields_ = [("epoch", _u32), ("tile0", _u32), ("ntiles", _u32), ("nunits", _u32), ("p_lo", _u32),
                ("p_hi", _u32), ("carry_in", _u32), ("carry_out", _u32)]


class PlanChunk(ctypes.Structure):
    _fields_ = [("epoch", _u32), ("p_lo", _u32), ("p_hi", _u32)]


def _rec(x):
    return {k: getattr(x, k) for k, _ in x._fields_}


class Result(ctypes.Structure):
    _fields_ = [("id", _u64), ("j0", _u64), ("nbits", _u64), ("composites", _u64),
                ("dev_bits", _vp), ("t_submit", _dbl), ("t_admit", _dbl), ("t_done", _dbl),
                ("status", _i32)]


def lib():
    """Load libgbsieve.so (raises if it is not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIBPATH):
            raise RuntimeError("libgbsieve.so is not built (run __graft_entry__.build())")
        L = ctypes.CDLL(_LIBPATH)
        sig = {
            "sieve_strerror": (ctypes.c_char_p, [_i32]),
            "sieve_last_cuda_error": (ctypes.c_char_p, []),
            "sieve_init": (_i32, [ctypes.POINTER(_vp), _i32, _u64, ctypes.c_size_t]),
            "sieve_destroy": (None, [_vp]),
            "sieve_segments": (_i32, [_vp, _u32, _u64, _u64, _vp, _vp]),
            "sieve_f_from_midpoint": (_i32, [_u32, _u64, _u64, _u32, ctypes.POINTER(_u64)]),
            "sieve_segments_midpoint": (_i32, [_vp, _u32, _u64, _u32, _u64, _vp, _vp]),
            "sieve_segments_host": (_i32, [_vp, _u32, _u64, _u64, _vp, _vp]),
            "sieve_count_segments": (_i32, [_vp, _u32, _u64, _u64, _vp, _vp, _vp]),
            "sieve_goldbach": (_i32, [_vp, _vp, _u64, _u64, _u64, _u64, _u32, _u32, _vp, _vp]),
            "sieve_count": (_i32, [_vp, _vp, _u64, ctypes.POINTER(_u64), _vp]),
            "sieve_sync": (_i32, [_vp, _vp]),
            "sieve_set_streaming": (_i32, [_vp, _i32]),
            "sieve_batch": (_i32, [_vp, ctypes.POINTER(Req), _u32, _vp, _vp, _vp]),
            "sieve_get_tuning": (_i32, [_vp, _u32, ctypes.POINTER(Tuning)]),
            "sieve_set_tuning": (_i32, [_vp, _u32, ctypes.POINTER(Tuning)]),
            "sieve_autotune": (_i32, [_vp, _u32, _u64, _u64, ctypes.POINTER(Tuning), _vp]),
            "sieve_autotune_batch": (_i32, [_vp, ctypes.POINTER(Req), _u32, _vp, _vp,
                                            ctypes.POINTER(Tuning), _vp]),
            "sieve_base_info": (_i32, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_u64), ctypes.POINTER(_u64)]),
            "sieve_profile_enable": (_i32, [_vp, _i32]),
            "sieve_profile_read": (_i32, [_vp, ctypes.POINTER(Profile), _vp]),
            "sieve_probe_smem_atomics": (_i32, [_i32, ctypes.POINTER(_dbl)]),
            "sieve_probe_dsmem_atomics": (_i32, [_i32, _u32, _i32, ctypes.POINTER(_dbl), ctypes.POINTER(_u32)]),
            "sieve_plan_describe": (_i32, [_vp, _u64, _u64, _u32, ctypes.POINTER(Req), _u32,
                                           ctypes.POINTER(Tuning), _u64, ctypes.POINTER(PlanInfo),
                                           ctypes.POINTER(PlanTile), _u64, ctypes.POINTER(PlanGroup), _u64,
                                           ctypes.POINTER(PlanChunk), _u64]),
            "sieve_server_create": (_i32, [_vp, ctypes.c_size_t, _u32, ctypes.POINTER(_vp)]),
            "sieve_server_submit": (_i32, [_vp, _u64, _u64, ctypes.POINTER(_u64)]),
            "sieve_server_poll": (_i32, [_vp, ctypes.POINTER(Result), _u32, ctypes.POINTER(_u32), _u32]),
            "sieve_server_release": (_i32, [_vp, _u64]),
            "sieve_server_now": (_dbl, [_vp]),
            "sieve_server_destroy": (None, [_vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(st, where):
    if st != 0:
        raise SieveError(st, where)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return _vp(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _nbytes(t):
    return t.numel() * t.element_size() if hasattr(t, "element_size") else t.nbytes


def _dev_ptr(t, what, need=0):
    """Device address of a contiguous CUDA tensor holding at least `need` bytes (the
    library takes plain pointers and cannot see the size: a short buffer would be
    written past its end)."""
    if not (hasattr(t, "is_cuda") and t.is_cuda):
        raise TypeError("%s must be a CUDA tensor" % what)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    if _nbytes(t) < need:
        raise ValueError("%s holds %d bytes, the call needs %d" % (what, _nbytes(t), need))
    return _vp(t.data_ptr())


def _table_bytes(l, n):
    return (int(n) << int(l)) // 8 if 0 <= int(l) < 64 else 0


def _batch_bytes(reqs):
    return max([(int(r[2]) + int(r[1]) // 32) * 4 for r in reqs] or [0])


class Ctx:
    """A context (resident base primes and scratch) on one device."""

    def __init__(self, handle, device):
        self.handle = handle
        self.device = device

    def close(self):
        if self.handle:
            lib().sieve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sieve_init(device=0, max_v=(1 << 62), mem_budget=0):
    h = _vp()
    _check(lib().sieve_init(ctypes.byref(h), device, max_v, mem_budget), "sieve_init")
    return Ctx(h, device)


def sieve_destroy(ctx):
    ctx.close()


def sieve_segments(ctx, l, f, n, dev_bits, stream=None):
    _check(lib().sieve_segments(ctx.handle, l, f, n, _dev_ptr(dev_bits, "dev_bits", _table_bytes(l, n)),
                                _stream(stream)),
           "sieve_segments")


def sieve_count_segments(ctx, l, f, n, dev_primes, dev_twins=None, stream=None):
    """Per-segment prime counts (and twin-pair counts when dev_twins is given) of the
    interval (l, f, n), without writing its table: CUDA int64 tensors of n entries."""
    _check(lib().sieve_count_segments(ctx.handle, l, f, n, _dev_ptr(dev_primes, "dev_primes", 8 * n),
                                      _dev_ptr(dev_twins, "dev_twins", 8 * n) if dev_twins is not None else None,
                                      _stream(stream)), "sieve_count_segments")


def sieve_goldbach(ctx, dev_bits, j0, nbits, n_lo, count, p_max, win_log2, dev_windows, stream=None):
    """Goldbach search on the table dev_bits (bits j0 .. j0+nbits-1) for the even numbers
    n_lo + 2i, i < count: dev_windows is a CUDA int64 tensor of 2 * ceil(count / 2^win_log2)
    entries (key, failures per window; decode with goldbach_windows)."""
    nwin = ((int(count) - 1) >> int(win_log2)) + 1 if count > 0 else 0
    _check(lib().sieve_goldbach(ctx.handle, _dev_ptr(dev_bits, "dev_bits", int(nbits) // 8), j0, nbits, n_lo,
                                count, p_max, win_log2, _dev_ptr(dev_windows, "dev_windows", 16 * nwin),
                                _stream(stream)), "sieve_goldbach")


def goldbach_windows(windows, n_lo, win_log2):
    """Decode sieve_goldbach's output (a host sequence of 2 * nwin int64): per window
    (largest minimal p, the first even N attaining it, failures); (0, None, f) for a
    window in which no N has a p."""
    out = []
    w = [int(x) & 0xFFFFFFFFFFFFFFFF for x in windows]
    for k in range(len(w) // 2):
        key, fail = w[2 * k], w[2 * k + 1]
        if key == 0:
            out.append((0, None, fail))
            continue
        off = 0xFFFFFFFF - (key & 0xFFFFFFFF)
        out.append((key >> 32, int(n_lo) + 2 * ((k << int(win_log2)) + off), fail))
    return out


def sieve_f_from_midpoint(l, n, mant, exp10):
    out = _u64()
    _check(lib().sieve_f_from_midpoint(l, n, mant, exp10, ctypes.byref(out)), "sieve_f_from_midpoint")
    return out.value


def sieve_segments_midpoint(ctx, l, mant, exp10, n, dev_bits, stream=None):
    _check(lib().sieve_segments_midpoint(ctx.handle, l, mant, exp10, n, _dev_ptr(dev_bits, "dev_bits", _table_bytes(l, n)),
                                         _stream(stream)), "sieve_segments_midpoint")


def sieve_segments_host(ctx, l, f, n, host_bits, stream=None):
    """host_bits: a CPU torch tensor or numpy array of n*2^(l-5) 32-bit words."""
    if hasattr(host_bits, "data_ptr"):
        if host_bits.is_cuda or not host_bits.is_contiguous():
            raise TypeError("host_bits must be a contiguous CPU tensor")
        ptr = host_bits.data_ptr()
    else:
        if not host_bits.flags["C_CONTIGUOUS"]:
            raise TypeError("host_bits must be a contiguous array")
        ptr = host_bits.ctypes.data
    if _nbytes(host_bits) < _table_bytes(l, n):
        raise ValueError("host_bits holds %d bytes, the call needs %d" % (_nbytes(host_bits), _table_bytes(l, n)))
    _check(lib().sieve_segments_host(ctx.handle, l, f, n, _vp(ptr), _stream(stream)), "sieve_segments_host")


def sieve_count(ctx, dev_bits, nbits, stream=None):
    out = _u64()
    _check(lib().sieve_count(ctx.handle, _dev_ptr(dev_bits, "dev_bits", int(nbits) // 8), nbits, ctypes.byref(out),
                             _stream(stream)), "sieve_count")
    return out.value


def sieve_set_streaming(ctx, enable=True):
    """Consecutive single-interval calls continue from each other's large-prime state."""
    _check(lib().sieve_set_streaming(ctx.handle, 1 if enable else 0), "sieve_set_streaming")


def sieve_sync(ctx, stream=None):
    _check(lib().sieve_sync(ctx.handle, _stream(stream)), "sieve_sync")


def _reqs(reqs):
    arr = (Req * len(reqs))()
    for i, r in enumerate(reqs):
        arr[i].j0, arr[i].nbits, arr[i].out_word_off = int(r[0]), int(r[1]), int(r[2])
    return arr


def sieve_batch(ctx, reqs, dev_arena, dev_counts, stream=None):
    """reqs: sequence of (j0, nbits, out_word_off); dev_counts: CUDA int64 tensor (len(reqs),)."""
    arr = _reqs(reqs)
    _check(lib().sieve_batch(ctx.handle, arr, len(reqs), _dev_ptr(dev_arena, "dev_arena", _batch_bytes(reqs)),
                             _dev_ptr(dev_counts, "dev_counts", 8 * len(reqs)), _stream(stream)), "sieve_batch")


def sieve_get_tuning(ctx, cls):
    t = Tuning()
    _check(lib().sieve_get_tuning(ctx.handle, cls, ctypes.byref(t)), "sieve_get_tuning")
    return t.as_dict()


def sieve_set_tuning(ctx, cls, **kw):
    t = Tuning()
    _check(lib().sieve_get_tuning(ctx.handle, cls, ctypes.byref(t)), "sieve_get_tuning")
    for k, v in kw.items():
        setattr(t, k, v)
    _check(lib().sieve_set_tuning(ctx.handle, cls, ctypes.byref(t)), "sieve_set_tuning")


def sieve_autotune(ctx, l, f, n, stream=None):
    t = Tuning()
    _check(lib().sieve_autotune(ctx.handle, l, f, n, ctypes.byref(t), _stream(stream)), "sieve_autotune")
    return t.as_dict()


def sieve_autotune_batch(ctx, reqs, dev_arena, dev_counts, stream=None):
    t = Tuning()
    arr = _reqs(reqs)
    _check(lib().sieve_autotune_batch(ctx.handle, arr, len(reqs), _dev_ptr(dev_arena, "dev_arena", _batch_bytes(reqs)),
                                      _dev_ptr(dev_counts, "dev_counts", 8 * len(reqs)), ctypes.byref(t),
                                      _stream(stream)),
           "sieve_autotune_batch")
    return t.as_dict()


def sieve_base_info(ctx):
    p, c, lim = _vp(), _u64(), _u64()
    _check(lib().sieve_base_info(ctx.handle, ctypes.byref(p), ctypes.byref(c), ctypes.byref(lim)),
           "sieve_base_info")
    return p.value, c.value, lim.value


def sieve_profile_enable(ctx, enable=True, serial=False):
    _check(lib().sieve_profile_enable(ctx.handle, (2 if serial else 1) if enable else 0), "sieve_profile_enable")


def sieve_profile_read(ctx, stream=None):
    p = Profile()
    _check(lib().sieve_profile_read(ctx.handle, ctypes.byref(p), _stream(stream)), "sieve_profile_read")
    return {"launches": list(p.launches), "ms": list(p.ms), "tiles": p.tiles, "bits": p.bits,
            "large_hits": p.large_hits, "medium_marks": p.medium_marks, "prime_reads": p.prime_reads,
            "continued": p.continued, "state_writes": p.state_writes}


def sieve_probe_smem_atomics(device=0):
    r = _dbl()
    _check(lib().sieve_probe_smem_atomics(device, ctypes.byref(r)), "sieve_probe_smem_atomics")
    return r.value


def sieve_probe_dsmem_atomics(device=0, cluster_size=2, peer=True):
    """(ORs per second, CTAs that ran) of the distributed shared memory probe."""
    r, n = _dbl(), _u32()
    _check(lib().sieve_probe_dsmem_atomics(device, cluster_size, 1 if peer else 0, ctypes.byref(r), ctypes.byref(n)),
           "sieve_probe_dsmem_atomics")
    return r.value, n.value


def sieve_plan_describe(primes, max_v, nsm, reqs, tuning=None, pool_entries=1 << 31, records=True):
    """The plan sieve_batch builds for reqs ((j0, nbits, out_word_off) each), on the host
    without a device, from the base `primes` (all odd primes <= isqrt(max_v), ascending).
    tuning: dict of sieve_tuning fields, or None for the class default.  Returns
    {"info": {...}} plus, with records, lists "tiles", "groups" and "chunks" of dicts."""
    import numpy as np
    pr = np.ascontiguousarray(primes, dtype=np.uint32)
    arr = _reqs(reqs)
    tp = None
    if tuning is not None:
        t = Tuning(**tuning)
        tp = ctypes.byref(t)
    info = PlanInfo()
    L = lib()

    def call(tiles, nt, groups, ng, chunks, nc):
        _check(L.sieve_plan_describe(pr.ctypes.data_as(_vp), len(pr), max_v, nsm, arr, len(reqs), tp,
                                     pool_entries, ctypes.byref(info), tiles, nt, groups, ng, chunks, nc),
               "sieve_plan_describe")
    call(None, 0, None, 0, None, 0)
    out = {"info": _rec(info)}
    if records:
        tiles = (PlanTile * info.ntiles)()
        groups = (PlanGroup * info.ngroups)()
        chunks = (PlanChunk * info.nchunks)()
        call(tiles, info.ntiles, groups, info.ngroups, chunks, info.nchunks)
        out["tiles"] = [_rec(x) for x in tiles]
        out["groups"] = [_rec(x) for x in groups]
        out["chunks"] = [_rec(x) for x in chunks]
    return out


class Server:
    """Continuous-batching request loop (sieve_server_*)."""

    def __init__(self, ctx, mem_cap, max_inflight=4):
        self.ctx = ctx  # keeps the context alive
        h = _vp()
        _check(lib().sieve_server_create(ctx.handle, mem_cap, max_inflight, ctypes.byref(h)), "sieve_server_create")
        self.handle = h

    def submit(self, j0, nbits):
        out = _u64()
        _check(lib().sieve_server_submit(self.handle, j0, nbits, ctypes.byref(out)), "sieve_server_submit")
        return out.value

    def poll(self, max_results=256, timeout_ms=0):
        buf = (Result * max_results)()
        n = _u32()
        _check(lib().sieve_server_poll(self.handle, buf, max_results, ctypes.byref(n), timeout_ms),
               "sieve_server_poll")
        return [{"id": r.id, "j0": r.j0, "nbits": r.nbits, "composites": r.composites,
                 "dev_bits": r.dev_bits, "t_submit": r.t_submit, "t_admit": r.t_admit,
                 "t_done": r.t_done, "status": r.status} for r in buf[:n.value]]

    def release(self, rid):
        _check(lib().sieve_server_release(self.handle, rid), "sieve_server_release")

    def now(self):
        return lib().sieve_server_now(self.handle)

    def close(self):
        if self.handle:
            lib().sieve_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sieve_server_create(ctx, mem_cap, max_inflight=4):
    return Server(ctx, mem_cap, max_inflight)
