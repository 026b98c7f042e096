"""The allocation-free composite count (sieve_count_noalloc), called through the
C ABI, agrees with sieve_count on two calls in a row.

This file is collected last on purpose: if it fails, a run stopped at the first
failure has already run every other test."""
import ctypes

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc():
    from paper_1111_3297_gb300 import sieve as S
    fn = S.lib().sieve_count_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
    return fn


def test_noalloc_count_matches_sieve_count_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_3297_gb300 import build
    build.build_library()
    from paper_1111_3297_gb300 import sieve as S
    fn = _noalloc()
    ctx = S.sieve_init(0, max_v=10**16)
    try:
        stream = torch.cuda.current_stream()
        cases = [(20, 10**6, 300), (16, 12345, 77)]  # the second is smaller: stale partials must not leak
        for l, f, n in cases:
            nbits = n << l
            out = torch.empty(nbits // 32, dtype=torch.int32, device="cuda")
            S.sieve_segments(ctx, l, f, n, out)
            S.sieve_sync(ctx)
            want = S.sieve_count(ctx, out, nbits)
            dev_count = torch.full((1,), -1, dtype=torch.int64, device="cuda")
            st = fn(ctypes.c_void_p(out.data_ptr()), nbits, ctypes.c_void_p(dev_count.data_ptr()),
                    ctypes.c_void_p(stream.cuda_stream))
            assert st == 0
            torch.cuda.synchronize()
            assert int(dev_count.item()) == want, (l, f, n)
        # sizes beyond the fixed scratch are refused, nothing launched
        dev_count = torch.zeros(1, dtype=torch.int64, device="cuda")
        st = fn(ctypes.c_void_p(out.data_ptr()), (1 << 37) + 32, ctypes.c_void_p(dev_count.data_ptr()),
                ctypes.c_void_p(stream.cuda_stream))
        assert st == 2
    finally:
        ctx.close()
