"""The C ABI library builds for sm_103a, loads, and exports every function that
include/*.h declares (no device calls: runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\(", text):
            name = m.group(1)
            if name.startswith("sieve_") and not name.endswith("_t"):
                names.add(name)
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import shutil
    from paper_1111_3297_gb300 import build
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc") \
            and not os.path.exists(build.LIB):
        pytest.skip("no nvcc to build the library")
    return ctypes.CDLL(build.build_library())


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["sieve_init", "sieve_segments", "sieve_count", "sieve_f_from_midpoint",
                 "sieve_segments_midpoint", "sieve_batch", "sieve_destroy", "sieve_strerror",
                 "sieve_server_create", "sieve_autotune"]:
        assert must in names


def test_library_exports_every_declared_function(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points_work_without_a_gpu(lib):
    lib.sieve_strerror.restype = ctypes.c_char_p
    assert lib.sieve_strerror(0) == b"ok"
    assert b"overflow" in lib.sieve_strerror(7)
    lib.sieve_last_cuda_error.restype = ctypes.c_char_p
    assert isinstance(lib.sieve_last_cuda_error(), bytes)
    f = ctypes.c_uint64()
    lib.sieve_f_from_midpoint.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                          ctypes.POINTER(ctypes.c_uint64)]
    assert lib.sieve_f_from_midpoint(20, 32768, 1 << 60, 0, ctypes.byref(f)) == 0
    assert f.value == 2**39 - 16384
    assert lib.sieve_f_from_midpoint(4, 1, 1, 0, ctypes.byref(f)) == 1
    assert lib.sieve_f_from_midpoint(20, 1, 5, 19, ctypes.byref(f)) == 2  # 5e19 > 2^64


def test_init_rejects_a_bucket_budget_below_64_mib(lib):
    # checked before any device call, so it answers without a GPU
    h = ctypes.c_void_p()
    lib.sieve_init.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_uint64, ctypes.c_size_t]
    assert lib.sieve_init(ctypes.byref(h), 0, 1 << 40, (64 << 20) - 1) == 1
    assert h.value is None


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    from paper_1111_3297_gb300 import sieve as S
    monkeypatch.setattr(S, "_lib", None)
    monkeypatch.setattr(S, "_LIBPATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        S.lib()


class _FakeCudaTensor:
    """Looks like a contiguous CUDA int32 tensor of n elements to the binding."""
    is_cuda = True

    def __init__(self, n):
        self.n = n

    def is_contiguous(self):
        return True

    def numel(self):
        return self.n

    def element_size(self):
        return 4

    def data_ptr(self):
        return 0x10000


class _FakeCtx:
    handle = None


def test_binding_refuses_buffers_smaller_than_the_call(lib):
    # the C ABI takes plain pointers; the binding checks sizes before any call
    import numpy as np
    from paper_1111_3297_gb300 import sieve as S
    with pytest.raises(ValueError):  # 2^20 bits need 2^15 words
        S.sieve_segments(_FakeCtx(), 20, 0, 1, _FakeCudaTensor((1 << 15) - 1))
    with pytest.raises(ValueError):
        S.sieve_segments_midpoint(_FakeCtx(), 20, 1, 15, 2, _FakeCudaTensor(1 << 15))
    with pytest.raises(ValueError):
        S.sieve_count(_FakeCtx(), _FakeCudaTensor(8), 8 * 32 + 32)
    reqs = [(0, 64, 0), (1 << 20, 96, 10)]  # the second ends at word 13
    with pytest.raises(ValueError):
        S.sieve_batch(_FakeCtx(), reqs, _FakeCudaTensor(12), _FakeCudaTensor(4))
    with pytest.raises(ValueError):  # two int64 counts need 16 bytes
        S.sieve_batch(_FakeCtx(), reqs, _FakeCudaTensor(13), _FakeCudaTensor(3))
    with pytest.raises(ValueError):
        S.sieve_segments_host(_FakeCtx(), 10, 0, 4, np.zeros(127, dtype=np.uint32))
