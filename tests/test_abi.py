"""Host-side checks of the C ABI: the library loads, exports every function
include/gbfft.h declares, and rejects bad arguments on the host before any
CUDA call.  None of these touch a GPU."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbfft.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1707_07263_gb300 import build_lib, _lib
    build_lib.build()
    return _lib.load()


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"GBFFT_API\s+[\w\s\*]+?\b(fft_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fft_plan_create", "fft_exec", "fft_destroy", "fft_plan_create_2d", "fft_plan_create_many",
                     "fft_plan_workspace_bytes", "fft_plan_set_workspace", "fft_last_error", "fft_error_string",
                     "fft_status"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1707_07263_gb300 import _lib
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} not exported"
        assert name in _lib.SIGNATURES, f"{name} has no binding signature"


def test_error_strings(lib):
    assert lib.fft_error_string(0) == b"ok"
    for code in range(-7, 0):
        assert lib.fft_error_string(code) not in (b"", b"unknown error")
    assert lib.fft_error_string(-99) == b"unknown error"


@pytest.mark.parametrize("n,batch,dir,prec", [
    (11, 1, 0, 0),        # a prime factor above 7
    (2 * 3 * 7 * 11, 1, 0, 0),
    (3 << 13, 1, 0, 0),   # 7-smooth but beyond the one-pass mixed-radix limit (14336)
    (0, 1, 0, 0),
    (1, 1, 0, 0),         # N=1 is not supported
    (-8, 1, 0, 0),
    (1 << 29, 1, 0, 0),   # beyond 2^28
    (16, 0, 0, 0),        # batch < 1
    (16, -3, 0, 0),
    (16, 1, 4, 0),        # unknown direction
    (16, 1, -1, 0),
    (16, 1, 0, 9),        # unknown precision
])
def test_plan_create_rejects(lib, n, batch, dir, prec):
    assert lib.fft_plan_create(n, batch, dir, prec) is None
    assert lib.fft_last_error() == -1


def test_mixed_radix_tensor_core_is_unsupported(lib):
    assert lib.fft_plan_create(12, 1, 0, 1) is None
    assert lib.fft_last_error() == -6


def test_plan_create_2d_rejects(lib):
    assert lib.fft_plan_create_2d(12, 16, 1, 0, 0) is None
    assert lib.fft_plan_create_2d(16, 1 << 15, 1, 0, 0) is None
    assert lib.fft_plan_create_2d(16, 16, 0, 0, 0) is None
    assert lib.fft_last_error() == -1


def test_plan_create_many_rejects(lib):
    assert lib.fft_plan_create_many(None, 3, 0, 0) is None
    arr = (ctypes.c_int64 * 2)(16, 32)
    assert lib.fft_plan_create_many(arr, 0, 0, 0) is None
    assert lib.fft_plan_create_many(arr, 2, 7, 0) is None
    assert lib.fft_last_error() == -1


def test_plan_create_r2c_rejects(lib):
    assert lib.fft_plan_create_r2c(12, 1, 0) is None      # not a power of two
    assert lib.fft_plan_create_r2c(2, 1, 0) is None       # below 4
    assert lib.fft_plan_create_r2c(1 << 29, 1, 0) is None  # above 2^28
    assert lib.fft_plan_create_r2c(16, 0, 0) is None
    assert lib.fft_last_error() == -1
    assert lib.fft_plan_create_r2c(16, 1, 1) is None      # tensor-core precisions: not for real data
    assert lib.fft_last_error() == -6


def test_null_plan_calls(lib):
    assert lib.fft_exec(None, None, None, None) == -1
    assert lib.fft_exec_dir(None, None, None, 0, None) == -1
    assert lib.fft_exec_filter(None, None, None, None, None) == -1
    assert lib.fft_pointer_usable(None, 8) == -1
    assert lib.fft_plan_workspace_bytes(None) == 0
    assert lib.fft_plan_set_workspace(None, None) == -1
    assert lib.fft_plan_launches(None) == 0
    assert lib.fft_plan_kind(None) == -1
    lib.fft_destroy(None)   # NULL-safe


def test_python_api_fails_loudly_without_cuda_tensor():
    import torch
    import paper_1707_07263_gb300 as gb
    with pytest.raises(TypeError):
        gb.fft(torch.zeros(16, dtype=torch.complex64))   # CPU tensor: no fallback
    with pytest.raises(TypeError):
        gb.range_compress(torch.zeros(16, dtype=torch.complex64), torch.zeros(16, dtype=torch.complex64))
    with pytest.raises(TypeError):
        gb.rfft(torch.zeros(16, dtype=torch.float32))
    with pytest.raises(TypeError):
        gb.irfft(torch.zeros(9, dtype=torch.complex64))
