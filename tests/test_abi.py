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
    with open(HEADER) as f:
        src = f.read()
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
    (13 * 1024, 1, 0, 0), # prime factor 13 beyond one on-chip pass
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


@pytest.mark.parametrize("n,cfg", [
    (1 << 10, {"radix": 2}),
    (1 << 10, {"radix": 32}),
    (1 << 10, {"radix": 12}),
    (1 << 14, {"radix": 8}),               # 2048 threads: not compiled
    (1 << 13, {"radix": 4}),
    (1 << 4, {"radix": 8}),                # below the compiled range
    (1 << 15, {"radix": 8}),               # multi-pass length
    (1 << 12, {"radix": 8, "npass": 2}),
    (1 << 12, {"radix": 4, "tma": 1}),
    (1 << 12, {"radix": 8, "tma": 3}),
    (1 << 12, {"radix": 8, "halves": 2}),
    (1 << 12, {"radix": 4, "fused": 1}),
])
def test_plan_config_radix_without_kernel_is_unsupported(lib, n, cfg):
    """A largest radix other than 16 exists only for one on-chip FP32 pass on
    the register path (radix 8: 2^5..2^13, radix 4: 2^5..2^12); everything
    else is refused before any launch or allocation."""
    from paper_1707_07263_gb300 import _lib
    c = _lib.FftPlanConfig.from_dict(cfg)
    assert lib.fft_plan_create_config(n, 1, 0, 0, ctypes.byref(c)) is None, cfg
    assert lib.fft_last_error() == -6
    c = _lib.FftPlanConfig.from_dict({"radix": 8})
    assert lib.fft_plan_create_config(1 << 10, 1, 0, 1, ctypes.byref(c)) is None   # tensor-core precision
    assert lib.fft_last_error() == -6


def test_plan_create_2d_rejects(lib):
    assert lib.fft_plan_create_2d(11, 16, 1, 0, 0) is None    # prime side
    assert lib.fft_plan_create_2d(16, 26, 1, 0, 0) is None    # side with factor 13
    assert lib.fft_plan_create_2d(1, 16, 1, 0, 0) is None
    assert lib.fft_plan_create_2d(16, 1 << 15, 1, 0, 0) is None
    assert lib.fft_plan_create_2d(16, 16, 0, 0, 0) is None
    assert lib.fft_last_error() == -1


def test_plan_create_many_rejects(lib):
    assert lib.fft_plan_create_many(None, 3, 0, 0) is None
    arr = (ctypes.c_int64 * 2)(16, 32)
    assert lib.fft_plan_create_many(arr, 0, 0, 0) is None
    assert lib.fft_plan_create_many(arr, 2, 7, 0) is None
    assert lib.fft_last_error() == -1


def test_plan_create_many_config_rejects(lib):
    """Out-of-range uneven-batch configurations fail before anything runs."""
    from paper_1707_07263_gb300 import _lib
    arr = (ctypes.c_int64 * 3)(1 << 13, 1 << 16, 256)
    bad = [{"gap": 17}, {"lg1": [8, 0, 0, 0]}, {"lg1": [6, 0, 0, 0]}, {"lg1": [0, 6, 0, 0]}, {"lg1": [0, 9, 0, 0]},
           {"lg1": [0, 0, 6, 0]}, {"lg1": [0, 0, 0, 7]}, {"lg1": [0, 0, 0, 9]}]
    for d in bad:
        c = _lib.FftManyConfig.from_dict(d)
        assert lib.fft_plan_create_many_config(arr, 3, 0, 0, ctypes.byref(c)) is None, d
        assert lib.fft_last_error() == -1
    c = _lib.FftManyConfig()
    assert lib.fft_plan_create_many_config(None, 3, 0, 0, ctypes.byref(c)) is None
    assert lib.fft_plan_get_many_config(None, ctypes.byref(c)) == -1
    us = ctypes.c_float()
    buf = ctypes.create_string_buffer(64)
    p = ctypes.cast(buf, ctypes.c_void_p)
    assert lib.fft_autotune_many(None, 3, 0, p, p, p, 64, None, 5, ctypes.byref(c), ctypes.byref(us)) == -1
    assert lib.fft_autotune_many(arr, 3, 0, p, p, p, 64, None, 0, ctypes.byref(c), ctypes.byref(us)) == -1
    assert lib.fft_autotune_many(arr, 0, 0, p, p, p, 64, None, 5, ctypes.byref(c), ctypes.byref(us)) == -1
    assert lib.fft_autotune_many(arr, 3, 1, p, p, p, 64, None, 5, ctypes.byref(c), ctypes.byref(us)) == -6


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
    assert lib.fft_exec_filter_dir(None, None, None, None, 0, None) == -1
    assert lib.fft_exec_filter_dir(None, None, None, None, 2, None) == -1
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


def test_plan_create_many_rejects_bad_lengths(lib):
    for bad in ((16, 3), (16, 1), (16, 1 << 17), (0, 16), (16, -32)):
        arr = (ctypes.c_int64 * len(bad))(*bad)
        assert lib.fft_plan_create_many(arr, len(bad), 0, 0) is None, bad
        assert lib.fft_last_error() == -1


def test_noalloc_rejects_before_launching(lib):
    buf = ctypes.create_string_buffer(64)
    p = ctypes.cast(buf, ctypes.c_void_p)
    odd = ctypes.c_void_p(p.value + 4)
    assert lib.fft_exec_noalloc(1000, 1, 0, p, p, None) == -1        # not a power of two
    assert lib.fft_exec_noalloc(1 << 14, 1, 0, p, p, None) == -1     # below 2^15
    assert lib.fft_exec_noalloc(1 << 23, 1, 0, p, p, None) == -1     # above 2^22
    assert lib.fft_exec_noalloc(1 << 16, 1 << 7, 0, p, p, None) == -1  # n * batch above 2^22
    assert lib.fft_exec_noalloc(1 << 16, 0, 0, p, p, None) == -1
    assert lib.fft_exec_noalloc(1 << 16, 1, 4, p, p, None) == -1     # unknown direction
    assert lib.fft_exec_noalloc(1 << 16, 1, 0, None, p, None) == -1
    assert lib.fft_exec_noalloc(1 << 16, 1, 0, odd, p, None) == -2   # 8-byte alignment


def test_null_plan_queries(lib):
    from paper_1707_07263_gb300 import _lib
    cfg = _lib.FftPlanConfig()
    assert lib.fft_plan_get_config(None, ctypes.byref(cfg)) == -1
    buf = ctypes.create_string_buffer(64)
    assert lib.fft_plan_describe(None, buf, 64) == -1
    assert lib.fft_status(None, None) == -1
    assert lib.fft_plan_length(None) == 0 and lib.fft_plan_batch(None) == 0


def test_autotune_rejects_before_running(lib):
    from paper_1707_07263_gb300 import _lib
    cfg = _lib.FftPlanConfig()
    us = ctypes.c_float()
    buf = ctypes.create_string_buffer(64)
    p = ctypes.cast(buf, ctypes.c_void_p)
    for n, batch, iters in ((1000, 1, 5), (1024, 0, 5), (1024, 1, 0)):
        assert lib.fft_autotune(n, batch, 0, p, p, p, 64, None, iters, ctypes.byref(cfg), ctypes.byref(us)) == -1
    assert lib.fft_autotune(1024, 1, 0, None, p, p, 64, None, 5, ctypes.byref(cfg), ctypes.byref(us)) == -1


def test_fp64_and_mixed_length_limits(lib):
    """Argument errors (-1) and valid requests beyond what is built (-6), all
    decided on the host before any device work."""
    from paper_1707_07263_gb300 import _lib
    fp64 = _lib.FFT_PREC_FP64
    assert lib.fft_plan_create(1 << 25, 1, 0, fp64) is None     # 4096 x 8192: no split into two FP64 passes
    assert lib.fft_last_error() == -6
    assert lib.fft_plan_create(7168 * 7168 * 2, 1, 0, fp64) is None   # beyond two FP64 passes
    assert lib.fft_last_error() == -6
    assert lib.fft_plan_create(3 ** 17, 1, 0, 0) is None        # 7-smooth, no split into two passes of <= 14336
    assert lib.fft_last_error() == -6
    assert lib.fft_plan_create(14336 * 14336 * 3, 1, 0, 0) is None   # beyond two mixed-radix passes
    assert lib.fft_last_error() == -6
    assert lib.fft_plan_create(13 * 16, 1, 0, fp64) is None     # prime factor 13
    assert lib.fft_last_error() == -1
    assert lib.fft_plan_create(1, 1, 0, fp64) is None
    assert lib.fft_last_error() == -1
    assert lib.fft_plan_create(14337, 1, 0, 0) is None          # 3^5 * 59
    assert lib.fft_last_error() == -1
    assert lib.fft_plan_create_2d(64, 8192, 1, 0, fp64) is None     # FP64 side beyond one pass
    assert lib.fft_last_error() == -6
    assert lib.fft_plan_create_2d(12, 16, 1, 0, 1) is None      # mixed 2-D on the tensor cores
    assert lib.fft_last_error() == -6
    arr = (ctypes.c_int64 * 2)(16, 32)
    assert lib.fft_plan_create_many(arr, 2, 0, fp64) is None
    assert lib.fft_last_error() == -6
    assert lib.fft_plan_create_r2c(22, 1, fp64) is None          # half length 11
    assert lib.fft_last_error() == -1
    assert lib.fft_plan_create_r2c(15, 1, fp64) is None          # odd
    assert lib.fft_last_error() == -1
    assert lib.fft_plan_create_r2c(2 * 7168 * 7168 * 2, 1, fp64) is None   # half beyond two FP64 passes
    assert lib.fft_last_error() == -6
    assert lib.fft_plan_create_r2c(24, 1, 1) is None             # real data on the tensor cores
    assert lib.fft_last_error() == -1


def test_pointers_that_are_not_live_plans(lib):
    """A pointer that no plan constructor returned (or one already destroyed)
    is refused by every entry point, and destroying it frees nothing."""
    from paper_1707_07263_gb300 import _lib
    fake_buf = ctypes.create_string_buffer(4096)
    fake = ctypes.c_void_p(ctypes.addressof(fake_buf))
    buf = ctypes.create_string_buffer(64)
    p = ctypes.cast(buf, ctypes.c_void_p)
    assert lib.fft_exec(fake, p, p, None) == -1
    assert lib.fft_exec_dir(fake, p, p, 0, None) == -1
    assert lib.fft_exec_filter(fake, p, p, p, None) == -1
    assert lib.fft_exec_filter_dir(fake, p, p, p, 2, None) == -1
    assert lib.fft_plan_set_workspace(fake, None) == -1
    assert lib.fft_status(fake, None) == -1
    assert lib.fft_plan_workspace_bytes(fake) == 0 and lib.fft_plan_launches(fake) == 0
    assert lib.fft_plan_length(fake) == 0 and lib.fft_plan_batch(fake) == 0 and lib.fft_plan_kind(fake) == -1
    assert lib.fft_plan_get_config(fake, ctypes.byref(_lib.FftPlanConfig())) == -1
    assert lib.fft_plan_describe(fake, buf, 64) == -1
    lib.fft_destroy(fake)
    assert lib.fft_last_error() == -1
    lib.fft_destroy(fake)                       # twice: still nothing freed
    assert fake_buf.raw == bytes(4096)
