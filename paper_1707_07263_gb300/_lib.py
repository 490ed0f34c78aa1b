"""ctypes loader for ``libgbfft.so`` (the C ABI declared in include/gbfft.h).

Argument marshalling only: every step of a transform runs in the library's
CUDA kernels.  Importing this module never builds anything; a missing library
raises immediately so no caller can fall back to another implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbfft.so")

FFT_FORWARD, FFT_INVERSE, FFT_ADJOINT = 0, 1, 2
FFT_PREC_FP32, FFT_PREC_TC_BF16, FFT_PREC_TC_FP16, FFT_PREC_TC_BF16_SPLIT, FFT_PREC_TC_FP16_SPLIT, FFT_PREC_FP64 = range(6)

FFT_OK = 0
ERRORS = {
    -1: "FFT_ERR_INVALID_ARG",
    -2: "FFT_ERR_ALIGN",
    -3: "FFT_ERR_NO_WORKSPACE",
    -4: "FFT_ERR_CUDA",
    -5: "FFT_ERR_TIMEOUT",
    -6: "FFT_ERR_UNSUPPORTED",
    -7: "FFT_ERR_ALLOC",
}

class FftPlanConfig(ctypes.Structure):
    """fft_plan_config of include/gbfft.h."""
    _fields_ = [(name, ctypes.c_int) for name in ("npass", "lg1", "lg2", "c1", "c2", "c3", "tma", "fused",
                                                  "halves", "radix")]

    def as_dict(self) -> dict:
        return {name: int(getattr(self, name)) for name, _ in self._fields_}

    @classmethod
    def from_dict(cls, d: dict) -> "FftPlanConfig":
        c = cls()
        c.tma = -1
        c.fused = -1
        for k, v in d.items():
            setattr(c, k, int(v))
        return c


class FftManyConfig(ctypes.Structure):
    """fft_many_config of include/gbfft.h (uneven-batch plans)."""
    _fields_ = [("gap", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("lg1", ctypes.c_int * 4)]

    def as_dict(self) -> dict:
        return {"gap": int(self.gap), "ctas_per_sm": int(self.ctas_per_sm), "lg1": [int(v) for v in self.lg1]}

    @classmethod
    def from_dict(cls, d: dict) -> "FftManyConfig":
        c = cls()
        c.gap = int(d.get("gap", 0))
        c.ctas_per_sm = int(d.get("ctas_per_sm", 0))
        for i, v in enumerate(d.get("lg1", [0, 0, 0, 0])):
            c.lg1[i] = int(v)
        return c


# name -> (restype, argtypes); the full exported surface of include/gbfft.h
_i64, _int, _vp, _sz = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t
SIGNATURES = {
    "fft_plan_create": (_vp, [_i64, _i64, _int, _int]),
    "fft_plan_create_2d": (_vp, [_i64, _i64, _i64, _int, _int]),
    "fft_plan_create_many": (_vp, [ctypes.POINTER(_i64), _i64, _int, _int]),
    "fft_plan_create_r2c": (_vp, [_i64, _i64, _int]),
    "fft_plan_create_many_config": (_vp, [ctypes.POINTER(_i64), _i64, _int, _int, ctypes.POINTER(FftManyConfig)]),
    "fft_plan_get_many_config": (_int, [_vp, ctypes.POINTER(FftManyConfig)]),
    "fft_autotune_many": (_int, [ctypes.POINTER(_i64), _i64, _int, _vp, _vp, _vp, _sz, _vp, _int,
                                 ctypes.POINTER(FftManyConfig), ctypes.POINTER(ctypes.c_float)]),
    "fft_exec": (_int, [_vp, _vp, _vp, _vp]),
    "fft_exec_dir": (_int, [_vp, _vp, _vp, _int, _vp]),
    "fft_destroy": (None, [_vp]),
    "fft_plan_workspace_bytes": (_sz, [_vp]),
    "fft_plan_set_workspace": (_int, [_vp, _vp]),
    "fft_plan_length": (_i64, [_vp]),
    "fft_plan_batch": (_i64, [_vp]),
    "fft_plan_launches": (_int, [_vp]),
    "fft_plan_kind": (_int, [_vp]),
    "fft_plan_describe": (_int, [_vp, ctypes.c_char_p, _sz]),
    "fft_status": (_int, [_vp, _vp]),
    "fft_exec_noalloc": (_int, [_i64, _i64, _int, _vp, _vp, _vp]),
    "fft_plan_create_config": (_vp, [_i64, _i64, _int, _int, ctypes.POINTER(FftPlanConfig)]),
    "fft_plan_get_config": (_int, [_vp, ctypes.POINTER(FftPlanConfig)]),
    "fft_autotune": (_int, [_i64, _i64, _int, _vp, _vp, _vp, _sz, _vp, _int, ctypes.POINTER(FftPlanConfig),
                            ctypes.POINTER(ctypes.c_float)]),
    "fft_pointer_usable": (_int, [_vp, _sz]),
    "fft_exec_filter": (_int, [_vp, _vp, _vp, _vp, _vp]),
    "fft_exec_filter_dir": (_int, [_vp, _vp, _vp, _vp, _int, _vp]),
    "fft_last_error": (_int, []),
    "fft_error_string": (ctypes.c_char_p, [_int]),
}

_lib = None


class GbfftError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        name = ERRORS.get(code, str(code))
        super().__init__(f"{what}: {name}" if what else name)


def load(path: str | None = None):
    """Load the library once; raise if it has not been built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with __graft_entry__.build() "
                           "(there is no fallback implementation)")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def check(code: int, what: str = "") -> int:
    if code != FFT_OK:
        raise GbfftError(code, what)
    return code
