"""GB300-native power-of-two complex FFT (Cooley-Tukey, forward/inverse/adjoint)
after "A GPU Based Memory Optimized Parallel Method For FFT Implementation".

The compute path is ``libgbfft.so`` (hand-written sm_103a CUDA behind the C ABI
of include/gbfft.h); this package is its thin PyTorch binding.  Importing the
package does not load the library: the first transform does, and raises if
the library is missing.
"""
from __future__ import annotations

from ._lib import (FFT_ADJOINT, FFT_FORWARD, FFT_INVERSE, FFT_PREC_FP32, FFT_PREC_FP64, FFT_PREC_TC_BF16,  # noqa: F401
                   FFT_PREC_TC_BF16_SPLIT, FFT_PREC_TC_FP16, FFT_PREC_TC_FP16_SPLIT, GbfftError)


def __getattr__(name):
    # lazy: torch and the CUDA library are only touched when the API is used
    if name in ("fft", "ifft", "fft2", "ifft2", "fft_many", "fft_host", "HostPipeline", "range_compress", "rfft", "irfft", "Plan", "get_plan",
                "clear_plan_cache", "PREC"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
