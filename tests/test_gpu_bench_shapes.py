"""GPU parity at the benchmark's exact shapes and plans, against the FP64 oracle.

The benchmark's step transforms 2^26 points per length N in {2^10, 2^12, 2^14}
(batch 2^26 / N), forward and inverse, with the plans the autotuner ships for
those shapes.  At these batches the persistent kernels loop: the TMA-staged
2^10 kernel runs ~36 tiles per CTA, so its staging buffer is refilled and its
mbarrier phase flips dozens of times per CTA -- a regime the small-batch parity
tests never reach.  Here every row of the full batch is compared with the
oracle (recursive radix-2 in FP64, a few seconds per direction), so a fault in
any CTA's later tiles shows up.

The TMA-staged kernel's other default lengths (2^9 and 2^11) run here too,
at batches of at least eight tiles per CTA with a ragged last tile.
"""
from __future__ import annotations

import ctypes
import re

import numpy as np
import pytest
import torch

import oracle
from paper_1707_07263_gb300 import _lib, tune, workloads

pytestmark = pytest.mark.gpu

TOTAL = 1 << 26


def tol32(n: int) -> float:
    return 5e-7 * max(1.0, np.log2(n))


@pytest.fixture(scope="module")
def lib():
    return _lib.load()


@pytest.fixture(scope="module")
def bench_input():
    """The benchmark's input: one CN(0,1) draw of 2^26 points (seed of the
    batched-FFT workload), read as batch x N for every N."""
    return workloads.cgauss(TOTAL, 1, seed=workloads.seed_for(1)).reshape(-1)


def describe(lib, h) -> dict:
    buf = ctypes.create_string_buffer(512)
    lib.fft_plan_describe(h, buf, 512)
    return {k: v for k, v in re.findall(r"(\w+)=(\S+)", buf.value.decode())}


def plan_like_bench(lib, n: int, batch: int):
    """The plan bench.py builds by default: the autotuner's configuration."""
    cfg = _lib.FftPlanConfig.from_dict(tune.tuned_config(n, batch, 0, torch.device("cuda", 0)))
    h = lib.fft_plan_create_config(n, batch, 0, 0, ctypes.byref(cfg))
    assert h, _lib.ERRORS.get(lib.fft_last_error())
    return ctypes.c_void_p(h), cfg


def run(lib, h, x: torch.Tensor, d: int) -> np.ndarray:
    out = torch.empty_like(x)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.fft_exec_dir(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), d, s)
    assert rc == 0, _lib.ERRORS.get(rc, rc)
    torch.cuda.synchronize()
    assert lib.fft_status(h, s) == 0
    return out.cpu().numpy()


def check_all_rows(got: np.ndarray, x: np.ndarray, d: int, n: int, what: str) -> None:
    batch = got.size // n
    ref = oracle.fft(x.reshape(batch, n).astype(np.complex128), oracle.INVERSE if d else oracle.FORWARD)
    got = got.reshape(batch, n)
    assert np.all(np.isfinite(got)), f"{what}: non-finite output"
    errs = oracle.rel_l2_rows(got, ref)
    assert errs.max() <= tol32(n), f"{what}: row {int(errs.argmax())} rel-L2 {errs.max():.3e} > {tol32(n):.2e}"


@pytest.mark.parametrize("lg", [10, 12, 14])
@pytest.mark.parametrize("d", [0, 1], ids=["fwd", "inv"])
def test_bench_shape_every_row(lib, bench_input, lg, d):
    n = 1 << lg
    batch = TOTAL // n
    h, cfg = plan_like_bench(lib, n, batch)
    try:
        if lg == 10:
            # the shipped 2^10 plan is the persistent TMA-staged kernel, and at
            # this batch every CTA loops over many tiles
            info = describe(lib, h)
            assert cfg.tma == 1, "the 2^10 benchmark plan is the TMA-staged kernel"
            grid = int(info["tma_grid"])
            assert grid > 0 and batch / (4 * grid) >= 8, f"tiles per CTA {batch / (4 * grid):.1f}"
        x = torch.from_numpy(bench_input).cuda()
        got = run(lib, h, x, d)
        del x
        check_all_rows(got, bench_input, d, n, f"bench shape 2^{lg} x {batch} dir {d}")
    finally:
        lib.fft_destroy(h)


@pytest.mark.parametrize("lg", [9, 10, 11])
def test_tma_kernel_loops_with_ragged_tail(lib, lg):
    """Default plan (TMA-staged at 2^9..2^11) at >= 8 tiles per CTA, with a
    batch that leaves the last tile partly empty."""
    n = 1 << lg
    h0 = ctypes.c_void_p(lib.fft_plan_create(n, 1 << 16, 0, 0))
    assert h0.value
    info = describe(lib, h0)
    grid = int(info["tma_grid"])
    lib.fft_destroy(h0)
    assert grid > 0, "default plan at 2^9..2^11 is the TMA-staged kernel"
    cols = max(1, 4096 // n)         # transforms per tile: at most 4096 points per tile
    batch = 8 * grid * cols + cols // 2 + 1
    h = ctypes.c_void_p(lib.fft_plan_create(n, batch, 0, 0))
    try:
        assert int(describe(lib, h)["tma_grid"]) == grid
        x = workloads.cgauss(n, batch, seed=7100 + lg)
        for d in (0, 1):
            got = run(lib, h, torch.from_numpy(x.reshape(-1)).cuda(), d)
            check_all_rows(got, x, d, n, f"TMA 2^{lg} x {batch} dir {d}")
    finally:
        lib.fft_destroy(h)
