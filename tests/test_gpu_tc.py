"""Tensor-core radix-16 variants against the FP64 oracle.

Bounds per variant follow from the operand precision (unit roundoff u of
the 16-bit type; about u^2 for the hi+lo split), the number p of radix-16
passes and the FP32 accumulation:
    plain  BF16  u = 2^-8    bound 4 u sqrt(p)
    plain  FP16  u = 2^-11   bound 4 u sqrt(p)
    split  BF16  ~u^2 = 2^-16 bound 4 * 2^-16 sqrt(p) + FP32 bound
    split  FP16  ~u^2 = 2^-22 bound 1e-5 (the stated target), checked
The measured errors are printed for the record.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1707_07263_gb300 import _lib, workloads

pytestmark = pytest.mark.gpu

PRECS = {"tc_bf16": 1, "tc_fp16": 2, "tc_bf16_split": 3, "tc_fp16_split": 4}


def radix16_passes(n: int) -> int:
    lg = int(np.log2(n))
    if lg <= 14:
        return lg // 4
    lg2 = (lg + 1) // 2
    return (lg - lg2) // 4 + lg2 // 4


def bound(prec: str, n: int) -> float:
    p = max(1, radix16_passes(n))
    fp32 = 5e-7 * np.log2(n)
    if prec == "tc_bf16":
        return 4 * 2.0 ** -8 * np.sqrt(p)
    if prec == "tc_fp16":
        return 4 * 2.0 ** -11 * np.sqrt(p)
    if prec == "tc_bf16_split":
        return 4 * 2.0 ** -16 * np.sqrt(p) + fp32
    return 1e-5


def run(lib, x: np.ndarray, prec: int, d: int) -> np.ndarray:
    batch, n = x.shape
    h = ctypes.c_void_p(lib.fft_plan_create(n, batch, d, prec))
    assert h.value, _lib.ERRORS.get(lib.fft_last_error())
    ws = lib.fft_plan_workspace_bytes(h)
    wsb = torch.empty(max(ws, 1), dtype=torch.uint8, device="cuda")
    if ws:
        assert lib.fft_plan_set_workspace(h, ctypes.c_void_p(wsb.data_ptr())) == 0
    xt = torch.from_numpy(x).cuda()
    out = torch.empty_like(xt)
    rc = lib.fft_exec(h, ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, _lib.ERRORS.get(rc)
    torch.cuda.synchronize()
    lib.fft_destroy(h)
    return out.cpu().numpy()


@pytest.fixture(scope="module")
def lib():
    return _lib.load()


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("lg", [8, 10, 12, 16, 20])
def test_tc_forward(lib, prec, lg):
    n = 1 << lg
    batch = max(1, min(16, (1 << 20) // n))
    x = workloads.cgauss(n, batch, seed=4000 + lg)
    got = run(lib, x, PRECS[prec], 0)
    errs = oracle.rel_l2_rows(got, oracle.transform(x.astype(np.complex128)))
    print(f"{prec} N=2^{lg}: max rel-L2 {errs.max():.3e} (bound {bound(prec, n):.2e})")
    assert np.all(np.isfinite(got))
    assert errs.max() <= bound(prec, n)


@pytest.mark.parametrize("prec", ["tc_fp16_split", "tc_bf16"])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_tc_directions(lib, prec, d):
    n = 1 << 12
    x = workloads.uniform(n, 3, seed=4100 + d)
    got = run(lib, x, PRECS[prec], d)
    x64 = x.astype(np.complex128)
    ref = {1: oracle.fft(x64, oracle.INVERSE), 2: oracle.fft(x64, oracle.ADJOINT),
           3: oracle.fft(x64, oracle.FORWARD) / n}[d]
    assert oracle.rel_l2_rows(got, ref).max() <= bound(prec, n)


def test_tc_unsupported_length(lib):
    assert lib.fft_plan_create(1 << 14, 1, 0, 4) is None
    assert lib.fft_last_error() == -6
