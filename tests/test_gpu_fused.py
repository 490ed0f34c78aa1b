"""The fused two-pass launch (both four-step passes in one persistent kernel,
slabs pipelined through an L2-resident workspace ring) against the oracle."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1707_07263_gb300 import _lib, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    return _lib.load()


def run(lib, x: np.ndarray, d: int, inplace: bool = False):
    batch, n = x.shape
    c = _lib.FftPlanConfig.from_dict({"fused": 1})
    h = ctypes.c_void_p(lib.fft_plan_create_config(n, batch, d, 0, ctypes.byref(c)))
    assert h.value, _lib.ERRORS.get(lib.fft_last_error())
    cfg = _lib.FftPlanConfig()
    assert lib.fft_plan_get_config(h, ctypes.byref(cfg)) == 0 and cfg.fused == 1
    assert lib.fft_plan_launches(h) == 1
    ws = lib.fft_plan_workspace_bytes(h)
    wsb = torch.empty(ws, dtype=torch.uint8, device="cuda")
    assert lib.fft_plan_set_workspace(h, ctypes.c_void_p(wsb.data_ptr())) == 0
    xt = torch.from_numpy(x.reshape(-1)).cuda()
    out = xt if inplace else torch.empty_like(xt)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.fft_exec(h, ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(out.data_ptr()), s) == 0
    torch.cuda.synchronize()
    st = lib.fft_status(h, s)
    lib.fft_destroy(h)
    return out.cpu().numpy().reshape(batch, n), st, ws


@pytest.mark.parametrize("lg", [13, 14, 15, 16, 17, 18])
@pytest.mark.parametrize("batch", [1, 7, 40])
def test_fused_forward_small_slabs(hooks_lib, monkeypatch, lg, batch):
    # 1 MB slabs (a test-build override): many slabs per launch, both workspace slots reused
    monkeypatch.setenv("GBFFT_SLAB_MB", "1")
    n = 1 << lg
    x = workloads.cgauss(n, batch, seed=9000 + lg + batch)
    got, st, ws = run(hooks_lib, x, 0)
    assert st == 0
    errs = oracle.rel_l2_rows(got, oracle.transform(x.astype(np.complex128)))
    assert errs.max() <= 5e-7 * lg


@pytest.mark.parametrize("d", [1, 2, 3])
def test_fused_directions_and_in_place(hooks_lib, monkeypatch, d):
    monkeypatch.setenv("GBFFT_SLAB_MB", "2")
    n = 1 << 14
    x = workloads.uniform(n, 33, seed=9100 + d)
    got, st, _ = run(hooks_lib, x, d, inplace=True)
    assert st == 0
    x64 = x.astype(np.complex128)
    ref = {1: oracle.fft(x64, oracle.INVERSE), 2: oracle.fft(x64, oracle.ADJOINT),
           3: oracle.fft(x64, oracle.FORWARD) / n}[d]
    assert oracle.rel_l2_rows(got, ref).max() <= 5e-7 * 14


def test_fused_full_size_sampled(lib):
    """The benchmark's 2^14 x 4096 shape with default slabs: every 97th
    transform against the oracle."""
    n, batch = 1 << 14, 4096
    x = workloads.cgauss(n, batch, seed=workloads.seed_for(1))
    got, st, _ = run(lib, x, 0)
    assert st == 0
    rows = np.arange(0, batch, 97)
    errs = oracle.rel_l2_rows(got[rows], oracle.fft(x[rows].astype(np.complex128)))
    assert errs.max() <= 5e-7 * 14
