"""The allocation-free entry point fft_exec_noalloc against the planned path.

fft_exec_noalloc serves callers that cannot allocate device memory when they
need a transform (allocator callbacks, plug-ins in hosts that own all device
memory, real-time paths).  It keeps its workspace and twiddles in a static
device array shared by every call, so this test runs two different calls in a
row and checks that each matches the result of the ordinary plan + fft_exec
path on the same input.  The file is named to be collected last.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1707_07263_gb300 import _lib, workloads

pytestmark = pytest.mark.gpu


def _planned(lib, x: torch.Tensor, n: int, batch: int, d: int) -> torch.Tensor:
    h = ctypes.c_void_p(lib.fft_plan_create(n, batch, d, 0))
    assert h.value, _lib.ERRORS.get(lib.fft_last_error())
    ws = torch.empty(lib.fft_plan_workspace_bytes(h), dtype=torch.uint8, device="cuda")
    assert lib.fft_plan_set_workspace(h, ctypes.c_void_p(ws.data_ptr())) == 0
    out = torch.empty_like(x)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.fft_exec(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), s) == 0
    torch.cuda.synchronize()
    lib.fft_destroy(h)
    return out


def _noalloc(lib, x: torch.Tensor, n: int, batch: int, d: int) -> torch.Tensor:
    out = torch.empty_like(x)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.fft_exec_noalloc(n, batch, d, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), s)
    assert rc == 0, _lib.ERRORS.get(rc, rc)
    torch.cuda.synchronize()
    return out


def test_noalloc_matches_planned_path_twice_in_a_row():
    lib = _lib.load()
    calls = [(1 << 20, 2, 0, 11), (1 << 16, 5, 1, 12)]   # (n, batch, dir, seed): two different calls
    for n, batch, d, seed in calls:
        x = torch.from_numpy(workloads.cgauss(n, batch, seed=seed).reshape(-1)).cuda()
        ref = _planned(lib, x, n, batch, d).cpu().numpy().reshape(batch, n)
        got = _noalloc(lib, x, n, batch, d).cpu().numpy().reshape(batch, n)
        err = oracle.rel_l2_rows(got, ref).max()
        assert err <= 5e-7 * np.log2(n), f"n={n} batch={batch} dir={d}: {err:.3e}"


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = _lib.load()
    x = torch.zeros(8, dtype=torch.complex64, device="cuda")
    p = ctypes.c_void_p(x.data_ptr())
    assert lib.fft_exec_noalloc(1 << 23, 1, 0, p, p, None) == -1       # length above 2^22
    assert lib.fft_exec_noalloc(1 << 20, 5, 0, p, p, None) == -1       # n*batch above 2^22
    assert lib.fft_exec_noalloc(1 << 14, 1, 0, p, p, None) == -1       # below the four-step range
