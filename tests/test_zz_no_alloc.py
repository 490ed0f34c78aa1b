"""The allocation-free entry point fft_exec_noalloc against the oracle and the
planned path.

fft_exec_noalloc serves callers that cannot allocate device memory when they
need a transform (allocator callbacks, plug-ins in hosts that own all device
memory, real-time paths).  It keeps its workspace and twiddles in a static
device array shared by every call, so this test runs several different calls
in a row -- even and uneven splits of n, every direction, one in place -- and
checks each against the FP64 oracle and against the ordinary plan + fft_exec
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


def _noalloc(lib, x: torch.Tensor, n: int, batch: int, d: int, in_place: bool = False) -> torch.Tensor:
    out = x if in_place else torch.empty_like(x)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.fft_exec_noalloc(n, batch, d, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), s)
    assert rc == 0, _lib.ERRORS.get(rc, rc)
    torch.cuda.synchronize()
    return out


def _oracle(x: np.ndarray, d: int) -> np.ndarray:
    """Every direction code: forward (Eq. 1), inverse (Eq. 2), adjoint of the
    forward (conjugate direction, no 1/N), adjoint of the inverse (forward / N)."""
    x = x.astype(np.complex128)
    if d == 3:
        return oracle.fft(x, oracle.FORWARD) / x.shape[-1]
    return oracle.fft(x, d)


# (n, batch, dir, seed, in place): calls in a row that differ in length, split
# (2^15 and 2^21 split unevenly, 2^20 and 2^16 evenly), direction and placement
CALLS = [(1 << 20, 2, 0, 11, False), (1 << 16, 5, 1, 12, False), (1 << 15, 128, 2, 13, False),
         (1 << 21, 2, 3, 14, True), (1 << 20, 2, 0, 11, False)]


def test_noalloc_matches_oracle_and_planned_path_calls_in_a_row():
    lib = _lib.load()
    for n, batch, d, seed, in_place in CALLS:
        x = workloads.cgauss(n, batch, seed=seed)
        xt = torch.from_numpy(x.reshape(-1)).cuda()
        planned = _planned(lib, xt, n, batch, d).cpu().numpy().reshape(batch, n)
        got = _noalloc(lib, xt, n, batch, d, in_place).cpu().numpy().reshape(batch, n)
        tol = 5e-7 * np.log2(n)
        what = f"n=2^{int(np.log2(n))} batch={batch} dir={d} in_place={in_place}"
        err = oracle.rel_l2_rows(got, _oracle(x, d)).max()
        assert err <= tol, f"{what}: vs oracle {err:.3e}"
        err = oracle.rel_l2_rows(got, planned).max()
        assert err <= tol, f"{what}: vs planned path {err:.3e}"


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = _lib.load()
    x = torch.zeros(8, dtype=torch.complex64, device="cuda")
    p = ctypes.c_void_p(x.data_ptr())
    assert lib.fft_exec_noalloc(1 << 23, 1, 0, p, p, None) == -1       # length above 2^22
    assert lib.fft_exec_noalloc(1 << 20, 5, 0, p, p, None) == -1       # n*batch above 2^22
    assert lib.fft_exec_noalloc(1 << 14, 1, 0, p, p, None) == -1       # below the four-step range
