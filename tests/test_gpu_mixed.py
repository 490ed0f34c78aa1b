"""Lengths that are not powers of two (N = 2^a 3^b 5^c 7^d <= 14336, mixed
radix) against the FP64 oracle (the O(N^2) sum of Eq. 1) on the same seeded
inputs: radix-3/5/7 passes alone and mixed with radix-16/8/4/2 passes, ragged
batches, every direction, in place, and the gradient.

Bar: relative L2 error of every transform <= 5e-7 * log2(N), the FP32 bound
of the power-of-two path."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1707_07263_gb300 as gb
from paper_1707_07263_gb300 import _lib as L
from paper_1707_07263_gb300 import workloads

pytestmark = pytest.mark.gpu

LENGTHS = [3, 5, 6, 7, 9, 10, 12, 14, 15, 21, 24, 25, 27, 35, 48, 49, 60, 80, 96, 100, 105, 120, 125, 243,
           343, 360, 384, 500, 625, 720, 1000, 1080, 1200, 1500, 1536, 2000, 2187, 2400, 2401, 3000, 3072, 4000,
           4800, 5000,
           6000, 7000, 8000, 9000, 10000, 12000, 12288, 14000, 14336]


def tol(n: int) -> float:
    return 5e-7 * max(1.0, np.log2(n))


def run(x: np.ndarray, d: int, inplace: bool = False) -> np.ndarray:
    lib = L.load()
    batch, n = x.shape
    h = ctypes.c_void_p(lib.fft_plan_create(n, batch, d, 0))
    assert h.value, L.ERRORS.get(lib.fft_last_error())
    assert lib.fft_plan_kind(h) == 5
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = xt if inplace else torch.empty_like(xt)
    assert lib.fft_exec(h, ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    torch.cuda.synchronize()
    lib.fft_destroy(h)
    return out.cpu().numpy()


def ref(x: np.ndarray, d: int) -> np.ndarray:
    x64 = x.astype(np.complex128)
    n = x.shape[-1]
    if d == 0:
        return oracle.transform(x64, oracle.FORWARD)
    if d == 1:
        return oracle.transform(x64, oracle.INVERSE)
    if d == 2:
        return oracle.transform(x64, oracle.ADJOINT)
    return oracle.transform(x64, oracle.FORWARD) / n


@pytest.mark.parametrize("n", LENGTHS)
def test_forward(n):
    c = max(1, 4096 // n) if n <= 4096 else 1
    batch = min(2 * c + 1, 9) if n <= 1000 else 2
    x = workloads.cgauss(n, batch, seed=7000 + n)
    assert oracle.rel_l2_rows(run(x, 0), ref(x, 0)).max() <= tol(n), f"N={n}"


@pytest.mark.parametrize("n", [6, 105, 1000, 12000])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_directions(n, d):
    x = workloads.uniform(n, 3, seed=7100 + n + d)
    assert oracle.rel_l2_rows(run(x, d), ref(x, d)).max() <= tol(n)


@pytest.mark.parametrize("n", [7, 360, 5000, 14336])
def test_in_place(n):
    x = workloads.cgauss(n, 3, seed=7200 + n)
    assert oracle.rel_l2_rows(run(x, 0, inplace=True), ref(x, 0)).max() <= tol(n)


def test_large_batch_sampled():
    """Many transforms per launch (4096 // 96 = 42 per CTA, ragged last tile)."""
    n, batch = 96, 10007
    x = workloads.cgauss(n, batch, seed=7300)
    got = run(x, 0)
    rows = np.concatenate([np.arange(0, batch, 997), [batch - 1]])
    assert oracle.rel_l2_rows(got[rows], ref(x[rows], 0)).max() <= tol(n)


def test_round_trip_and_gradient_through_the_api():
    n = 3000
    x = workloads.cgauss(n, 2, seed=7400)
    w = workloads.real_weights(n, seed=7401)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    X = gb.fft(xt)
    back = gb.ifft(X).detach().cpu().numpy()
    assert oracle.rel_l2_rows(back, x).max() <= 2 * tol(n)
    (torch.abs(X * torch.from_numpy(w).cuda()) ** 2).sum().backward()
    x64, w64 = x.astype(np.complex128), w.astype(np.float64)
    g_ref = np.stack([2 * oracle.transform(w64 ** 2 * oracle.transform(r), oracle.ADJOINT) for r in x64])
    assert oracle.rel_l2(xt.grad.cpu().numpy(), g_ref) <= 2 * tol(n)


# lengths with a compile-time three-pass schedule of composite radices
# (10, 12, 15, 20, 24, 25 points in registers)
COMPILED = [1000, 1200, 1500, 2000, 2400, 3000, 4000, 5000, 6000, 8000, 10000, 12000]


@pytest.mark.parametrize("n", COMPILED)
@pytest.mark.parametrize("d", [0, 1, 2, 3])
def test_compiled_schedules(n, d):
    """Every compiled length, every direction, with a batch that leaves the
    last tile partly filled (tiles hold floor(4096 / N) transforms), and in
    place for the forward direction."""
    c = max(1, 4096 // n)
    batch = 3 * c + 1 if c > 1 else 5
    x = workloads.cgauss(n, batch, seed=7700 + n + d)
    got = run(x, d)
    assert oracle.rel_l2_rows(got, ref(x, d)).max() <= tol(n), f"N={n} dir={d}"
    if d == 0:
        got_ip = run(x, 0, inplace=True)
        assert np.array_equal(got_ip, got), f"in place N={n}"
