"""Transforms that take two strided mixed-radix passes, against the FP64
oracle on the same seeded inputs:

* FP64 (complex128) 1-D lengths beyond one on-chip pass (N > 7168): the
  four-step split N = N1 N2 of Sec. 2.3.2, powers of two up to 2^24 and
  7-smooth lengths up to 7168^2;
* FP32 7-smooth lengths beyond one on-chip pass (N > 14336, not powers of two);
* 2-D transforms in FP64, and in FP32 with sides that are not powers of two.

Whole transforms are compared where the oracle finishes in seconds (the
radix-2 recursion for powers of two, the O(N^2) sum up to ~10^4 points);
longer 7-smooth lengths are compared at sampled outputs, each summed term by
term (oracle.dft_bins).  Ragged tiles (columns not a multiple of the
columns per CTA), every direction, in place (2-D), the workspace contract and
the autograd path are covered.

Bars: FP64 5e-15 log2 N + 2e-16 sqrt(N) per transform (the FP64 bar of the
one-pass kernel: u log2 N of FP64 plus the oracle's own O(N^2)-sum error),
FP32 5e-7 log2 N (the FP32 bar of every other path)."""
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

KIND_MIXED_PASSES = 6


def tol64(n: int) -> float:
    return 5e-15 * max(1.0, np.log2(n)) + 2e-16 * np.sqrt(n)


def tol32(n: int) -> float:
    return 5e-7 * max(1.0, np.log2(n))


def _exec(h, xt, out, d):
    lib = L.load()
    assert lib.fft_exec_dir(h, ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(out.data_ptr()), d,
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    torch.cuda.synchronize()


def run1d(x: np.ndarray, d: int, prec: int) -> np.ndarray:
    """One plan through the C ABI with a library-allocated workspace."""
    lib = L.load()
    batch, n = x.shape
    h = ctypes.c_void_p(lib.fft_plan_create(n, batch, d, prec))
    assert h.value, L.ERRORS.get(lib.fft_last_error())
    try:
        assert lib.fft_plan_kind(h) == KIND_MIXED_PASSES
        assert lib.fft_plan_launches(h) == 2
        esz = 16 if prec == L.FFT_PREC_FP64 else 8
        assert lib.fft_plan_workspace_bytes(h) == n * batch * esz
        xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        out = torch.empty_like(xt)
        # without a workspace the two-pass plan refuses to run
        assert lib.fft_exec(h, ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                            ctypes.c_void_p(0)) == -3   # FFT_ERR_NO_WORKSPACE
        assert lib.fft_plan_set_workspace(h, None) == 0
        _exec(h, xt, out, d)
        return out.cpu().numpy()
    finally:
        lib.fft_destroy(h)


def ref(x: np.ndarray, d: int) -> np.ndarray:
    x64 = x.astype(np.complex128)
    n = x.shape[-1]
    f = oracle.fft if (n & (n - 1)) == 0 else oracle.dft
    return {0: lambda: f(x64, oracle.FORWARD), 1: lambda: f(x64, oracle.INVERSE),
            2: lambda: f(x64, oracle.ADJOINT), 3: lambda: f(x64, oracle.FORWARD) / n}[d]()


def ref_bins(x: np.ndarray, ks, d: int) -> np.ndarray:
    x64 = x.astype(np.complex128)
    n = x.shape[-1]
    return {0: lambda: oracle.dft_bins(x64, ks, oracle.FORWARD), 1: lambda: oracle.dft_bins(x64, ks, oracle.INVERSE),
            2: lambda: oracle.dft_bins(x64, ks, oracle.ADJOINT),
            3: lambda: oracle.dft_bins(x64, ks, oracle.FORWARD) / n}[d]()


def sample_bins(n: int, count: int, seed: int) -> np.ndarray:
    g = np.random.Generator(np.random.PCG64(seed))
    return np.unique(np.concatenate([[0, 1, n // 2, n - 1], g.integers(0, n, count)]))


# ---- FP64 four-step ----------------------------------------------------------

@pytest.mark.parametrize("n", [1 << 13, 1 << 14, 1 << 15, 1 << 16, 1 << 18, 1 << 20])
def test_fp64_pow2_full(n):
    batch = 3 if n <= 1 << 16 else 2
    x = workloads.cgauss128(n, batch, seed=9500 + n % 1009)
    err = oracle.rel_l2_rows(run1d(x, 0, L.FFT_PREC_FP64), ref(x, 0)).max()
    assert err <= tol64(n), f"N={n}: {err:.2e}"


# splits N1 x N2: 7200 = 80 x 90 (ragged tiles in both passes), 10000 = 100 x 100,
# 14000 = 112 x 125 (odd rows)
@pytest.mark.parametrize("n,batch", [(7200, 2), (10000, 1), (14000, 1)])
def test_fp64_mixed_full(n, batch):
    x = workloads.cgauss128(n, batch, seed=9600 + n % 1013)
    err = oracle.rel_l2_rows(run1d(x, 0, L.FFT_PREC_FP64), ref(x, 0)).max()
    assert err <= tol64(n), f"N={n}: {err:.2e}"


# 21504 = 128 x 168, 10^5 = 250 x 400, 10^6 = 1000 x 1000, 3^13 = 729 x 2187,
# 5^9 = 625 x 3125, 7^8 = 2401 x 2401
@pytest.mark.parametrize("n", [3 * 7168, 100000, 10 ** 6, 3 ** 13, 5 ** 9, 7 ** 8])
def test_fp64_mixed_sampled(n):
    x = workloads.cgauss128(n, 2, seed=9700 + n % 1019)
    ks = sample_bins(n, 8, seed=n % 1021)
    got = run1d(x, 0, L.FFT_PREC_FP64)[:, ks]
    err = oracle.rel_l2_rows(got, ref_bins(x, ks, 0)).max()
    assert err <= tol64(n), f"N={n}: {err:.2e}"


def test_fp64_largest_lengths_sampled():
    """The largest FP64 lengths: 2^24 = 4096 x 4096 and 7168^2 = 51,380,224
    (both sub-transforms at the one-pass limit, one column per CTA; 7168 in
    the unpadded layout)."""
    for n in (1 << 24, 7168 * 7168):
        x = workloads.cgauss128(n, 1, seed=9800 + n % 1031)
        ks = sample_bins(n, 2, seed=n % 1033)
        got = run1d(x, 0, L.FFT_PREC_FP64)[:, ks]
        err = oracle.rel_l2_rows(got, ref_bins(x, ks, 0)).max()
        assert err <= tol64(n), f"N={n}: {err:.2e}"


@pytest.mark.parametrize("n", [1 << 14, 7200])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_fp64_directions(n, d):
    x = workloads.cgauss128(n, 2, seed=9900 + n % 1039 + d)
    err = oracle.rel_l2_rows(run1d(x, d, L.FFT_PREC_FP64), ref(x, d)).max()
    assert err <= tol64(n), f"N={n} dir={d}: {err:.2e}"


# ---- FP32 mixed-radix four-step ------------------------------------------------

# 15000 = 120 x 125, 16000 = 125 x 128
@pytest.mark.parametrize("n", [15000, 16000])
def test_fp32_mixed_full(n):
    x = workloads.cgauss(n, 1, seed=10000 + n % 1049)
    err = oracle.rel_l2_rows(run1d(x, 0, L.FFT_PREC_FP32), ref(x, 0)).max()
    assert err <= tol32(n), f"N={n}: {err:.2e}"


# 3^9 = 81 x 243, 20000 = 125 x 160, 10^6 = 1000 x 1000, 6^9 = 2916 x 3456,
# 14336 * 4096 = 7168 x 8192
@pytest.mark.parametrize("n,batch,nbins", [(3 ** 9, 3, 12), (20000, 2, 12), (10 ** 6, 2, 8), (6 ** 9, 2, 2),
                                           (14336 * 4096, 1, 2)])
def test_fp32_mixed_sampled(n, batch, nbins):
    x = workloads.cgauss(n, batch, seed=10100 + n % 1051)
    ks = sample_bins(n, nbins, seed=n % 1061)
    got = run1d(x, 0, L.FFT_PREC_FP32)[:, ks]
    err = oracle.rel_l2_rows(got, ref_bins(x, ks, 0)).max()
    assert err <= tol32(n), f"N={n}: {err:.2e}"


def test_fp32_largest_length_sampled():
    """The largest FP32 mixed-radix length, 14336^2 = 205,520,896 points:
    both passes of 14336 points, one column per CTA, unpadded."""
    n = 14336 * 14336
    x = workloads.cgauss(n, 1, seed=10150)
    ks = np.array([1, 12345677])
    got = run1d(x, 0, L.FFT_PREC_FP32)[:, ks]
    err = oracle.rel_l2_rows(got, ref_bins(x, ks, 0)).max()
    assert err <= tol32(n), f"N={n}: {err:.2e}"


@pytest.mark.parametrize("d", [1, 2, 3])
def test_fp32_mixed_directions(d):
    n = 15000
    x = workloads.uniform(n, 3, seed=10200 + d)
    ks = sample_bins(n, 12, seed=10210 + d)
    got = run1d(x, d, L.FFT_PREC_FP32)[:, ks]
    assert oracle.rel_l2_rows(got, ref_bins(x, ks, d)).max() <= tol32(n)


# ---- 2-D -------------------------------------------------------------------------

def run2d(x: np.ndarray, d: int, prec: int, inplace: bool = False) -> np.ndarray:
    lib = L.load()
    batch, ny, nx = x.shape
    h = ctypes.c_void_p(lib.fft_plan_create_2d(ny, nx, batch, d, prec))
    assert h.value, L.ERRORS.get(lib.fft_last_error())
    try:
        assert lib.fft_plan_kind(h) == KIND_MIXED_PASSES
        assert lib.fft_plan_workspace_bytes(h) == 0
        xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        out = xt if inplace else torch.empty_like(xt)
        _exec(h, xt, out, d)
        return out.cpu().numpy()
    finally:
        lib.fft_destroy(h)


def ref2d(x: np.ndarray, d: int) -> np.ndarray:
    x64 = x.astype(np.complex128)
    n = x.shape[-1] * x.shape[-2]
    return {0: lambda: oracle.fft2(x64, oracle.FORWARD), 1: lambda: oracle.fft2(x64, oracle.INVERSE),
            2: lambda: oracle.fft2(x64, oracle.ADJOINT), 3: lambda: oracle.fft2(x64, oracle.FORWARD) / n}[d]()


def err2d(got, want) -> float:
    b = got.shape[0]
    return float(oracle.rel_l2_rows(got.reshape(b, -1), want.reshape(b, -1)).max())


@pytest.mark.parametrize("ny,nx", [(2, 2), (64, 64), (12, 20), (1000, 7), (7, 1000), (256, 4096), (7168, 3),
                                   (3, 7168), (1024, 1024)])
def test_fp64_2d(ny, nx):
    batch = 2 if ny * nx <= 1 << 16 else 1
    x = workloads.cgauss128(ny * nx, batch, seed=10300 + ny + nx).reshape(batch, ny, nx)
    err = err2d(run2d(x, 0, L.FFT_PREC_FP64), ref2d(x, 0))
    assert err <= tol64(ny * nx), f"{ny}x{nx}: {err:.2e}"


@pytest.mark.parametrize("d", [1, 2, 3])
def test_fp64_2d_directions_in_place(d):
    ny, nx = 48, 80
    x = workloads.cgauss128(ny * nx, 3, seed=10400 + d).reshape(3, ny, nx)
    err = err2d(run2d(x, d, L.FFT_PREC_FP64, inplace=True), ref2d(x, d))
    assert err <= tol64(ny * nx)


@pytest.mark.parametrize("ny,nx", [(12, 20), (3, 64), (100, 360), (100, 1000), (625, 16), (14336, 2)])
def test_fp32_mixed_2d(ny, nx):
    batch = 2 if ny * nx <= 1 << 15 else 1
    x = workloads.cgauss(ny * nx, batch, seed=10500 + ny + nx).reshape(batch, ny, nx)
    err = err2d(run2d(x, 0, L.FFT_PREC_FP32), ref2d(x, 0))
    assert err <= tol32(ny * nx), f"{ny}x{nx}: {err:.2e}"


# every sub-length with a compiled schedule, as the column pass of a 2-D plan
# (ny x nx images, nx a multiple of 3 and at least the schedule's columns per
# CTA, so that the plan is a mixed-radix one; the rows of nx points run on the
# run-time kernel)
COMPILED = [64, 100, 120, 125, 128, 160, 200, 240, 250, 256, 320, 400, 500, 512, 625, 1000, 1024, 1250, 2000,
            2048, 2500, 3125, 4000, 4096]


@pytest.mark.parametrize("ny", COMPILED)
def test_fp32_compiled_sub_lengths(ny):
    nx = 48 if ny <= 256 else (24 if ny <= 512 else 12)
    batch = 2 if ny < 1000 else 1
    x = workloads.cgauss(ny * nx, batch, seed=10550 + ny).reshape(batch, ny, nx)
    err = err2d(run2d(x, 0, L.FFT_PREC_FP32), ref2d(x, 0))
    assert err <= tol32(ny * nx), f"{ny}x{nx}: {err:.2e}"


@pytest.mark.parametrize("d", [1, 2, 3])
def test_fp32_mixed_2d_directions_in_place(d):
    ny, nx = 30, 96
    x = workloads.uniform(ny * nx, 2, seed=10600 + d).reshape(2, ny, nx)
    err = err2d(run2d(x, d, L.FFT_PREC_FP32, inplace=True), ref2d(x, d))
    assert err <= tol32(ny * nx)


# ---- the Python API ----------------------------------------------------------------

def test_api_fp64_long_and_2d_with_gradient():
    """gb.fft / gb.ifft / gb.fft2 on complex128 beyond one pass, and the
    gradient of L = sum |w X|^2 against the oracle's 2 F^H (w^2 F x)."""
    n = 1 << 15
    x = workloads.cgauss128(n, 2, seed=10700)
    w = workloads.real_weights(n, seed=10701).astype(np.float64)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    X = gb.fft(xt)
    assert X.dtype == torch.complex128
    assert oracle.rel_l2_rows(X.detach().cpu().numpy(), oracle.fft(x)).max() <= tol64(n)
    back = gb.ifft(X).detach().cpu().numpy()
    assert oracle.rel_l2_rows(back, x).max() <= 2 * tol64(n)
    (torch.abs(X * torch.from_numpy(w).cuda()) ** 2).sum().backward()
    g_ref = np.stack([oracle.spectral_loss_grad(r, w) for r in x])
    assert oracle.rel_l2(xt.grad.cpu().numpy(), g_ref) <= 4 * tol64(n)
    img = workloads.cgauss128(60 * 48, 2, seed=10702).reshape(2, 60, 48)
    it = torch.from_numpy(img).cuda()
    assert err2d(gb.fft2(it).cpu().numpy(), oracle.fft2(img)) <= tol64(60 * 48)
    assert err2d(gb.ifft2(gb.fft2(it)).cpu().numpy(), img) <= 2 * tol64(60 * 48)
