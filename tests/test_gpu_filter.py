"""SAR range compression (fft_exec_filter and range_compress) against the
FP64 oracle on the same seeded inputs: every one-pass length through the fused
kernel, multi-pass lengths through the passes run twice, in place, the filter
special cases (identity, delay), the matched filter on synthetic range lines,
full-size sampled rows, the gradient, and argument errors.

Bar: per row, ||y - y_ref|| <= 1e-6 * log2(N) * max|H| * ||x||: two FP32
transforms (5e-7 log2 N each, relative to their own input) around a product
with a filter of gain at most max|H|, which bounds ||y|| by max|H| ||x||.
"""
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


def tol(n: int) -> float:
    return 1e-6 * max(1.0, np.log2(n))


def assert_rc(got, x, H, what):
    ref = oracle.range_compress(x.astype(np.complex128), H.astype(np.complex128))
    g = np.asarray(got, dtype=np.complex128).reshape(ref.shape)
    scale = np.max(np.abs(H)) * np.sqrt(np.sum(np.abs(x.astype(np.complex128)) ** 2, axis=-1))
    err = np.sqrt(np.sum(np.abs(g - ref) ** 2, axis=-1)) / np.where(scale > 0, scale, 1.0)
    n = x.shape[-1]
    assert err.max() <= tol(n), f"{what}: max normalised error {err.max():.3e} > {tol(n):.2e} (row {err.argmax()})"


def run(x: np.ndarray, H: np.ndarray, config=None, inplace=False) -> np.ndarray:
    n = x.shape[-1]
    batch = x.size // n
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    Hd = torch.from_numpy(np.ascontiguousarray(H)).cuda()
    if config is None:
        p = gb.get_plan("1d", (n,), batch)
    else:
        p = gb.Plan("1d", (n,), batch, config=config)
    out = xd if inplace else torch.empty_like(xd)
    p.exec_filter_ptr(xd.data_ptr(), out.data_ptr(), Hd.data_ptr())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def jj_cols(lg):
    return 1 if lg >= 12 else (4096 >> lg if lg >= 4 else 256)


@pytest.mark.parametrize("lg", list(range(1, 15)))
def test_fused_every_length(lg):
    """Random filter, ragged last tile (batch not a multiple of the rows per CTA)."""
    n = 1 << lg
    batch = min(3 * jj_cols(lg) + 1, max(2, (1 << 17) // n))
    x = workloads.cgauss(n, batch, seed=4000 + lg)
    H = workloads.cgauss(n, 1, seed=4100 + lg)[0]
    assert_rc(run(x, H), x, H, f"N=2^{lg} batch={batch}")


@pytest.mark.parametrize("lg,batch", [(15, 3), (16, 2), (18, 2), (20, 1), (22, 1), (23, 1), (24, 1)])
def test_multipass(lg, batch):
    n = 1 << lg
    x = workloads.cgauss(n, batch, seed=4200 + lg)
    H = workloads.cgauss(n, 1, seed=4300 + lg)[0]
    assert_rc(run(x, H), x, H, f"multi-pass N=2^{lg}")


@pytest.mark.parametrize("cfg", [{"npass": 3}, {"npass": 2, "lg1": 6}, {"npass": 2, "lg1": 10, "c2": 2},
                                 {"npass": 2, "tma": 1}])
def test_multipass_configs(cfg):
    n = 1 << 16
    x = workloads.cgauss(n, 2, seed=4400)
    H = workloads.cgauss(n, 1, seed=4401)[0]
    assert_rc(run(x, H, config=cfg), x, H, f"2^16 {cfg}")


@pytest.mark.parametrize("cfg", [{"tma": 1}, {"halves": 2}])
def test_single_configs(cfg):
    """One-pass plans built with other kernels still run the fused kernel."""
    n = 1 << 12
    x = workloads.cgauss(n, 5, seed=4500)
    H = workloads.cgauss(n, 1, seed=4501)[0]
    assert_rc(run(x, H, config=cfg), x, H, f"2^12 {cfg}")


@pytest.mark.parametrize("lg", [10, 14, 17])
def test_in_place(lg):
    n = 1 << lg
    x = workloads.cgauss(n, 3, seed=4600 + lg)
    H = workloads.cgauss(n, 1, seed=4601 + lg)[0]
    assert_rc(run(x, H, inplace=True), x, H, f"in place N=2^{lg}")


@pytest.mark.parametrize("lg", [4, 12, 14, 16])
def test_identity_and_delay(lg):
    """H = 1 returns the input; H = W^{k d} delays every row by d samples."""
    n = 1 << lg
    x = workloads.cgauss(n, 2, seed=4700 + lg)
    ones = np.ones(n, np.complex64)
    y = run(x, ones)
    assert oracle.rel_l2(y, x) <= tol(n)
    d = n // 3 + 1
    k = np.arange(n)
    H = np.exp(-2j * np.pi * ((k * d) % n) / n).astype(np.complex64)
    assert oracle.rel_l2(run(x, H), np.roll(x, d, axis=-1)) <= tol(n)


@pytest.mark.parametrize("n,P", [(4096, 1000), (16384, 3000)])
def test_matched_filter_range_lines(n, P):
    """Synthetic SAR range lines with the closed-form matched filter: parity,
    and every single-target line compresses to a peak at its delay."""
    x = workloads.range_lines(n, 8, P, n_targets=6, seed=4800 + n)
    H = workloads.range_filter(n, P)
    assert_rc(run(x, H), x, H, f"range lines N={n}")
    x1 = workloads.range_lines(n, 4, P, n_targets=1, noise=0.0, seed=4900)
    y = np.abs(run(x1, H))
    ref = np.abs(oracle.range_compress(x1.astype(np.complex128), H.astype(np.complex128)))
    assert np.array_equal(np.argmax(y, axis=1), np.argmax(ref, axis=1))


@pytest.mark.parametrize("lg,batch", [(12, 16384), (14, 4096)])
def test_full_size_sampled(lg, batch):
    """The benchmark's shapes (2^26 points); rows sampled for the oracle."""
    n = 1 << lg
    x = workloads.cgauss(n, batch, seed=5000 + lg)
    H = workloads.range_filter(n, n // 4)
    y = run(x, H)
    rows = np.random.Generator(np.random.PCG64(lg)).choice(batch, size=24, replace=False)
    rows = np.concatenate([rows, [0, batch - 1]])
    assert_rc(y[rows], x[rows], H, f"full size N=2^{lg} sampled")


def test_range_compress_autograd():
    """L = sum |w y|^2, y = range_compress(x, H): dL/dx = A^H (2 w^2 y) with
    A^H the range compression by conj(H)."""
    n, batch = 2048, 3
    x = workloads.cgauss(n, batch, seed=5100)
    H = workloads.cgauss(n, 1, seed=5101)[0]
    w = workloads.real_weights(n, seed=5102)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    y = gb.range_compress(xt, torch.from_numpy(H).cuda())
    loss = (torch.abs(y * torch.from_numpy(w).cuda()) ** 2).sum()
    loss.backward()
    y64 = oracle.range_compress(x.astype(np.complex128), H.astype(np.complex128))
    g_ref = oracle.range_compress(2 * (w.astype(np.float64) ** 2) * y64, np.conj(H.astype(np.complex128)))
    assert oracle.rel_l2(xt.grad.cpu().numpy(), g_ref) <= 2 * tol(n)


@pytest.mark.parametrize("lg,batch", [(1, 3), (6, 70), (10, 9), (12, 5), (14, 3), (16, 2), (20, 1)])
def test_adjoint_direction(lg, batch):
    """fft_exec_filter_dir(FFT_ADJOINT) is range compression with conj(H):
    one-pass lengths through the fused kernel, longer ones through the passes
    run twice."""
    n = 1 << lg
    x = workloads.cgauss(n, batch, seed=5300 + lg)
    H = workloads.cgauss(n, 1, seed=5400 + lg)[0]
    xd, Hd = torch.from_numpy(x).cuda(), torch.from_numpy(H).cuda()
    p = gb.get_plan("1d", (n,), batch)
    out = torch.empty_like(xd)
    p.exec_filter_ptr(xd.data_ptr(), out.data_ptr(), Hd.data_ptr(), dir=L.FFT_ADJOINT)
    torch.cuda.synchronize()
    assert_rc(out.cpu().numpy(), x, np.conj(H), f"adjoint N=2^{lg}")


def test_range_compress_shapes_and_empty():
    n = 256
    x = workloads.cgauss(n, 6, seed=5200).reshape(2, 3, n)
    H = workloads.cgauss(n, 1, seed=5201)[0]
    y = gb.range_compress(torch.from_numpy(x).cuda(), torch.from_numpy(H).cuda()).cpu().numpy()
    assert_rc(y.reshape(6, n), x.reshape(6, n), H, "3-D input")
    e = gb.range_compress(torch.empty(0, n, dtype=torch.complex64, device="cuda"), torch.from_numpy(H).cuda())
    assert e.shape == (0, n)
    with pytest.raises(TypeError):
        gb.range_compress(torch.from_numpy(x).cuda(), torch.from_numpy(H[:128]).cuda())


def test_filter_errors():
    lib = L.load()
    d = torch.zeros(4096 * 2, dtype=torch.complex64, device="cuda")
    H = torch.ones(4096 + 1, dtype=torch.complex64, device="cuda")
    p = gb.get_plan("1d", (4096,), 2)
    nul = ctypes.c_void_p(0)
    dp = ctypes.c_void_p(d.data_ptr())
    assert lib.fft_exec_filter(p.handle, dp, dp, nul, nul) == -1
    assert lib.fft_exec_filter(None, dp, dp, ctypes.c_void_p(H.data_ptr()), nul) == -1
    odd = ctypes.c_void_p(H.data_ptr() + 4)
    assert lib.fft_exec_filter(p.handle, dp, dp, odd, nul) == -2
    Hp = ctypes.c_void_p(H.data_ptr())
    for bad in (L.FFT_INVERSE, L.FFT_INVERSE | L.FFT_ADJOINT, 7, -1):
        assert lib.fft_exec_filter_dir(p.handle, dp, dp, Hp, bad, nul) == -1
    p2 = gb.get_plan("2d", (64, 64), 1)
    assert lib.fft_exec_filter(p2.handle, dp, dp, ctypes.c_void_p(H.data_ptr()), nul) == -6
    ptc = gb.get_plan("1d", (4096,), 2, prec="tc_bf16")
    assert lib.fft_exec_filter(ptc.handle, dp, dp, ctypes.c_void_p(H.data_ptr()), nul) == -6
    torch.cuda.synchronize()
