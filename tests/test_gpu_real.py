"""Real-data transforms (fft_plan_create_r2c, rfft / irfft) against the FP64
oracle on the same seeded inputs: every fused length 2^2..2^15 with ragged
batches, multi-pass lengths, the ignored imaginary parts of X[0] and X[N/2],
round trips, gradients, and argument errors.

Bar: relative L2 error of every row <= 5e-7 * log2(N), the FP32 bound of the
complex transforms (one transform of length N/2 plus a split step of a few
roundings per value)."""
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
    return 5e-7 * max(1.0, np.log2(n))


def real_rows(n, batch, seed):
    return workloads.uniform(n, batch, seed=seed).real.astype(np.float32).copy()


def half_spectrum(n, batch, seed):
    return workloads.cgauss(n // 2 + 1, batch, seed=seed)


def jj_cols(lg):
    return 1 if lg >= 12 else (4096 >> lg if lg >= 4 else 256)


def batch_for(n):
    lgm = int(np.log2(n)) - 1
    return min(3 * jj_cols(lgm) + 1, max(2, (1 << 17) // n)) if lgm <= 14 else max(1, (1 << 21) // n)


# 2^16..2^22: the split folded into the row pass of the complex plan
@pytest.mark.parametrize("lg", list(range(2, 16)) + [16, 17, 19, 20, 21, 22])
def test_rfft_matches_oracle(lg):
    n = 1 << lg
    batch = batch_for(n)
    x = real_rows(n, batch, seed=6000 + lg)
    got = gb.rfft(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.rfft(x.astype(np.float64))
    assert got.shape == (batch, n // 2 + 1)
    assert oracle.rel_l2_rows(got, ref).max() <= tol(n), f"N=2^{lg}"


# 2^16..2^21: the split folded into the column pass of the complex plan
@pytest.mark.parametrize("lg", list(range(2, 16)) + [16, 17, 18, 19, 20, 21])
def test_irfft_matches_oracle(lg):
    """Random half spectra, including nonzero Im X[0] and Im X[N/2], which the
    transform must ignore."""
    n = 1 << lg
    batch = batch_for(n)
    X = half_spectrum(n, batch, seed=6100 + lg)
    got = gb.irfft(torch.from_numpy(X).cuda(), n).cpu().numpy()
    ref = oracle.irfft(X.astype(np.complex128), n)
    assert got.shape == (batch, n)
    assert oracle.rel_l2_rows(got, ref).max() <= tol(n), f"N=2^{lg}"


@pytest.mark.parametrize("lg", [4, 11, 15, 18])
def test_round_trip(lg):
    n = 1 << lg
    x = real_rows(n, 5, seed=6200 + lg)
    xt = torch.from_numpy(x).cuda()
    back = gb.irfft(gb.rfft(xt), n).cpu().numpy()
    assert oracle.rel_l2_rows(back, x).max() <= 2 * tol(n)


@pytest.mark.parametrize("lg", [22, 24])
def test_large_sampled(lg):
    """Long rows (2^22: both splits folded; 2^24: the complex plan plus a split
    kernel); whole rows checked."""
    n = 1 << lg
    x = real_rows(n, 2, seed=6300 + lg)
    got = gb.rfft(torch.from_numpy(x).cuda()).cpu().numpy()
    assert oracle.rel_l2_rows(got, oracle.rfft(x.astype(np.float64))).max() <= tol(n)
    X = half_spectrum(n, 1, seed=6301 + lg)
    got2 = gb.irfft(torch.from_numpy(X).cuda(), n).cpu().numpy()
    assert oracle.rel_l2_rows(got2, oracle.irfft(X.astype(np.complex128), n)).max() <= tol(n)


@pytest.mark.parametrize("lg,batch", [(13, 8192), (15, 2048), (16, 1024)])
def test_full_size_sampled(lg, batch):
    """The shapes of the real-data workload (2^26 reals), both directions,
    rows sampled."""
    n = 1 << lg
    x = real_rows(n, batch, seed=6400 + lg)
    got = gb.rfft(torch.from_numpy(x).cuda()).cpu().numpy()
    rows = np.concatenate([np.random.Generator(np.random.PCG64(lg)).choice(batch, 16, replace=False), [0, batch - 1]])
    assert oracle.rel_l2_rows(got[rows], oracle.rfft(x[rows].astype(np.float64))).max() <= tol(n)
    X = half_spectrum(n, batch, seed=6450 + lg)
    back = gb.irfft(torch.from_numpy(X).cuda(), n).cpu().numpy()
    assert oracle.rel_l2_rows(back[rows], oracle.irfft(X[rows].astype(np.complex128), n)).max() <= tol(n)


def test_rfft_gradient():
    """L = sum_k w_k |X_k|^2, X = rfft(x): dL/dx_n = Re(sum_{k<=N/2} g_k W^{-nk})
    with g = 2 w^2 X, written here as N * Re(Eq. 2 of g zero-padded to N)."""
    n, batch = 1024, 3
    x = real_rows(n, batch, seed=6500)
    w = workloads.real_weights(n // 2 + 1, seed=6501)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    X = gb.rfft(xt)
    (torch.from_numpy(w).cuda() * torch.abs(X) ** 2).sum().backward()
    X64 = oracle.rfft(x.astype(np.float64))
    g = 2 * w.astype(np.float64) * X64
    pad = np.zeros((batch, n), complex)
    pad[:, : n // 2 + 1] = g
    ref = n * oracle.transform(pad, oracle.INVERSE).real
    assert oracle.rel_l2(xt.grad.cpu().numpy(), ref) <= 2 * tol(n)


def test_irfft_gradient_finite_differences():
    """L = sum_n w_n x_n^2, x = irfft(X): FP64 central differences of the
    oracle against the GPU gradient, every real and imaginary part."""
    n = 16
    X = half_spectrum(n, 1, seed=6600)[0]
    w = workloads.real_weights(n, seed=6601).astype(np.float64)
    Xt = torch.from_numpy(X).cuda().requires_grad_(True)
    x = gb.irfft(Xt, n)
    (torch.from_numpy(w.astype(np.float32)).cuda() * x ** 2).sum().backward()
    X64 = X.astype(np.complex128)

    def loss(Z):
        return float(np.sum(w * oracle.irfft(Z, n) ** 2))

    h = 1e-4
    fd = np.empty(n // 2 + 1, complex)
    for k in range(n // 2 + 1):
        e = np.zeros(n // 2 + 1, complex)
        e[k] = h
        fd[k] = (loss(X64 + e) - loss(X64 - e)) / (2 * h) + 1j * (loss(X64 + 1j * e) - loss(X64 - 1j * e)) / (2 * h)
    assert oracle.rel_l2(Xt.grad.cpu().numpy(), fd) <= 1e-5


@pytest.mark.parametrize("lg", [2, 3, 5, 8, 11, 12, 15, 16, 18, 20, 21, 22])
def test_real_adjoints_match_oracle(lg):
    """The adjoints of the real transforms (FFT_ADJOINT and FFT_INVERSE |
    FFT_ADJOINT on a real plan) against their definitions written with the
    oracle:  R2C^T g = Re(sum_{k<=n/2} g_k W^{-mk})  (Eq. 4 over the kept bins,
    i.e. the oracle's adjoint transform of g zero-padded to n, real part), and
    C2R^T g = Eq. 1 of g with bins 1..n/2-1 times 2/n and bins 0, n/2 times 1/n.
    Also the adjoint identity <R2C x, g> = <x, R2C^T g> on the GPU's results."""
    n = 1 << lg
    h = n // 2
    batch = batch_for(n)
    p = gb.get_plan("r2c", (n,), batch)
    g = half_spectrum(n, batch, seed=6700 + lg)           # nonzero Im g[0], Im g[n/2] must not enter
    gt = torch.from_numpy(g).cuda()
    y = torch.empty(batch, n, dtype=torch.float32, device="cuda")
    p.exec_ptr(gt.data_ptr(), y.data_ptr(), L.FFT_ADJOINT)
    pad = np.zeros((batch, n), complex)
    pad[:, : h + 1] = g.astype(np.complex128)
    ref = oracle.transform(pad, oracle.ADJOINT).real
    yh = y.cpu().numpy()
    assert oracle.rel_l2_rows(yh, ref).max() <= tol(n), f"R2C adjoint N=2^{lg}"

    r = real_rows(n, batch, seed=6800 + lg)
    rt = torch.from_numpy(r).cuda()
    c = torch.empty(batch, h + 1, dtype=torch.complex64, device="cuda")
    p.exec_ptr(rt.data_ptr(), c.data_ptr(), L.FFT_INVERSE | L.FFT_ADJOINT)
    wts = np.full(h + 1, 2.0 / n)
    wts[0] = wts[h] = 1.0 / n
    ref2 = oracle.rfft(r.astype(np.float64)) * wts
    assert oracle.rel_l2_rows(c.cpu().numpy(), ref2).max() <= tol(n), f"C2R adjoint N=2^{lg}"

    # <R2C r, g>_R = <r, R2C^T g>: both sides from the GPU's own outputs
    X = gb.rfft(rt).cpu().numpy().astype(np.complex128)
    lhs = np.sum((np.conj(X) * g.astype(np.complex128)).real, axis=-1)
    rhs = np.sum(r.astype(np.float64) * yh.astype(np.float64), axis=-1)
    scale = np.linalg.norm(X, axis=-1) * np.linalg.norm(g, axis=-1)
    assert np.max(np.abs(lhs - rhs) / scale) <= tol(n)


def test_real_plan_errors():
    lib = L.load()
    p = gb.get_plan("r2c", (1024,), 2)
    d = torch.zeros(4096, dtype=torch.complex64, device="cuda")
    e = torch.zeros(4096, dtype=torch.complex64, device="cuda")
    nul = ctypes.c_void_p(0)
    dp, ep = ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(e.data_ptr())
    assert lib.fft_exec_dir(p.handle, dp, ep, 4, nul) == -1            # no such direction
    assert lib.fft_exec_dir(p.handle, dp, dp, 2, nul) == -1            # adjoint, in place
    assert lib.fft_exec_dir(p.handle, dp, dp, 0, nul) == -1            # in place
    assert lib.fft_exec_dir(p.handle, ctypes.c_void_p(d.data_ptr() + 4), ep, 0, nul) == -2
    assert lib.fft_plan_kind(p.handle) == 4
    h = ctypes.c_void_p(lib.fft_plan_create_r2c(1 << 18, 2, 0))        # multi-pass, no workspace set
    assert h.value and lib.fft_plan_workspace_bytes(h) > 0
    assert lib.fft_exec_dir(h, dp, ep, 0, nul) == -3
    lib.fft_destroy(h)
    with pytest.raises(ValueError):
        gb.irfft(d[:10], 16)
    torch.cuda.synchronize()
