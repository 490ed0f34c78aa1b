"""Backpropagation through the hand-written adjoint: gradients of the spectral
loss L = sum |w * FFT(x)|^2 against the oracle gradient 2 F^H (w^2 F x) and
against FP64 finite differences, plus the adjoint identity on the GPU."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_1707_07263_gb300 as gb
from paper_1707_07263_gb300 import workloads

pytestmark = pytest.mark.gpu


def _loss_grad_gpu(x: np.ndarray, w: np.ndarray):
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    wt = torch.from_numpy(w).cuda()
    y = gb.fft(xt)
    loss = (torch.abs(y * wt) ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    return float(loss.item()), xt.grad.cpu().numpy()


@pytest.mark.parametrize("lg", [1, 4, 8, 12, 14, 16, 20])
def test_fft_grad_matches_oracle(lg):
    n = 1 << lg
    x = workloads.cgauss(n, 1, seed=700 + lg)[0]
    w = workloads.real_weights(n, seed=800 + lg)
    loss, g = _loss_grad_gpu(x, w)
    g_ref = oracle.spectral_loss_grad(x.astype(np.complex128), w.astype(np.float64))
    assert oracle.rel_l2(g, g_ref) <= 1e-6 * max(1, lg)
    assert abs(loss - oracle.spectral_loss(x.astype(np.complex128), w.astype(np.float64))) <= 1e-5 * abs(loss)


@pytest.mark.parametrize("n", [16, 256])
def test_fft_grad_finite_differences(n):
    """FP64 central differences of the oracle loss (exact for a quadratic)
    against the GPU gradient, component by component."""
    x = workloads.cgauss(n, 1, seed=900 + n)[0]
    w = workloads.real_weights(n, seed=901 + n)
    _, g = _loss_grad_gpu(x, w)
    x64, w64 = x.astype(np.complex128), w.astype(np.float64)
    h = 1e-3
    fd = np.empty(n, complex)
    for i in range(n):
        e = np.zeros(n, complex)
        e[i] = h
        dre = (oracle.spectral_loss(x64 + e, w64) - oracle.spectral_loss(x64 - e, w64)) / (2 * h)
        dim = (oracle.spectral_loss(x64 + 1j * e, w64) - oracle.spectral_loss(x64 - 1j * e, w64)) / (2 * h)
        fd[i] = dre + 1j * dim
    assert oracle.rel_l2(g, fd) <= 1e-6 * np.log2(n)


def test_ifft_grad():
    """y = IFFT(x): the gradient of sum |y|^2 w^2 is 2 (1/N) F (w^2 y)."""
    n = 1024
    x = workloads.cgauss(n, 1, seed=11)[0]
    w = workloads.real_weights(n, seed=12)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    wt = torch.from_numpy(w).cuda()
    y = gb.ifft(xt)
    (torch.abs(y * wt) ** 2).sum().backward()
    y64 = oracle.transform(x.astype(np.complex128), oracle.INVERSE)
    g_ref = 2.0 * oracle.transform((w.astype(np.float64) ** 2) * y64, oracle.FORWARD) / n
    assert oracle.rel_l2(xt.grad.cpu().numpy(), g_ref) <= 1e-6 * 10


def test_fft2_and_many_grads():
    ny, nx = 64, 128
    x = workloads.cgauss(ny * nx, 1, seed=21).reshape(ny, nx)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    (torch.abs(gb.fft2(xt)) ** 2).sum().backward()
    # sum |F2 x|^2 = N sum |x|^2 (Parseval) -> gradient 2 N x
    assert oracle.rel_l2(xt.grad.cpu().numpy(), 2 * ny * nx * x.astype(np.complex128)) <= 1e-6 * 13

    lengths = [256, 4096, 1 << 15, 32]
    xp = workloads.packed_cgauss(lengths, seed=22)
    w = workloads.real_weights(len(xp), seed=23)
    xt = torch.from_numpy(xp).cuda().requires_grad_(True)
    wt = torch.from_numpy(w).cuda()
    (torch.abs(gb.fft_many(xt, lengths) * wt) ** 2).sum().backward()
    o = 0
    g = xt.grad.cpu().numpy()
    for n in lengths:
        ref = oracle.spectral_loss_grad(xp[o:o + n].astype(np.complex128), w[o:o + n].astype(np.float64))
        assert oracle.rel_l2(g[o:o + n], ref) <= 1e-6 * np.log2(n)
        o += n


@pytest.mark.parametrize("lg", [10, 18])
def test_adjoint_identity(lg):
    """<F x, y> = <x, F^H y> with F^H the library's adjoint direction."""
    n = 1 << lg
    x = torch.from_numpy(workloads.cgauss(n, 1, seed=31)[0]).cuda()
    y = torch.from_numpy(workloads.cgauss(n, 1, seed=32)[0]).cuda()
    p = gb.get_plan("1d", (n,), 1)
    fx = p(x, dir=0)
    fhy = p(y, dir=2)
    lhs = torch.vdot(y.to(torch.complex128), fx.to(torch.complex128)).item()
    rhs = torch.vdot(fhy.to(torch.complex128), x.to(torch.complex128)).item()
    # each side carries an FP32 transform error of ~eps * ||F x|| = eps * sqrt(n) ||x||
    bound = 5e-7 * lg * np.sqrt(n) * float(torch.linalg.norm(x)) * float(torch.linalg.norm(y))
    assert abs(lhs - rhs) <= bound
