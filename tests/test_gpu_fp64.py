"""FP64 (complex128) one-pass transforms against the FP64 oracle on the same
seeded inputs: powers of two up to 4096 and 7-smooth lengths up to 7168, every
direction, in place, the gradient, and the limits (the two-pass FP64 lengths
and FP64 2-D are in test_gpu_mixed_passes.py).

Bar: relative L2 error of every transform <= 5e-15 * log2(N) + 2e-16 * sqrt(N):
FP64 arithmetic with twiddles correct to an ulp gives errors of order
u log2 N (u = 2^-53), and the oracle's O(N^2) sum (the route for every N that
is not a power of two, and for N <= 1024) adds its own ~u sqrt(N).  An FP32
path would miss this by six orders of magnitude."""
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

POW2 = [2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096]
MIXED = [3, 5, 6, 7, 12, 15, 100, 105, 360, 1000, 2187, 2401, 3000, 5000, 6000, 7000, 7168]


def tol(n: int) -> float:
    return 5e-15 * max(1.0, np.log2(n)) + 2e-16 * np.sqrt(n)


def c128(n, batch, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    return g.normal(0, np.sqrt(0.5), (batch, n)) + 1j * g.normal(0, np.sqrt(0.5), (batch, n))


def run(x: np.ndarray, d: int, inplace=False) -> np.ndarray:
    lib = L.load()
    batch, n = x.shape
    h = ctypes.c_void_p(lib.fft_plan_create(n, batch, d, L.FFT_PREC_FP64))
    assert h.value, L.ERRORS.get(lib.fft_last_error())
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = xt if inplace else torch.empty_like(xt)
    assert lib.fft_exec(h, ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    torch.cuda.synchronize()
    lib.fft_destroy(h)
    return out.cpu().numpy()


def ref(x, d):
    n = x.shape[-1]
    return {0: lambda: oracle.transform(x, oracle.FORWARD), 1: lambda: oracle.transform(x, oracle.INVERSE),
            2: lambda: oracle.transform(x, oracle.ADJOINT), 3: lambda: oracle.transform(x, oracle.FORWARD) / n}[d]()


@pytest.mark.parametrize("n", POW2 + MIXED)
def test_forward(n):
    c = max(1, 2048 // n)
    batch = min(2 * c + 1, 9) if n <= 1000 else 2
    x = c128(n, batch, 9000 + n)
    err = oracle.rel_l2_rows(run(x, 0), ref(x, 0)).max()
    assert err <= tol(n), f"N={n}: {err:.2e}"


@pytest.mark.parametrize("n", [16, 1000, 4096, 7000])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_directions(n, d):
    x = c128(n, 3, 9100 + n + d)
    assert oracle.rel_l2_rows(run(x, d), ref(x, d)).max() <= tol(n)


@pytest.mark.parametrize("n", [4, 360, 4096, 7168])
def test_in_place(n):
    x = c128(n, 3, 9200 + n)
    assert oracle.rel_l2_rows(run(x, 0, inplace=True), ref(x, 0)).max() <= tol(n)


def test_api_complex128_and_gradient():
    n = 2048
    x = c128(n, 2, 9300)
    w = np.random.Generator(np.random.PCG64(9301)).uniform(0, 1, n)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    X = gb.fft(xt)
    assert X.dtype == torch.complex128
    back = gb.ifft(X).detach().cpu().numpy()
    assert oracle.rel_l2_rows(back, x).max() <= 2 * tol(n)
    (torch.abs(X * torch.from_numpy(w).cuda()) ** 2).sum().backward()
    g_ref = np.stack([oracle.spectral_loss_grad(r, w) for r in x])
    assert oracle.rel_l2(xt.grad.cpu().numpy(), g_ref) <= 4 * tol(n)


def test_limits():
    lib = L.load()
    assert lib.fft_plan_create(1 << 25, 1, 0, L.FFT_PREC_FP64) is None    # no split into two FP64 passes
    assert lib.fft_last_error() == -6
    assert lib.fft_plan_create(11, 1, 0, L.FFT_PREC_FP64) is None         # prime factor above 7
    assert lib.fft_last_error() == -1
    assert lib.fft_plan_create_2d(64, 7200, 1, 0, L.FFT_PREC_FP64) is None  # side beyond one FP64 pass
    assert lib.fft_last_error() == -6
    for n in (8192, 7200):                                                   # two passes from 7169 on
        h = ctypes.c_void_p(lib.fft_plan_create(n, 1, 0, L.FFT_PREC_FP64))
        assert h.value and lib.fft_plan_kind(h) == 6
        lib.fft_destroy(h)
    h = ctypes.c_void_p(lib.fft_plan_create(1024, 2, 0, L.FFT_PREC_FP64))
    buf = torch.zeros(2 * 1024 + 1, dtype=torch.complex128, device="cuda")
    p8 = ctypes.c_void_p(buf.data_ptr() + 8)
    assert lib.fft_exec(h, p8, p8, ctypes.c_void_p(0)) == -2                # 16-byte alignment
    lib.fft_destroy(h)
    with pytest.raises(ValueError):
        gb.fft(torch.zeros(16, dtype=torch.complex128, device="cuda"), prec="fp32")


# ---- FP64 real-data transforms (float64 rows, complex128 spectra) ----------------

def real64(n, batch, seed):
    return np.random.Generator(np.random.PCG64(seed)).uniform(-1.0, 1.0, (batch, n))


def half64(n, batch, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    return g.normal(0, 1, (batch, n // 2 + 1)) + 1j * g.normal(0, 1, (batch, n // 2 + 1))


# one-pass inner lengths (n/2 <= 7168, powers of two and 7-smooth, odd n/2
# included) and two-pass ones (n/2 > 7168)
@pytest.mark.parametrize("n", [4, 6, 16, 30, 1024, 2000, 2250, 14336, 1 << 14, 20000, 1 << 20])
def test_real_fp64_matches_oracle(n):
    batch = 3 if n <= 1 << 14 else 1
    x = real64(n, batch, 9400 + n % 997)
    X = gb.rfft(torch.from_numpy(x).cuda())
    assert X.dtype == torch.complex128 and X.shape == (batch, n // 2 + 1)
    Xh = X.cpu().numpy()
    H = half64(n, batch, 9500 + n % 997)
    back = gb.irfft(torch.from_numpy(H).cuda(), n)
    assert back.dtype == torch.float64 and back.shape == (batch, n)
    if n <= 1 << 14 or (n & (n - 1)) == 0:
        assert oracle.rel_l2_rows(Xh, oracle.rfft(x)).max() <= tol(n), f"rfft N={n}"
        assert oracle.rel_l2_rows(back.cpu().numpy(), oracle.irfft(H, n)).max() <= tol(n), f"irfft N={n}"
    else:
        ks = np.array([0, 1, 7, n // 4, n // 2 - 1, n // 2])
        assert oracle.rel_l2_rows(Xh[:, ks], oracle.dft_bins(x.astype(np.complex128), ks)).max() <= tol(n)
    rt = gb.irfft(X, n).cpu().numpy()
    assert oracle.rel_l2_rows(rt, x).max() <= 2 * tol(n), f"round trip N={n}"


@pytest.mark.parametrize("n", [16, 2000, 1 << 14])
def test_real_fp64_adjoints_and_gradient(n):
    """The adjoints of both directions (the gradients of rfft and irfft)
    against their definitions, through autograd."""
    x = real64(n, 2, 9600 + n)
    w = np.random.Generator(np.random.PCG64(9601 + n)).uniform(0, 1, n // 2 + 1)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    X = gb.rfft(xt)
    (torch.abs(X * torch.from_numpy(w).cuda()) ** 2).sum().backward()
    # L = sum_k w_k^2 |X_k|^2 over the kept bins: dL/dx_m = Re sum_k 2 w_k^2 X_k W^{-mk} (k <= n/2)
    Xr = oracle.rfft(x)
    g = np.zeros((2, n), dtype=np.complex128)
    g[:, : n // 2 + 1] = 2 * w ** 2 * Xr
    g_ref = oracle.transform(g, oracle.ADJOINT).real
    assert oracle.rel_l2(xt.grad.cpu().numpy(), g_ref) <= 4 * tol(n)
    H = half64(n, 2, 9700 + n)
    Ht = torch.from_numpy(H).cuda().requires_grad_(True)
    y = gb.irfft(Ht, n)
    v = real64(n, 2, 9701 + n)
    (y * torch.from_numpy(v).cuda()).sum().backward()
    # d/dH of sum v * irfft(H): Eq. 1 of v with bins 1..n/2-1 times 2/n and bins 0, n/2 times 1/n
    V = oracle.rfft(v)
    scale = np.full(n // 2 + 1, 2.0 / n)
    scale[0] = scale[-1] = 1.0 / n
    assert oracle.rel_l2(Ht.grad.cpu().numpy(), V * scale) <= 4 * tol(n)
