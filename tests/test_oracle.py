"""CPU-only tests that pin the FP64 oracle (no GPU, no CUDA library)."""
from __future__ import annotations

import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import oracle_pins as pins


@pytest.fixture(scope="module")
def lib():
    return oracle.load_library()


@pytest.mark.parametrize("check", pins.ALL_CHECKS, ids=lambda c: c.__name__)
def test_pin(lib, check):
    check(lib)


def test_rejects_bad_arguments(lib):
    with pytest.raises(ValueError):
        oracle.fft(np.ones(12, complex), lib=lib)   # not a power of two
    with pytest.raises(ValueError):
        oracle.fft(np.ones(8, complex), dir=5, lib=lib)
    # the O(N^2) sum accepts any length (Eq. 1 has no power-of-two condition)
    x = pins._cvec(12, seed=3)
    assert oracle.rel_l2(oracle.dft(x, lib=lib), np.fft.fft(x)) < 1e-14


def test_transform_route(lib):
    x = pins._cvec(2048, seed=5)
    assert oracle.rel_l2(oracle.transform(x), np.fft.fft(x)) < 1e-13
    y = pins._cvec(256, seed=6)
    assert oracle.rel_l2(oracle.transform(y), np.fft.fft(y)) < 1e-13


@pytest.mark.parametrize("n", [16, 64, 256])
def test_loss_gradient_finite_differences(n):
    """L = sum |w X|^2 is quadratic in (Re x, Im x), so a central difference is
    exact up to rounding: compare every component of the oracle gradient."""
    g = np.random.Generator(np.random.PCG64(n))
    x = g.standard_normal(n) + 1j * g.standard_normal(n)
    w = g.uniform(0, 1, n)
    grad = oracle.spectral_loss_grad(x, w)
    h = 1e-3
    fd = np.empty(n, complex)
    for i in range(n):
        for part, unit in ((0, 1.0), (1, 1j)):
            xp = x.copy()
            xm = x.copy()
            xp[i] += h * unit
            xm[i] -= h * unit
            d = (oracle.spectral_loss(xp, w) - oracle.spectral_loss(xm, w)) / (2 * h)
            if part == 0:
                fd[i] = d
            else:
                fd[i] += 1j * d
    assert oracle.rel_l2(grad, fd) < 1e-9


def test_loss_gradient_closed_form():
    """With w = 1, L = ||F x||^2 = N ||x||^2 (Parseval), so the gradient is 2 N x."""
    n = 128
    g = np.random.Generator(np.random.PCG64(9))
    x = g.standard_normal(n) + 1j * g.standard_normal(n)
    assert oracle.rel_l2(oracle.spectral_loss_grad(x, np.ones(n)), 2 * n * x) < 1e-13
    assert abs(oracle.spectral_loss(x, np.ones(n)) - n * np.sum(np.abs(x) ** 2)) < 1e-10 * n * n


# --- the pins must catch plausible mistakes ---------------------------------
# Each mutation is planted in a temporary copy of the oracle's C source, on the
# CPU; the battery above must then fail at least once.
MUTATIONS = {
    "wrong_sign": ("*wi = (double)s * sin(a);", "*wi = -(double)s * sin(a);"),
    "dropped_term": ("acc_i += xr * wi + xi * wr;", "acc_i += xr * wi;"),
    "butterfly_sign": ("y[2 * (h + k)] = er - tr;", "y[2 * (h + k)] = er + tr;"),
    "butterfly_index": ("oracle_w(k, n, s, &wr, &wi);", "oracle_w(k, h, s, &wr, &wi);"),
    "no_inverse_scale": ("return dir == 1 ? 1.0 / (double)n : 1.0;", "return 1.0;"),
    "transposed_2d": ("col[2 * y] = out[2 * (y * nx + x)];", "col[2 * y] = out[2 * (x * ny + y)];"),  # in bounds
    "swapped_halves": ("fft_rec(h, x, 2 * stride, y, s);", "fft_rec(h, x + 2 * stride, 2 * stride, y, s);"),
    "bins_wrong_output": ("(unsigned __int128)j * (unsigned __int128)bin)", "(unsigned __int128)j * (unsigned __int128)b)"),
    "bins_dropped_term": ("sum_r += in[2 * j] * wr - in[2 * j + 1] * wi;", "sum_r += in[2 * j] * wr;"),
}


def _mutated_lib(tmpdir, name, old, new):
    with open(os.path.join(os.path.dirname(oracle.__file__), "fft_oracle.c")) as f:
        src = f.read()
    assert old in src, f"mutation {name}: anchor not found"
    path = os.path.join(tmpdir, f"{name}.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new, 1))
    so = os.path.join(tmpdir, f"lib{name}.so")
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", path, "-o", so, "-lm"])
    return oracle.load_library(so)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(name):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    old, new = MUTATIONS[name]
    with tempfile.TemporaryDirectory() as d:
        lib = _mutated_lib(d, name, old, new)
        failures = 0
        for check in pins.ALL_CHECKS:
            try:
                check(lib)
            except (AssertionError, ValueError):
                failures += 1
        assert failures > 0, f"no pin caught mutation {name}"


# Plausible mistakes in composing the range compression (planted in a copy of
# the function, on the CPU); its pin must fail for each.
RC_MUTATIONS = {
    "filter_conjugated": lambda x, H: oracle.transform(oracle.transform(x) * np.conj(H), oracle.INVERSE),
    "adjoint_not_inverse": lambda x, H: oracle.transform(oracle.transform(x) * H, oracle.ADJOINT),
    "forward_twice": lambda x, H: oracle.transform(oracle.transform(x) * H, oracle.FORWARD),
    "filter_reversed": lambda x, H: oracle.transform(oracle.transform(x) * np.asarray(H)[::-1], oracle.INVERSE),
    "filter_on_input": lambda x, H: oracle.transform(oracle.transform(np.asarray(x) * H), oracle.INVERSE),
}


@pytest.mark.parametrize("name", sorted(RC_MUTATIONS))
def test_range_pin_catches_mutation(lib, name):
    with pytest.raises(AssertionError):
        pins.check_range_compress(lib, rc=RC_MUTATIONS[name])


def test_range_compress_rejects_bad_filter():
    with pytest.raises(ValueError):
        oracle.range_compress(np.ones((2, 8)), np.ones(4))


def test_range_workload_compresses():
    """The synthetic SAR lines and the closed-form matched filter fit each
    other: one noiseless echo per line compresses to a sharp peak at its
    delay (the generator draws noise, amplitudes, phases, then delays)."""
    from paper_1707_07263_gb300 import workloads
    n, P, seed = 4096, 1000, 5
    x = workloads.range_lines(n, 4, P, n_targets=1, noise=0.0, seed=seed)
    y = np.abs(oracle.range_compress(x, workloads.range_filter(n, P)))
    g = np.random.Generator(np.random.PCG64(seed))
    g.normal(size=(4, n)), g.normal(size=(4, n)), g.uniform(size=(4, 1)), g.uniform(size=(4, 1))
    delays = g.integers(0, n, size=(4, 1)).ravel()
    assert np.array_equal(np.argmax(y, axis=1), delays)
    assert np.all(y.max(axis=1) > 1000 * np.median(y, axis=1))


# Plausible mistakes in the real-data transforms (planted in copies of the
# functions, on the CPU); the real-transform pin must fail for each.
def _irfft_no_scale(X, n):
    X = np.asarray(X, dtype=np.complex128)
    h = n // 2
    full = np.empty(X.shape[:-1] + (n,), dtype=np.complex128)
    full[..., : h + 1] = X
    full[..., 0] = X[..., 0].real
    full[..., h] = X[..., h].real
    full[..., h + 1:] = np.conj(X[..., 1:h][..., ::-1])
    return oracle.transform(full, oracle.ADJOINT).real


def _irfft_no_conj(X, n):
    X = np.asarray(X, dtype=np.complex128)
    h = n // 2
    full = np.empty(X.shape[:-1] + (n,), dtype=np.complex128)
    full[..., : h + 1] = X
    full[..., 0] = X[..., 0].real
    full[..., h] = X[..., h].real
    full[..., h + 1:] = X[..., 1:h][..., ::-1]
    return oracle.transform(full, oracle.INVERSE).real


def _irfft_unreversed(X, n):
    X = np.asarray(X, dtype=np.complex128)
    h = n // 2
    full = np.empty(X.shape[:-1] + (n,), dtype=np.complex128)
    full[..., : h + 1] = X
    full[..., 0] = X[..., 0].real
    full[..., h] = X[..., h].real
    full[..., h + 1:] = np.conj(X[..., 1:h])
    return oracle.transform(full, oracle.INVERSE).real


REAL_MUTATIONS = {
    "rfft_drops_nyquist": (lambda x: np.concatenate([oracle.rfft(x)[..., :-1], np.zeros(np.shape(x)[:-1] + (1,))],
                                                   axis=-1), None),
    "rfft_inverse_sign": (lambda x: oracle.transform(np.asarray(x, complex), oracle.ADJOINT)[..., : np.shape(x)[-1] // 2 + 1],
                          None),
    "irfft_no_scale": (None, _irfft_no_scale),
    "irfft_no_conj": (None, _irfft_no_conj),
    "irfft_unreversed": (None, _irfft_unreversed),
}


@pytest.mark.parametrize("name", sorted(REAL_MUTATIONS))
def test_real_pin_catches_mutation(lib, name):
    rf, irf = REAL_MUTATIONS[name]
    with pytest.raises(AssertionError):
        pins.check_real_transforms(lib, rf=rf, irf=irf)


def test_real_transforms_reject_bad_lengths():
    with pytest.raises(ValueError):
        oracle.rfft(np.ones(7))
    with pytest.raises(ValueError):
        oracle.irfft(np.ones(5, complex), 16)
