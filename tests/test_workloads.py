"""The seeded input generators (no transform arithmetic): deterministic per
seed, the stated shapes, dtypes and distributions, and the properties the
SAR generators promise (unit-modulus pulse, band-limited unit-gain filter)."""
from __future__ import annotations

import numpy as np

from paper_1707_07263_gb300 import workloads as w


def test_deterministic_and_seed_dependent():
    a, b, c = w.cgauss(64, 3, seed=5), w.cgauss(64, 3, seed=5), w.cgauss(64, 3, seed=6)
    assert a.dtype == np.complex64 and a.shape == (3, 64)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.array_equal(w.uneven_lengths(50, seed=1), w.uneven_lengths(50, seed=1))


def test_distributions():
    z = w.cgauss(1 << 16, 4, seed=11).astype(np.complex128)
    assert abs(np.mean(np.abs(z) ** 2) - 1.0) < 0.01            # CN(0,1): E|z|^2 = 1
    assert abs(np.var(z.real) - 0.5) < 0.01 and abs(np.var(z.imag) - 0.5) < 0.01
    u = w.uniform(1 << 14, 2, seed=12)
    assert u.real.min() >= -1 and u.real.max() <= 1 and u.imag.min() >= -1 and u.imag.max() <= 1
    lens = w.uneven_lengths(4096, seed=13)
    e = np.log2(lens).astype(int)
    assert e.min() == 8 and e.max() == 16 and np.all(lens == (1 << e))
    assert np.all(np.bincount(e)[8:] > 300)                      # every exponent drawn
    wt = w.real_weights(1000, seed=14)
    assert wt.dtype == np.float32 and wt.min() >= 0 and wt.max() <= 1


def test_sar_image_scatterers():
    img = w.sar_image(64, 64, n_scatterers=10, amplitude=100.0, seed=15)
    assert img.shape == (64, 64) and img.dtype == np.complex64
    assert np.sum(np.abs(img) > 50) == 10                         # distinct pixels, amplitude 100


def test_lfm_pulse_and_filter():
    n, P = 4096, 1000
    s = w.lfm_pulse(n, P)
    assert np.allclose(np.abs(s[:P]), 1.0, atol=1e-6) and np.all(s[P:] == 0)
    H = w.range_filter(n, P, bw=0.8)
    k = np.arange(n)
    f = np.where(k < n / 2, k / n, k / n - 1.0)
    inband = np.abs(f) <= 0.4
    assert np.allclose(np.abs(H[inband]), 1.0, atol=1e-6) and np.all(H[~inband] == 0)
    x = w.range_lines(n, 2, P, n_targets=3, seed=16)
    assert x.shape == (2, n) and x.dtype == np.complex64
