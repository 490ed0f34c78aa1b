"""Seeded synthetic inputs shaped like the paper's remote-sensing (SAR) FFT
workloads (Sec. 3 names SAR imaging with transform lengths from a few
thousand to tens of thousands of points).

This module only draws random numbers; it holds none of the transform's
arithmetic.  Both the CUDA path's tests/benchmark and the FP64 oracle take
their inputs from here, so the two sides always see the same complex64
values.  Every value is drawn in FP64 from numpy's PCG64 generator and cast
once to complex64.

Distributions:
* ``uniform``   -- real and imaginary parts i.i.d. U[-1, 1].
* ``cgauss``    -- circular complex Gaussian CN(0, 1): real and imaginary
                   parts i.i.d. N(0, 1/2), so E|z|^2 = 1.
* ``sar_image`` -- unit CN(0,1) speckle plus point scatterers of amplitude A
                   and uniform random phase at distinct random pixels.
* ``uneven_lengths`` -- lengths 2^e with e uniform over the integers lo..hi.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20170723


def seed_for(config_index: int, salt: int = 0) -> int:
    """Fixed seed per workload: SEED_BASE + config index (+ an optional salt
    for a second, independent draw such as loss weights)."""
    return SEED_BASE + int(config_index) + 1000 * int(salt)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform(n: int, batch: int = 1, seed: int = SEED_BASE) -> np.ndarray:
    """complex64 array (batch, n) with re, im ~ U[-1, 1]."""
    g = _rng(seed)
    re = g.uniform(-1.0, 1.0, size=(batch, n))
    im = g.uniform(-1.0, 1.0, size=(batch, n))
    return (re + 1j * im).astype(np.complex64)


def cgauss(n: int, batch: int = 1, seed: int = SEED_BASE) -> np.ndarray:
    """complex64 array (batch, n) with entries CN(0, 1)."""
    g = _rng(seed)
    s = np.sqrt(0.5)
    re = g.normal(0.0, s, size=(batch, n))
    im = g.normal(0.0, s, size=(batch, n))
    return (re + 1j * im).astype(np.complex64)


def sar_image(ny: int, nx: int, n_scatterers: int = 64, amplitude: float = 100.0,
              seed: int = SEED_BASE) -> np.ndarray:
    """complex64 (ny, nx) image: CN(0,1) speckle plus ``n_scatterers`` point
    targets of the given amplitude and phase ~ U[0, 2*pi) at distinct pixels
    (sampled without replacement)."""
    g = _rng(seed)
    s = np.sqrt(0.5)
    img = g.normal(0.0, s, size=(ny, nx)) + 1j * g.normal(0.0, s, size=(ny, nx))
    k = min(int(n_scatterers), ny * nx)
    pix = g.choice(ny * nx, size=k, replace=False)
    phase = g.uniform(0.0, 2.0 * np.pi, size=k)
    flat = img.reshape(-1)
    flat[pix] += amplitude * np.exp(1j * phase)
    return img.astype(np.complex64)


def uneven_lengths(count: int, lo_exp: int = 8, hi_exp: int = 16, seed: int = SEED_BASE) -> np.ndarray:
    """int64 array of ``count`` lengths 2^e, e uniform over lo_exp..hi_exp."""
    g = _rng(seed)
    e = g.integers(lo_exp, hi_exp + 1, size=count)
    return (np.int64(1) << e.astype(np.int64)).astype(np.int64)


def packed_cgauss(lengths, seed: int = SEED_BASE) -> np.ndarray:
    """One flat complex64 array holding CN(0,1) inputs for transforms of the
    given lengths back to back (offsets are the prefix sums of the lengths)."""
    total = int(np.sum(np.asarray(lengths, dtype=np.int64)))
    return cgauss(total, 1, seed).reshape(-1)


def real_weights(n: int, seed: int = SEED_BASE) -> np.ndarray:
    """float32 weights ~ U[0, 1] (the spectral-loss weights w)."""
    g = _rng(seed)
    return g.uniform(0.0, 1.0, size=n).astype(np.float32)
