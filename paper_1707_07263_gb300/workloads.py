"""Seeded synthetic inputs shaped like the paper's remote-sensing (SAR) FFT
workloads (Sec. 3: SAR imaging, transforms of roughly 10^3 to a few 10^4
points).

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
* ``lfm_pulse`` / ``range_lines`` / ``range_filter`` -- SAR range lines: a
  linear-FM (chirp) pulse, echoes of it from point targets at random delays
  in CN(0,1) receiver noise, and the frequency-domain matched filter written
  in closed form by the principle of stationary phase (no transform is
  computed here).
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


def cgauss128(n: int, batch: int = 1, seed: int = SEED_BASE) -> np.ndarray:
    """complex128 array (batch, n) with entries CN(0, 1), drawn and kept in FP64
    (inputs of FP64 transforms)."""
    g = _rng(seed)
    s = np.sqrt(0.5)
    return g.normal(0.0, s, size=(batch, n)) + 1j * g.normal(0.0, s, size=(batch, n))


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


def lfm_pulse(n: int, n_pulse: int, bw: float = 0.8) -> np.ndarray:
    """complex64 (n,): a unit-amplitude linear-FM pulse of n_pulse samples,
    s[t] = exp(i pi K (t - n_pulse/2)^2) for t < n_pulse and 0 after, swept
    over bw cycles per sample (chirp rate K = bw / n_pulse)."""
    t = np.arange(n, dtype=np.float64)
    K = bw / n_pulse
    s = np.exp(1j * np.pi * K * (t - n_pulse / 2.0) ** 2)
    s[n_pulse:] = 0.0
    return s.astype(np.complex64)


def range_lines(n: int, batch: int, n_pulse: int, n_targets: int = 8, bw: float = 0.8,
                noise: float = 1.0, seed: int = SEED_BASE) -> np.ndarray:
    """complex64 (batch, n) raw range lines: per line, n_targets echoes of
    lfm_pulse (amplitudes U[1, 10], phases U[0, 2 pi), circular delays
    uniform over 0..n-1) plus CN(0, noise^2) receiver noise."""
    g = _rng(seed)
    s = lfm_pulse(n, n_pulse, bw).astype(np.complex128)
    sc = np.sqrt(0.5) * noise
    out = g.normal(0.0, sc, size=(batch, n)) + 1j * g.normal(0.0, sc, size=(batch, n))
    amp = g.uniform(1.0, 10.0, size=(batch, n_targets))
    ph = g.uniform(0.0, 2.0 * np.pi, size=(batch, n_targets))
    dl = g.integers(0, n, size=(batch, n_targets))
    for b in range(batch):
        for t in range(n_targets):
            out[b] += amp[b, t] * np.exp(1j * ph[b, t]) * np.roll(s, dl[b, t])
    return out.astype(np.complex64)


def range_filter(n: int, n_pulse: int, bw: float = 0.8) -> np.ndarray:
    """complex64 (n,): the matched filter of lfm_pulse in the frequency domain
    by stationary phase, H(f) = exp(i pi f^2 / K) exp(2 pi i f n_pulse / 2)
    for |f| <= bw/2 (zero outside), f = k/n for k < n/2 and k/n - 1 above
    (cycles per sample), K = bw / n_pulse."""
    k = np.arange(n, dtype=np.float64)
    f = np.where(k < n / 2, k / n, k / n - 1.0)
    K = bw / n_pulse
    H = np.exp(1j * np.pi * f * f / K) * np.exp(2j * np.pi * f * (n_pulse / 2.0))
    H[np.abs(f) > bw / 2.0] = 0.0
    return H.astype(np.complex64)
