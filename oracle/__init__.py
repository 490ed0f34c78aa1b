"""FP64 CPU oracle for the complex power-of-two DFT (paper Sec. 2.1, Eqs. 1-5).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline / reference arm may import this package.  The
product path (the CUDA library and ``paper_1707_07263_gb300``) never imports
it, and the two share no code: this file and ``fft_oracle.c`` hold their own
arithmetic, written from the paper's definitions.

Functions (all FP64, numpy ``complex128`` in and out):

* ``dft(x, dir)``       -- Eq. 1 (dir 0) / Eq. 2 (dir 1) / adjoint (dir 2),
                           summed term by term, O(N^2), over the last axis.
* ``fft(x, dir)``       -- recursive radix-2 decimation in time (the butterfly
                           of Sec. 2.1), over the last axis.
* ``dft_bins(x, ks, dir)`` -- the same sum as ``dft`` at the outputs ks only
                           (O(N) each), for transforms too long for ``dft``.
* ``fft2(x, dir)``      -- 2-D transform of the last two axes, rows then
                           columns (Sec. 2.3.2 treats the data as 2-D/3-D and
                           transforms each dimension in turn); sides that are
                           not powers of two go through ``transform``.
* ``range_compress(x, H)`` -- SAR range compression by fast convolution, the
  FFT-based SAR processing that Sec. 3 and Sec. 4 name as the method's
  application: every row becomes Eq. 2 applied to H * (Eq. 1 applied to the
  row), i.e. the circular convolution of the row with the inverse transform
  of H (for a matched filter H, the correlation with the transmitted pulse).
* ``rfft(x)`` / ``irfft(X, n)`` -- transforms of real rows: Eq. 1 of a real
  sequence keeps its n/2 + 1 non-redundant outputs (X[n-k] = conj(X[k]));
  the inverse extends X[0..n/2] to the full Hermitian spectrum (the
  imaginary parts of X[0] and X[n/2] do not enter) and returns the real part
  of Eq. 2.
* ``spectral_loss(x, w)`` and ``spectral_loss_grad(x, w)`` -- the loss
  L = sum_k |w_k X_k|^2 with X = Eq. 1 applied to x, and its gradient in
  PyTorch's convention (dL/dRe + i dL/dIm) = 2 F^H (w^2 * F x), where F^H is
  the adjoint (conjugate-direction transform without the 1/N, Eq. 4).

Parity of every function here is pinned by ``tests/test_oracle.py`` against
closed forms, invariants, hand-worked small cases, brute force and an
independent library routine (numpy's pocketfft).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

FORWARD, INVERSE, ADJOINT = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fft_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``fft_oracle.c`` into ``liboracle.so`` with gcc (plain -O2, no
    fast-math, so FP64 rounding follows IEEE order)."""
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-fno-fast-math",
             "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def load_library(path: str | None = None):
    """Load the compiled oracle (building it first if needed).  ``path`` lets a
    test load a deliberately mutated copy."""
    global _lib
    if path is None and _lib is not None:
        return _lib
    lib = ctypes.CDLL(path or build())
    i64, vp, ci = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
    for name in ("oracle_dft", "oracle_fft"):
        fn = getattr(lib, name)
        fn.argtypes = [i64, vp, vp, ci]
        fn.restype = ci
    for name in ("oracle_dft_batch", "oracle_fft_batch"):
        fn = getattr(lib, name)
        fn.argtypes = [i64, i64, vp, vp, ci]
        fn.restype = ci
    lib.oracle_fft2.argtypes = [i64, i64, vp, vp, ci]
    lib.oracle_fft2.restype = ci
    lib.oracle_dft_bins.argtypes = [i64, vp, i64, vp, vp, ci]
    lib.oracle_dft_bins.restype = ci
    if path is None:
        _lib = lib
    return lib


def _prep(x) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x), dtype=np.complex128)
    return a


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _run_batch(name: str, x, dir: int, lib=None) -> np.ndarray:
    lib = lib or load_library()
    a = _prep(x)
    n = a.shape[-1]
    out = np.empty_like(a)
    if a.size == 0:
        return out
    batch = a.size // n
    rc = getattr(lib, name)(n, batch, _ptr(a), _ptr(out), dir)
    if rc != 0:
        raise ValueError(f"{name}: rejected n={n}, dir={dir} (rc={rc})")
    return out


def dft(x, dir: int = FORWARD, lib=None) -> np.ndarray:
    """Eq. 1 / Eq. 2 summed directly over the last axis (any N >= 1)."""
    return _run_batch("oracle_dft_batch", x, dir, lib)


def fft(x, dir: int = FORWARD, lib=None) -> np.ndarray:
    """Recursive radix-2 DIT over the last axis (N a power of two)."""
    return _run_batch("oracle_fft_batch", x, dir, lib)


def dft_bins(x, ks, dir: int = FORWARD, lib=None) -> np.ndarray:
    """Eq. 1 / Eq. 2 / the adjoint of every row of x (last axis) at the outputs
    ks only: result[..., i] = X[..., ks[i]], each a term-by-term sum."""
    lib = lib or load_library()
    a = _prep(x)
    n = a.shape[-1]
    k = np.ascontiguousarray(np.asarray(ks, dtype=np.int64).reshape(-1))
    rows = a.reshape(-1, n)
    out = np.empty((rows.shape[0], k.size), dtype=np.complex128)
    for i in range(rows.shape[0]):
        dst = np.empty(k.size, dtype=np.complex128)
        rc = lib.oracle_dft_bins(n, _ptr(rows[i]), k.size, k.ctypes.data, _ptr(dst), dir)
        if rc != 0:
            raise ValueError(f"oracle_dft_bins: rejected n={n}, dir={dir} (rc={rc})")
        out[i] = dst
    return out.reshape(a.shape[:-1] + (k.size,))


def fft2(x, dir: int = FORWARD, lib=None) -> np.ndarray:
    """2-D transform over the last two axes: rows, then columns.  Power-of-two
    sides run in the C routine; other sides take ``transform`` over the rows
    and then over the columns (the same definition, any 7-smooth side)."""
    lib = lib or load_library()
    a = _prep(x)
    ny, nx = a.shape[-2], a.shape[-1]
    if (ny & (ny - 1)) or (nx & (nx - 1)):
        rows = transform(a, dir, lib)
        cols = transform(np.swapaxes(rows, -1, -2), dir, lib)
        return np.ascontiguousarray(np.swapaxes(cols, -1, -2))
    out = np.empty_like(a)
    flat_in = a.reshape(-1, ny, nx)
    flat_out = out.reshape(-1, ny, nx)
    for i in range(flat_in.shape[0]):
        src = np.ascontiguousarray(flat_in[i])
        dst = np.empty_like(src)
        rc = lib.oracle_fft2(ny, nx, _ptr(src), _ptr(dst), dir)
        if rc != 0:
            raise ValueError(f"oracle_fft2: rejected {ny}x{nx} (rc={rc})")
        flat_out[i] = dst
    return out


def transform(x, dir: int = FORWARD, lib=None) -> np.ndarray:
    """The oracle's default route: the O(N^2) sum for N <= 1024 and for every
    N that is not a power of two (Eq. 1 holds for any N), the radix-2
    recursion for powers of two above 1024."""
    n = np.asarray(x).shape[-1]
    return dft(x, dir, lib) if (n <= 1024 or n & (n - 1)) else fft(x, dir, lib)


def range_compress(x, H, lib=None) -> np.ndarray:
    """Rows of x (last axis, length n) each become IDFT(H * DFT(row)): Eq. 1,
    the pointwise product with the n-point frequency-domain filter H (shared
    by every row, natural frequency order), then Eq. 2 with its 1/n."""
    x = np.asarray(x, dtype=np.complex128)
    H = np.asarray(H, dtype=np.complex128)
    if H.shape != x.shape[-1:]:
        raise ValueError(f"range_compress: filter of shape {H.shape} for rows of length {x.shape[-1]}")
    return transform(transform(x, FORWARD, lib) * H, INVERSE, lib)


def rfft(x, lib=None) -> np.ndarray:
    """X[k] = sum_n x[n] W_n^{nk} (Eq. 1) of real rows, k = 0..n/2."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[-1]
    if n < 2 or n % 2:
        raise ValueError(f"rfft: even length needed, got {n}")
    return transform(x.astype(np.complex128), FORWARD, lib)[..., : n // 2 + 1]


def irfft(X, n: int, lib=None) -> np.ndarray:
    """Real rows x of length n whose Eq. 1 has X[0..n/2] as its first half:
    Eq. 2 of the Hermitian extension F[k] = X[k] (k <= n/2), conj(X[n-k])
    (k > n/2), with Im X[0] and Im X[n/2] set to zero, real part kept."""
    X = np.asarray(X, dtype=np.complex128)
    if n < 2 or n % 2 or X.shape[-1] != n // 2 + 1:
        raise ValueError(f"irfft: {X.shape[-1]} values for length {n}")
    h = n // 2
    full = np.empty(X.shape[:-1] + (n,), dtype=np.complex128)
    full[..., : h + 1] = X
    full[..., 0] = X[..., 0].real
    full[..., h] = X[..., h].real
    full[..., h + 1:] = np.conj(X[..., 1:h][..., ::-1])
    return transform(full, INVERSE, lib).real


def spectral_loss(x, w) -> float:
    """L = sum_k |w_k * X_k|^2 with X the forward transform (Eq. 1) of x."""
    X = fft(x, FORWARD)
    return float(np.sum((np.asarray(w, dtype=np.float64) ** 2) * (X.real ** 2 + X.imag ** 2)))


def spectral_loss_grad(x, w) -> np.ndarray:
    """dL/dRe(x) + i dL/dIm(x) = 2 F^H (w^2 * F x); F^H is the adjoint
    transform (conjugate direction, no 1/N; Eq. 4)."""
    X = fft(x, FORWARD)
    w2 = np.asarray(w, dtype=np.float64) ** 2
    return 2.0 * fft(w2 * X, ADJOINT)


def rel_l2(got, ref) -> float:
    """||got - ref||_2 / ||ref||_2 over all elements, in FP64."""
    g = np.asarray(got, dtype=np.complex128)
    r = np.asarray(ref, dtype=np.complex128)
    den = np.linalg.norm(r.reshape(-1))
    num = np.linalg.norm((g - r).reshape(-1))
    return float(num / den) if den > 0 else float(num)


def rel_l2_rows(got, ref) -> np.ndarray:
    """Relative L2 error of each transform (last axis) separately."""
    g = np.asarray(got, dtype=np.complex128)
    r = np.asarray(ref, dtype=np.complex128)
    den = np.sqrt(np.sum(np.abs(r) ** 2, axis=-1))
    num = np.sqrt(np.sum(np.abs(g - r) ** 2, axis=-1))
    return num / np.where(den > 0, den, 1.0)
