"""Seeded random plans across every plan kind, against the FP64 oracle.

Each case draws a plan kind, a length or image shape, a batch, a direction
(forward, inverse, and both adjoints) and in place or not from a fixed seed,
so the set is the same on every run: 1-D powers of two (one pass, two and
three passes), 7-smooth lengths (one pass and the strided two-pass plans) in
FP32 and FP64, 2-D images (tile plans, the transposed two-pass plan, strided
mixed-radix plans), and real-data transforms in FP32 and FP64.  Whole
transforms are compared where the oracle is cheap, sampled outputs
(oracle.dft_bins) for long 7-smooth lengths.  Bars as everywhere: FP32
5e-7 log2 N, FP64 5e-15 log2 N + 2e-16 sqrt(N)."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1707_07263_gb300 import _lib as L

pytestmark = pytest.mark.gpu

SEED = 20260412
ODIR = {0: oracle.FORWARD, 1: oracle.INVERSE, 2: oracle.ADJOINT}


def smooth7(limit: int) -> list:
    out = []
    for a in range(0, 30):
        for b in range(0, 20):
            for c in range(0, 14):
                for d in range(0, 12):
                    v = 2 ** a * 3 ** b * 5 ** c * 7 ** d
                    if v > limit:
                        break
                    out.append(v)
    return sorted(set(v for v in out if v >= 2))


def tol(n: int, fp64: bool) -> float:
    return (5e-15 * max(1.0, np.log2(n)) + 2e-16 * np.sqrt(n)) if fp64 else 5e-7 * max(1.0, np.log2(n))


def oracle_dir(x, d, transform):
    n = x.shape[-1]
    if d == 3:
        return transform(x, oracle.FORWARD) / n
    return transform(x, ODIR[d])


def cases():
    g = np.random.Generator(np.random.PCG64(SEED))
    s32 = [v for v in smooth7(60000) if v & (v - 1)]
    s64 = smooth7(40000)
    out = []
    for i in range(96):
        kind = ["pow2", "pow2", "mixed32", "mixed64", "2d", "2d", "real32", "real64"][i % 8]
        d = int(g.integers(0, 4))
        inplace = bool(g.integers(0, 2))
        if kind == "pow2":
            lg = int(g.integers(1, 23))
            batch = int(g.integers(1, max(2, (1 << 22) >> lg) + 1))
            batch = min(batch, 7)
            out.append((kind, (1 << lg,), batch, d, inplace))
        elif kind == "mixed32":
            out.append((kind, (int(g.choice(s32)),), int(g.integers(1, 4)), d, inplace))
        elif kind == "mixed64":
            out.append((kind, (int(g.choice(s64)),), int(g.integers(1, 4)), d, inplace))
        elif kind == "2d":
            if g.integers(0, 2):
                ly, lx = int(g.integers(1, 13)), int(g.integers(1, 13))
                while ly + lx > 22:
                    ly -= 1
                shape = (1 << max(ly, 1), 1 << max(lx, 1))
            else:
                sm = smooth7(400)
                shape = (int(g.choice(sm)), int(g.choice(sm)))
            out.append((kind, shape, int(g.integers(1, 3)), d, inplace))
        elif kind == "real32":
            out.append((kind, (1 << int(g.integers(2, 21)),), int(g.integers(1, 4)), d, False))
        else:
            # half lengths: one-pass 7-smooth ones, and powers of two beyond one FP64 pass
            halves = smooth7(3000) + [8192, 16384, 32768]
            out.append((kind, (2 * int(g.choice(halves)),), int(g.integers(1, 4)), d, False))
    return [(i,) + c for i, c in enumerate(out)]


CASES = cases()


def _run(h, x: torch.Tensor, out: torch.Tensor, d: int):
    lib = L.load()
    assert lib.fft_plan_set_workspace(h, None) == 0
    rc = lib.fft_exec_dir(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), d,
                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert rc == 0, L.ERRORS.get(rc, rc)
    lib.fft_destroy(h)
    return out.cpu().numpy()


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{c[1]}-{'x'.join(map(str, c[2]))}-b{c[3]}-d{c[4]}"
                         + ("-ip" if c[5] else ""))
def test_random_plan(case):
    idx, kind, shape, batch, d, inplace = case
    lib = L.load()
    g = np.random.Generator(np.random.PCG64(SEED + 1000 + idx))
    if kind in ("pow2", "mixed32", "mixed64"):
        n = shape[0]
        fp64 = kind == "mixed64"
        x = g.normal(0, 0.7, (batch, n)) + 1j * g.normal(0, 0.7, (batch, n))
        x = x if fp64 else x.astype(np.complex64)
        h = ctypes.c_void_p(lib.fft_plan_create(n, batch, d, L.FFT_PREC_FP64 if fp64 else 0))
        assert h.value, L.ERRORS.get(lib.fft_last_error())
        xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        got = _run(h, xt, xt if inplace else torch.empty_like(xt), d)
        x64 = x.astype(np.complex128)
        pow2 = (n & (n - 1)) == 0
        if pow2 or n <= 3000:
            ref = oracle_dir(x64, d, oracle.fft if pow2 else oracle.dft)
            err = oracle.rel_l2_rows(got, ref).max()
        else:
            ks = np.unique(np.concatenate([[0, 1, n - 1], g.integers(0, n, 6)]))
            ref = oracle_dir(x64, d, lambda v, dd: oracle.dft_bins(v, ks, dd))
            err = oracle.rel_l2_rows(got[:, ks], ref).max()
        assert err <= tol(n, fp64), f"{case}: {err:.2e}"
    elif kind == "2d":
        ny, nx = shape
        x = (g.normal(0, 0.7, (batch, ny, nx)) + 1j * g.normal(0, 0.7, (batch, ny, nx))).astype(np.complex64)
        h = ctypes.c_void_p(lib.fft_plan_create_2d(ny, nx, batch, d, 0))
        assert h.value, L.ERRORS.get(lib.fft_last_error())
        xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        got = _run(h, xt, xt if inplace else torch.empty_like(xt), d)
        x64 = x.astype(np.complex128)
        ref = oracle_dir(x64, d, lambda v, dd: oracle.fft2(v, dd)) if d != 3 else oracle.fft2(x64) / (ny * nx)
        err = max(oracle.rel_l2(got[b], ref[b]) for b in range(batch))
        assert err <= tol(ny * nx, False), f"{case}: {err:.2e}"
    else:
        n = shape[0]
        fp64 = kind == "real64"
        prec = L.FFT_PREC_FP64 if fp64 else 0
        h = ctypes.c_void_p(lib.fft_plan_create_r2c(n, batch, prec))
        assert h.value, L.ERRORS.get(lib.fft_last_error())
        to_complex = d in (0, 3)
        if to_complex:
            x = g.uniform(-1, 1, (batch, n))
            x = x if fp64 else x.astype(np.float32)
            xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
            out = torch.empty((batch, n // 2 + 1), dtype=torch.complex128 if fp64 else torch.complex64, device="cuda")
            got = _run(h, xt, out, d)
            full = oracle.rfft(x.astype(np.float64))
            ref = full if d == 0 else full * np.concatenate([[1.0 / n], np.full(n // 2 - 1, 2.0 / n), [1.0 / n]])
        else:
            X = g.normal(0, 1, (batch, n // 2 + 1)) + 1j * g.normal(0, 1, (batch, n // 2 + 1))
            X = X if fp64 else X.astype(np.complex64)
            xt = torch.from_numpy(np.ascontiguousarray(X)).cuda()
            out = torch.empty((batch, n), dtype=torch.float64 if fp64 else torch.float32, device="cuda")
            got = _run(h, xt, out, d)
            X64 = X.astype(np.complex128)
            if d == 1:
                ref = oracle.irfft(X64, n)
            else:
                # adjoint of the real-to-complex transform: Re sum_{k <= n/2} X_k W^{-mk}
                pad = np.zeros((batch, n), dtype=np.complex128)
                pad[:, : n // 2 + 1] = X64
                pad[:, 0] = X64[:, 0].real
                pad[:, n // 2] = X64[:, n // 2].real
                ref = oracle.transform(pad, oracle.ADJOINT).real
        err = oracle.rel_l2_rows(got, ref).max()
        assert err <= tol(n, fp64), f"{case}: {err:.2e}"
