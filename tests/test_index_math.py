"""Host-side checks of two index identities the kernels rely on (no GPU).

1. The padded shared-memory index pidx(n) = n + floor(n/16) of the on-chip
   Stockham passes splits as pidx(base + d) = pidx(base) + pidx(d) for every
   butterfly's element offsets (reads d = r L/R from base j, writes d = q Ns
   from base (j div Ns) Ns R + (j mod Ns)), in the forward radix schedule
   (remainder pass first) and the reversed one (remainder last), with radix-16
   passes and with the radix-8 and radix-4 passes of the autotuner's
   smaller-radix single-pass variants.  The kernels
   address each butterfly's elements as one base register plus constants on
   the strength of it.
2. The mixed-radix kernel divides by run-time d with q = floor(n m / 2^32),
   m = ceil(2^32 / d); that equals floor(n / d) for every divisor d and index
   n the kernel can meet (d, n < 2^14 + 1024)."""
from __future__ import annotations

import os

import numpy as np
import pytest


def pidx(n):
    return n + (n >> 4)


def schedule(lg: int, rev: bool, lgm: int = 4):
    """log2 of the radices, pass by pass: full radix-2^lgm passes plus one
    smaller remainder pass (first, or last when rev)."""
    rest = [lgm] * (lg // lgm)
    if lg % lgm:
        rest = rest + [lg % lgm] if rev else [lg % lgm] + rest
    return rest


@pytest.mark.parametrize("rev,lgm", [(False, 4), (True, 4), (False, 3), (False, 2)])
@pytest.mark.parametrize("lg", range(1, 15))
def test_padded_index_splits(lg, rev, lgm):
    L = 1 << lg
    lgns = 0
    for lgr in schedule(lg, rev, lgm):
        R, Ns = 1 << lgr, 1 << lgns
        j = np.arange(L // R)
        r = np.arange(R)[:, None]
        d_read = r * (L // R)
        assert np.array_equal(pidx(j + d_read), pidx(j) + pidx(d_read)), ("read", lg, rev, lgm, R, Ns)
        base = (j // Ns) * Ns * R + (j % Ns)
        d_write = r * Ns
        assert np.array_equal(pidx(base + d_write), pidx(base) + pidx(d_write)), ("write", lg, rev, lgm, R, Ns)
        lgns += lgr
    assert lgns == lg


def test_reciprocal_division_is_exact():
    n = np.arange(0, (1 << 14) + 1024, dtype=np.uint64)
    for d in range(2, (1 << 14) + 1):
        m = np.uint64(((1 << 32) + d - 1) // d)
        q = (n * m) >> np.uint64(32)
        assert np.array_equal(q, n // np.uint64(d)), d


def test_compile_time_twiddle_constants(tmp_path):
    """The compile-time cos / sin of 2 pi m / R that the compiled mixed-radix
    schedules use as inner twiddles (csrc/ct_trig.h, a Taylor series after
    octant reduction) agree with a 30-digit evaluation (mpmath) to 4e-16
    (two units in the last place at magnitude 1) for every m of R = 1..64,
    including negative m and m >= R."""
    import subprocess
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "t.cpp"
    src.write_text('#include <cstdio>\n#include "ct_trig.h"\n'
                   'int main() { for (int R = 1; R <= 64; ++R) for (int m = -R; m < 2 * R; ++m) '
                   'printf("%d %d %.17g %.17g\\n", m, R, gbfft::ct_cos(m, R), gbfft::ct_sin(m, R)); return 0; }\n')
    exe = tmp_path / "t"
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-I", os.path.join(root, "paper_1707_07263_gb300", "csrc"),
                           str(src), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    worst = 0.0
    count = 0
    for line in out:
        if not line:
            continue
        m, r, c, s = line.split()
        m, r = int(m), int(r)
        ang = 2 * mpmath.pi * mpmath.mpf(m % r) / r
        worst = max(worst, abs(float(c) - float(mpmath.cos(ang))), abs(float(s) - float(mpmath.sin(ang))))
        count += 1
    assert count == sum(3 * r for r in range(1, 65))
    assert worst <= 4e-16, worst
