"""Pins for the FP64 oracle: checks that tie it to something other than itself.

Each check takes the oracle's compiled library (so the mutation test can run
the same battery against deliberately broken copies) and raises
AssertionError on failure.  Sources of truth, none of them the oracle:

* hand-worked values from Eq. 1 / Eq. 2 (tests/golden/dft_worked_examples.txt,
  and mixed_length_worked_examples.txt for N = 3, 5, 6);
* the N=2 butterfly and the N=4 DFT matrix written out by hand;
* closed forms: delta, shifted delta, single tone, constant, cosine;
* invariants: Parseval, linearity, inverse round trip, Hermitian symmetry of
  a real input's spectrum, the circular shift theorem, the adjoint identity;
* brute force (the O(N^2) sum) against the radix-2 recursion;
* an independent library routine: numpy's pocketfft in FP64.
"""
from __future__ import annotations

import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "dft_worked_examples.txt")

TIGHT = 1e-12     # FP64 oracle tolerance (relative L2) for O(N log N)-size sums


def _rng(seed=1):
    return np.random.Generator(np.random.PCG64(seed))


def _cvec(n, seed=1, batch=None):
    g = _rng(seed)
    shape = (n,) if batch is None else (batch, n)
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def _close(got, ref, tol, what):
    err = oracle.rel_l2(got, ref) if np.linalg.norm(ref) > 0 else float(np.max(np.abs(got - ref)))
    assert err <= tol, f"{what}: relative error {err:.3e} > {tol:.1e}"


def load_golden(path=GOLDEN):
    cases = []
    cur = None
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "example":
                cur = {"name": tok[1], "dir": tok[2], "n": int(tok[3])}
                cases.append(cur)
            elif tok[0] in ("in", "out"):
                vals = [complex(float(p.split(",")[0]), float(p.split(",")[1])) for p in tok[1:]]
                cur[tok[0]] = np.array(vals, dtype=np.complex128)
    for c in cases:
        assert len(c["in"]) == c["n"] and len(c["out"]) == c["n"], c["name"]
    return cases


def check_golden(lib):
    for c in load_golden():
        d = oracle.FORWARD if c["dir"] == "fwd" else oracle.INVERSE
        for fn in (oracle.dft, oracle.fft):
            got = fn(c["in"], d, lib=lib)
            assert np.max(np.abs(got - c["out"])) <= 1e-12 * max(1.0, np.max(np.abs(c["out"]))), \
                f"golden {c['name']} via {fn.__name__}: {got} vs {c['out']}"


GOLDEN_MIXED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                            "mixed_length_worked_examples.txt")


def check_golden_mixed(lib):
    """Hand-worked examples at N = 3, 5, 6 through the O(N^2) sum and the
    oracle's default route (which sends such lengths to that sum)."""
    cases = load_golden(GOLDEN_MIXED)
    assert {c["n"] for c in cases} == {3, 5, 6}
    for c in cases:
        d = oracle.FORWARD if c["dir"] == "fwd" else oracle.INVERSE
        for fn in (oracle.dft, oracle.transform):
            got = fn(c["in"], d, lib=lib)
            assert np.max(np.abs(got - c["out"])) <= 1e-12 * max(1.0, np.max(np.abs(c["out"]))), \
                f"golden {c['name']} via {fn.__name__}: {got} vs {c['out']}"


GOLDEN_REAL = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                           "real_and_filter_worked_examples.txt")


def load_golden_real():
    cases, cur = [], None
    with open(GOLDEN_REAL) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "example":
                cur = {"name": tok[1], "kind": tok[2], "n": int(tok[3])}
                cases.append(cur)
            elif tok[0] in ("in", "out", "filt"):
                cur[tok[0]] = np.array([complex(float(p.split(",")[0]), float(p.split(",")[1])) for p in tok[1:]],
                                       dtype=np.complex128)
    return cases


def check_golden_real_and_filter(lib):
    cases = load_golden_real()
    assert {c["kind"] for c in cases} == {"rfft", "irfft", "rc"}
    for c in cases:
        n = c["n"]
        if c["kind"] == "rfft":
            got = oracle.rfft(c["in"].real, lib=lib)
        elif c["kind"] == "irfft":
            got = oracle.irfft(c["in"], n, lib=lib)
        else:
            got = oracle.range_compress(c["in"], c["filt"], lib=lib)
        assert np.max(np.abs(got - c["out"])) <= 1e-12 * max(1.0, np.max(np.abs(c["out"]))), \
            f"golden {c['name']}: {got} vs {c['out']}"


def check_small_by_hand(lib):
    a, b = 0.3 - 1.1j, -2.0 + 0.5j
    for fn in (oracle.dft, oracle.fft):
        got = fn(np.array([a, b]), oracle.FORWARD, lib=lib)
        assert np.allclose(got, [a + b, a - b], rtol=0, atol=1e-15), f"N=2 butterfly via {fn.__name__}"
        got = fn(np.array([a, b]), oracle.INVERSE, lib=lib)
        assert np.allclose(got, [(a + b) / 2, (a - b) / 2], rtol=0, atol=1e-15), f"N=2 inverse via {fn.__name__}"
    # The 4-point DFT matrix, entries W_4^{nk} = (-i)^{nk}, written out by hand.
    F4 = np.array([[1, 1, 1, 1],
                   [1, -1j, -1, 1j],
                   [1, -1, 1, -1],
                   [1, 1j, -1, -1j]], dtype=np.complex128)
    x = _cvec(4, seed=7)
    ref = F4 @ x
    for fn in (oracle.dft, oracle.fft):
        _close(fn(x, oracle.FORWARD, lib=lib), ref, 1e-15, f"N=4 matrix via {fn.__name__}")
        _close(fn(x, oracle.ADJOINT, lib=lib), F4.conj().T @ x, 1e-15, f"N=4 adjoint via {fn.__name__}")
        _close(fn(x, oracle.INVERSE, lib=lib), F4.conj().T @ x / 4, 1e-15, f"N=4 inverse via {fn.__name__}")


def check_closed_forms(lib, sizes=(2, 8, 64, 256, 1024, 4096)):
    for n in sizes:
        fns = (oracle.dft, oracle.fft) if n <= 1024 else (oracle.fft,)
        k = np.arange(n)
        for fn in fns:
            tag = f"{fn.__name__} N={n}"
            delta = np.zeros(n, complex)
            delta[0] = 1
            _close(fn(delta, lib=lib), np.ones(n), 1e-14, f"delta {tag}")
            n0 = (3 * n) // 7 + 1 if n > 2 else 1
            sd = np.zeros(n, complex)
            sd[n0] = 1
            ramp = np.exp(-2j * np.pi * ((k * n0) % n) / n)
            _close(fn(sd, lib=lib), ramp, 1e-13, f"shifted delta {tag}")
            m = (5 * n) // 11 % n
            tone = np.exp(2j * np.pi * ((k * m) % n) / n)
            spike = np.zeros(n, complex)
            spike[m] = n
            _close(fn(tone, lib=lib), spike, 1e-13, f"tone {tag}")
            const = np.full(n, 2.5 - 0.5j)
            cs = np.zeros(n, complex)
            cs[0] = n * (2.5 - 0.5j)
            _close(fn(const, lib=lib), cs, 1e-14, f"constant {tag}")
            if n >= 4:
                mc = max(1, n // 4 - 1)
                cosine = np.cos(2 * np.pi * ((k * mc) % n) / n).astype(complex)
                two = np.zeros(n, complex)
                two[mc] = n / 2
                two[n - mc] = n / 2
                _close(fn(cosine, lib=lib), two, 1e-13, f"cosine {tag}")


def check_invariants(lib, sizes=(16, 512, 2048, 16384)):
    for n in sizes:
        fn = oracle.dft if n <= 512 else oracle.fft
        x = _cvec(n, seed=n)
        y = _cvec(n, seed=n + 1)
        X = fn(x, lib=lib)
        Y = fn(y, lib=lib)
        # Parseval: sum |X|^2 = N sum |x|^2
        px, pX = np.sum(np.abs(x) ** 2), np.sum(np.abs(X) ** 2)
        assert abs(pX - n * px) <= 1e-12 * n * px, f"Parseval N={n}"
        # linearity
        a, b = 0.7 - 0.2j, -1.3 + 2.0j
        _close(fn(a * x + b * y, lib=lib), a * X + b * Y, 1e-13, f"linearity N={n}")
        # round trip (Eq. 2 undoes Eq. 1)
        _close(fn(X, oracle.INVERSE, lib=lib), x, TIGHT, f"round trip N={n}")
        # Hermitian symmetry for a real input: X(N-k) = conj X(k)
        r = fn(x.real.astype(complex), lib=lib)
        _close(r[(-np.arange(n)) % n], np.conj(r), 1e-13, f"Hermitian N={n}")
        # circular shift theorem: x(n - s) -> W_N^{sk} X(k)
        s = n // 3 + 1
        ph = np.exp(-2j * np.pi * ((np.arange(n) * s) % n) / n)
        _close(fn(np.roll(x, s), lib=lib), ph * X, 1e-13, f"shift N={n}")
        # adjoint identity <F x, y> = <x, F^H y>
        lhs = np.vdot(y, X)
        rhs = np.vdot(fn(y, oracle.ADJOINT, lib=lib), x)
        assert abs(lhs - rhs) <= 1e-12 * n * np.linalg.norm(x) * np.linalg.norm(y), f"adjoint N={n}"


def check_dft_vs_fft(lib, max_log2=10):
    for lg in range(1, max_log2 + 1):
        n = 1 << lg
        x = _cvec(n, seed=100 + lg, batch=3)
        for d in (oracle.FORWARD, oracle.INVERSE, oracle.ADJOINT):
            _close(oracle.fft(x, d, lib=lib), oracle.dft(x, d, lib=lib), 1e-13, f"dft vs fft N={n} dir={d}")


def check_numpy(lib, sizes=(2, 4, 32, 1024, 4096, 65536)):
    for n in sizes:
        x = _cvec(n, seed=200 + n, batch=2)
        fns = (oracle.fft, oracle.dft) if n <= 1024 else (oracle.fft,)
        for fn in fns:
            _close(fn(x, oracle.FORWARD, lib=lib), np.fft.fft(x, axis=-1), 1e-13, f"numpy fwd {fn.__name__} N={n}")
            _close(fn(x, oracle.INVERSE, lib=lib), np.fft.ifft(x, axis=-1), 1e-13, f"numpy inv {fn.__name__} N={n}")
            _close(fn(x, oracle.ADJOINT, lib=lib), n * np.fft.ifft(x, axis=-1), 1e-13, f"numpy adj {fn.__name__} N={n}")


def check_fft2(lib, shapes=((4, 8), (32, 16), (64, 128))):
    for ny, nx in shapes:
        g = _rng(ny * 1000 + nx)
        x = g.standard_normal((ny, nx)) + 1j * g.standard_normal((ny, nx))
        _close(oracle.fft2(x, oracle.FORWARD, lib=lib), np.fft.fft2(x), 1e-13, f"fft2 {ny}x{nx}")
        _close(oracle.fft2(x, oracle.INVERSE, lib=lib), np.fft.ifft2(x), 1e-13, f"ifft2 {ny}x{nx}")
        # 2-D closed form: a delta at (y0, x0) -> W_ny^{y0 ky} W_nx^{x0 kx}
        d = np.zeros((ny, nx), complex)
        y0, x0 = ny // 3, nx // 5 + 1
        d[y0, x0] = 1
        ky, kx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        ref = np.exp(-2j * np.pi * (((ky * y0) % ny) / ny + ((kx * x0) % nx) / nx))
        _close(oracle.fft2(d, lib=lib), ref, 1e-13, f"fft2 delta {ny}x{nx}")


def check_range_compress(lib, rc=None):
    """Range compression (fast convolution) against definitions that do not
    go through a transform: the circular-convolution sum, the shift theorem,
    the identity filter and the matched-filter peak of a linear-FM pulse."""
    if rc is None:
        def rc(x, H):
            return oracle.range_compress(x, H, lib=lib)
    # (a) brute force: H = sum_t h[t] e^{-2 pi i k t / n} written out here;
    #     y[m] = sum_t x[t] h[(m - t) mod n]
    for n in (1, 2, 4, 8, 16, 32):
        x = _cvec(n, seed=500 + n, batch=3)
        h = _cvec(n, seed=600 + n)
        t = np.arange(n)
        H = np.array([np.sum(h * np.exp(-2j * np.pi * ((k * t) % n) / n)) for k in range(n)])
        ref = np.array([[np.sum(row * h[(m - t) % n]) for m in range(n)] for row in x])
        _close(rc(x, H), ref, 1e-12, f"range compression = circular convolution, n={n}")
    # (b) shift theorem: H[k] = W_n^{k d} delays every row by d samples
    for n, d in ((64, 5), (2048, 1000), (4096, 4095)):
        x = _cvec(n, seed=700 + n, batch=2)
        k = np.arange(n)
        H = np.exp(-2j * np.pi * ((k * d) % n) / n)
        _close(rc(x, H), np.roll(x, d, axis=-1), 1e-12, f"range compression shift n={n} d={d}")
    # (c) identity filter
    x = _cvec(512, seed=801, batch=2)
    _close(rc(x, np.ones(512)), x, 1e-13, "range compression identity")
    # (d) matched filter of a unit-amplitude LFM pulse of P samples: the echo
    #     delayed by d compresses to a peak of height P (the pulse energy) at d
    n, P, d = 1024, 200, 333
    t = np.arange(n)
    s = np.where(t < P, np.exp(1j * np.pi * (0.8 / P) * (t - P / 2) ** 2), 0)
    y = rc(np.roll(s, d)[None, :], np.conj(np.fft.fft(s)))[0]
    assert int(np.argmax(np.abs(y))) == d, "matched-filter peak position"
    assert abs(y[d] - P) <= 1e-9 * P, f"matched-filter peak height {y[d]} != {P}"
    assert np.max(np.abs(np.delete(y, d))) < 0.5 * P, "matched-filter sidelobes"


def check_real_transforms(lib, rf=None, irf=None):
    """rfft / irfft against definitions written out here: the real-input DFT
    sum, the cosine / sine closed forms, the round trip, and numpy's pocketfft
    real transforms (an independent library)."""
    if rf is None:
        def rf(x):
            return oracle.rfft(x, lib=lib)
    if irf is None:
        def irf(X, n):
            return oracle.irfft(X, n, lib=lib)
    # (a) brute force: X[k] = sum_n x[n] (cos(2 pi nk/N) - i sin(2 pi nk/N)), k <= N/2
    for n in (2, 4, 8, 16, 64):
        g = _rng(900 + n)
        x = g.standard_normal((2, n))
        t = np.arange(n)
        ref = np.array([[np.sum(row * (np.cos(2 * np.pi * ((k * t) % n) / n) - 1j * np.sin(2 * np.pi * ((k * t) % n) / n)))
                         for k in range(n // 2 + 1)] for row in x])
        _close(rf(x), ref, 1e-12, f"rfft brute force N={n}")
        _close(irf(ref, n), x, 1e-12, f"irfft of the brute-force spectrum N={n}")
    # (b) closed forms: cos(2 pi m n / N) -> N/2 at k = m; sin -> -i N/2 at k = m;
    #     the Nyquist cosine (-1)^n -> N at k = N/2
    for n, m in ((32, 3), (1024, 100), (4096, 2047)):
        t = np.arange(n)
        c = np.zeros(n // 2 + 1, complex)
        c[m] = n / 2
        _close(rf(np.cos(2 * np.pi * ((m * t) % n) / n)), c, 1e-12, f"rfft cos N={n} m={m}")
        sn = np.zeros(n // 2 + 1, complex)
        sn[m] = -1j * n / 2
        _close(rf(np.sin(2 * np.pi * ((m * t) % n) / n)), sn, 1e-12, f"rfft sin N={n} m={m}")
        ny = np.zeros(n // 2 + 1, complex)
        ny[n // 2] = n
        _close(rf((-1.0) ** t), ny, 1e-12, f"rfft Nyquist N={n}")
        _close(irf(c, n), np.cos(2 * np.pi * ((m * t) % n) / n), 1e-12, f"irfft cos N={n}")
    # (c) imaginary parts of X[0] and X[N/2] do not enter the inverse
    n = 64
    X = _cvec(n // 2 + 1, seed=901)
    Y = X.copy()
    Y[0] += 5j
    Y[-1] -= 3j
    _close(irf(Y, n), irf(X, n), 1e-13, "irfft ignores Im X[0], Im X[N/2]")
    # (d) round trip and numpy's real transforms
    for n in (2, 128, 2048, 65536):
        x = _rng(902 + n).standard_normal((2, n))
        _close(irf(rf(x), n), x, 1e-12, f"irfft(rfft(x)) N={n}")
        _close(rf(x), np.fft.rfft(x, axis=-1), 1e-13, f"rfft vs numpy N={n}")
        X = _cvec(n // 2 + 1, seed=903 + n, batch=2)
        _close(irf(X, n), np.fft.irfft(X, n, axis=-1), 1e-12, f"irfft vs numpy N={n}")


def check_mixed_lengths(lib):
    """Lengths that are not powers of two (products of 2, 3, 5, 7) through the
    default route: numpy's pocketfft, the delayed-delta closed form
    (delta[n - n0] -> W_N^{k n0}), Parseval and the round trip."""
    for n in (3, 5, 6, 7, 12, 15, 35, 100, 360, 1000):
        x = _cvec(n, seed=1000 + n, batch=2)
        _close(oracle.transform(x, oracle.FORWARD, lib=lib), np.fft.fft(x, axis=-1), 1e-12, f"mixed N={n} vs numpy")
        X = oracle.transform(x, oracle.FORWARD, lib=lib)
        _close(oracle.transform(X, oracle.INVERSE, lib=lib), x, 1e-12, f"mixed N={n} round trip")
        assert abs(np.sum(np.abs(X) ** 2) - n * np.sum(np.abs(x) ** 2)) <= 1e-10 * n * np.sum(np.abs(x) ** 2)
        n0 = n // 3 + 1
        d = np.zeros(n, complex)
        d[n0] = 1
        k = np.arange(n)
        _close(oracle.transform(d, lib=lib), np.exp(-2j * np.pi * ((k * n0) % n) / n), 1e-12, f"mixed N={n} delta")


def check_dft_bins(lib):
    """Single outputs of long transforms: numpy's pocketfft at powers of two
    and 7-smooth lengths up to 2^20, every direction, and two closed forms
    (delayed delta -> W_N^{k n0}; a pure tone -> N at its own bin, 0 at the
    others) at a length far beyond the O(N^2) route."""
    for n in (12, 64, 1000, 4096, 100000, 1 << 20):
        x = _cvec(n, seed=1200 + n % 997)
        ks = sorted({0, 1, n // 2, n - 1, (7 * n) // 13, (3 * n) // 5 + 1})
        fwd, inv = np.fft.fft(x), np.fft.ifft(x)
        _close(oracle.dft_bins(x, ks, oracle.FORWARD, lib=lib), fwd[ks], 1e-12, f"bins N={n} fwd")
        _close(oracle.dft_bins(x, ks, oracle.INVERSE, lib=lib), inv[ks], 1e-12, f"bins N={n} inv")
        _close(oracle.dft_bins(x, ks, oracle.ADJOINT, lib=lib), n * inv[ks], 1e-12, f"bins N={n} adj")
    n = 3 * 5 * 7 * 1024
    ks = np.array([0, 1, 2, 5, 1000, n // 3, n - 2, n - 1])
    n0 = 12345
    d = np.zeros(n, complex)
    d[n0] = 1
    _close(oracle.dft_bins(d, ks, lib=lib), np.exp(-2j * np.pi * ((ks * n0) % n) / n), 1e-12, "bins delta")
    m = 4321
    tone = np.exp(2j * np.pi * ((np.arange(n) * m) % n) / n)
    ks2 = np.array([m, m + 1, m - 1, 0, n - 1])
    want = np.array([n, 0, 0, 0, 0], dtype=complex)
    err = np.max(np.abs(oracle.dft_bins(tone, ks2, lib=lib) - want))
    assert err <= 1e-9 * n, f"bins tone: {err:.3e}"
    # batched rows keep their own outputs
    xb = _cvec(360, seed=1299, batch=3)
    _close(oracle.dft_bins(xb, [5, 17], lib=lib), np.fft.fft(xb, axis=-1)[:, [5, 17]], 1e-12, "bins batched")


def check_fft2_mixed(lib):
    """2-D transforms with sides that are not powers of two: numpy's fft2 /
    ifft2 and the separable delta closed form."""
    for ny, nx in ((12, 20), (3, 64), (35, 6)):
        g = _rng(ny * 100 + nx)
        x = g.standard_normal((2, ny, nx)) + 1j * g.standard_normal((2, ny, nx))
        _close(oracle.fft2(x, oracle.FORWARD, lib=lib), np.fft.fft2(x), 1e-13, f"fft2 {ny}x{nx}")
        _close(oracle.fft2(x, oracle.INVERSE, lib=lib), np.fft.ifft2(x), 1e-13, f"ifft2 {ny}x{nx}")
        d = np.zeros((ny, nx), complex)
        y0, x0 = ny // 3 + 1, nx // 5 + 1
        d[y0, x0] = 1
        ky, kx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        ref = np.exp(-2j * np.pi * (((ky * y0) % ny) / ny + ((kx * x0) % nx) / nx))
        _close(oracle.fft2(d, lib=lib), ref, 1e-13, f"fft2 delta {ny}x{nx}")


ALL_CHECKS = (check_golden, check_small_by_hand, check_closed_forms, check_invariants,
              check_dft_vs_fft, check_numpy, check_fft2, check_range_compress, check_real_transforms,
              check_mixed_lengths, check_golden_real_and_filter, check_golden_mixed, check_dft_bins,
              check_fft2_mixed)
