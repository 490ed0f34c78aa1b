"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded complex64 inputs.

Bar: relative L2 error of every transform <= 5e-7 * log2(N) for the FP32
path (the stated FP32 tolerance; an FP32 radix-16 FFT has an RMS error of a
few 1e-8 * sqrt(log2 N), so this leaves a wide margin while still catching a
wrong twiddle, which costs O(1)).
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1707_07263_gb300 import _lib, workloads

pytestmark = pytest.mark.gpu

DIRS = {"fwd": 0, "inv": 1, "adj": 2, "adj_inv": 3}


def tol32(n: int) -> float:
    return 5e-7 * max(1.0, np.log2(n))


def oracle_dir(x: np.ndarray, d: int) -> np.ndarray:
    """Oracle for every direction code of the ABI."""
    x = x.astype(np.complex128)
    n = x.shape[-1]
    if d == 0:
        return oracle.transform(x, oracle.FORWARD)
    if d == 1:
        return oracle.transform(x, oracle.INVERSE)
    if d == 2:
        return oracle.transform(x, oracle.ADJOINT)
    return oracle.transform(x, oracle.FORWARD) / n   # adjoint of the inverse


@pytest.fixture(scope="module")
def lib():
    return _lib.load()


class CPlan:
    """Minimal plan wrapper straight over the C ABI (no autograd layer)."""

    def __init__(self, lib, h):
        assert h, _lib.ERRORS.get(lib.fft_last_error())
        self.lib, self.h = lib, ctypes.c_void_p(h)
        ws = lib.fft_plan_workspace_bytes(self.h)
        self.ws = None
        if ws:
            self.ws = torch.empty(ws, dtype=torch.uint8, device="cuda")
            assert lib.fft_plan_set_workspace(self.h, ctypes.c_void_p(self.ws.data_ptr())) == 0

    def run(self, x: torch.Tensor, d: int, out=None) -> torch.Tensor:
        out = torch.empty_like(x) if out is None else out
        s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = self.lib.fft_exec_dir(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), d, s)
        assert rc == 0, _lib.ERRORS.get(rc, rc)
        return out

    def __del__(self):
        self.lib.fft_destroy(self.h)


def run_1d(lib, x: np.ndarray, d: int, inplace=False) -> np.ndarray:
    batch, n = x.shape
    p = CPlan(lib, lib.fft_plan_create(n, batch, d, 0))
    xt = torch.from_numpy(x).cuda()
    out = p.run(xt, d, out=xt if inplace else None)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def assert_rows(got, ref, tol, what):
    errs = oracle.rel_l2_rows(got, ref)
    assert np.all(np.isfinite(got)), f"{what}: non-finite output"
    assert errs.max() <= tol, f"{what}: max rel-L2 {errs.max():.3e} > {tol:.2e} (row {errs.argmax()})"


# --- single on-chip pass: every length 2^1..2^14, ragged batches -----------------
@pytest.mark.parametrize("lg", range(1, 15))
@pytest.mark.parametrize("batch", [1, 3, 37])
def test_single_pass_forward(lib, lg, batch):
    n = 1 << lg
    x = workloads.cgauss(n, batch, seed=1000 + lg * 7 + batch)
    got = run_1d(lib, x, 0)
    assert_rows(got, oracle_dir(x, 0), tol32(n), f"fwd N={n} batch={batch}")


@pytest.mark.parametrize("lg", [1, 2, 3, 4, 5, 7, 10, 12, 13, 14])
@pytest.mark.parametrize("d", ["inv", "adj", "adj_inv"])
def test_single_pass_directions(lib, lg, d):
    n = 1 << lg
    x = workloads.uniform(n, 5, seed=2000 + lg)
    got = run_1d(lib, x, DIRS[d])
    assert_rows(got, oracle_dir(x, DIRS[d]), tol32(n), f"{d} N={n}")


@pytest.mark.parametrize("lg", [3, 8, 10, 12, 13, 14])
def test_single_pass_register_path(hooks_lib, monkeypatch, lg):
    """The non-persistent kernel (no TMA staging) gives the same result."""
    monkeypatch.setenv("GBFFT_NO_TMA", "1")
    monkeypatch.setenv("GBFFT_HALVES", "1")
    n = 1 << lg
    x = workloads.cgauss(n, 11, seed=6000 + lg)
    got = run_1d(hooks_lib, x, 1)
    assert_rows(got, oracle_dir(x, 1), tol32(n), f"register path N={n}")


@pytest.mark.parametrize("lg", [6, 10, 12])
def test_single_pass_8byte_aligned_input(lib, lg):
    """An input that is 8- but not 16-byte aligned takes the register path."""
    n = 1 << lg
    batch = 5
    x = workloads.cgauss(n, batch, seed=6100 + lg)
    p = CPlan(lib, lib.fft_plan_create(n, batch, 0, 0))
    buf = torch.zeros(n * batch + 1, dtype=torch.complex64, device="cuda")
    src = buf[1:]
    src.copy_(torch.from_numpy(x.reshape(-1)))
    assert src.data_ptr() % 16 == 8
    out = p.run(src, 0)
    torch.cuda.synchronize()
    assert_rows(out.cpu().numpy().reshape(batch, n), oracle_dir(x, 0), tol32(n), "8-byte aligned")
    assert p.lib.fft_status(p.h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0


def test_single_pass_in_place(lib):
    x = workloads.cgauss(1024, 9, seed=77)
    got = run_1d(lib, x, 0, inplace=True)
    assert_rows(got, oracle_dir(x, 0), tol32(1024), "in-place N=1024")


def test_config1_round_trip(lib):
    """N=4096, batch 1, U[-1,1]: forward against the O(N^2) DFT and the
    inverse round trip."""
    n = 4096
    x = workloads.uniform(n, 1, workloads.seed_for(0))
    X = run_1d(lib, x, 0)
    ref = oracle.dft(x.astype(np.complex128))
    assert oracle.rel_l2(X, ref) <= tol32(n)
    back = run_1d(lib, X.astype(np.complex64), 1)
    assert oracle.rel_l2(back, x) <= 2 * tol32(n)


# --- four-step: 2^15 .. 2^22 at small batch --------------------------------------
@pytest.mark.parametrize("lg", [15, 16, 17, 18, 20, 22])
def test_fourstep_forward(lib, lg):
    n = 1 << lg
    batch = 2 if lg <= 18 else 1
    x = workloads.cgauss(n, batch, seed=3000 + lg)
    got = run_1d(lib, x, 0)
    assert_rows(got, oracle_dir(x, 0), tol32(n), f"four-step fwd N=2^{lg}")


@pytest.mark.parametrize("lg,passes", [(15, 2), (17, 2), (20, 2), (22, 3), (23, 3)])
@pytest.mark.parametrize("d", ["fwd", "inv"])
def test_fourstep_register_columns(hooks_lib, monkeypatch, lg, passes, d):
    """The column passes from registers instead of tensor-TMA boxes (the
    default multi-pass plans stage them by TMA)."""
    monkeypatch.setenv("GBFFT_COLTMA", "0")
    monkeypatch.setenv("GBFFT_PASSES", str(passes))
    n = 1 << lg
    x = workloads.cgauss(n, 1, seed=3100 + lg)
    got = run_1d(hooks_lib, x, DIRS[d])
    assert_rows(got, oracle_dir(x, DIRS[d]), tol32(n), f"register columns N=2^{lg} {d}")


@pytest.mark.parametrize("lg", [15, 19])
@pytest.mark.parametrize("d", ["inv", "adj", "adj_inv"])
def test_fourstep_directions(lib, lg, d):
    n = 1 << lg
    x = workloads.uniform(n, 1, seed=4000 + lg)
    got = run_1d(lib, x, DIRS[d])
    assert_rows(got, oracle_dir(x, DIRS[d]), tol32(n), f"four-step {d} N=2^{lg}")


def test_fourstep_in_place(lib):
    n = 1 << 16
    x = workloads.cgauss(n, 3, seed=99)
    got = run_1d(lib, x, 0, inplace=True)
    assert_rows(got, oracle_dir(x, 0), tol32(n), "four-step in place")


@pytest.mark.parametrize("split", [7, 9, 12])
def test_fourstep_other_splits(hooks_lib, monkeypatch, split):
    """The same transform through different N1 x N2 splits."""
    monkeypatch.setenv("GBFFT_FORCE_SPLIT", str(split))
    n = 1 << 20
    x = workloads.cgauss(n, 1, seed=5000 + split)
    got = run_1d(hooks_lib, x, 0)
    assert_rows(got, oracle_dir(x, 0), tol32(n), f"split 2^{split} x 2^{20 - split}")


@pytest.mark.parametrize("lg,batch", [(15, 2), (18, 2), (21, 1), (23, 1)])
@pytest.mark.parametrize("d", ["fwd", "inv"])
def test_three_pass_split(hooks_lib, monkeypatch, lg, batch, d):
    """N = N1*N2*N3 in three passes (the default from 2^22 up), forced at
    smaller sizes too."""
    monkeypatch.setenv("GBFFT_PASSES", "3")
    n = 1 << lg
    x = workloads.cgauss(n, batch, seed=5500 + lg)
    got = run_1d(hooks_lib, x, DIRS[d])
    assert_rows(got, oracle_dir(x, DIRS[d]), tol32(n), f"three-pass {d} N=2^{lg}")


def test_two_pass_forced_at_2_24(hooks_lib, monkeypatch):
    monkeypatch.setenv("GBFFT_PASSES", "2")
    n = 1 << 24
    x = workloads.uniform(n, 1, seed=5600)
    got = run_1d(hooks_lib, x, 0)
    assert_rows(got, oracle.fft(x.astype(np.complex128)), tol32(n), "two-pass 2^24")


# Row passes of 2^10 / 2^11 points store their output tile with tensor TMA
# (2^18 = 2^8 x 2^10, 2^19 = 2^8 x 2^11, 2^21 = 2^10 x 2^11): whole 2^26-point
# launches (every CTA's boxes), rows sampled, both directions, in place, and
# the plain store path of the test build (GBFFT_ROWTMAS=0) bit-identical.
@pytest.mark.parametrize("lg", [18, 19, 21])
def test_tma_store_row_pass_full_size(lib, hooks_lib, monkeypatch, lg):
    n = 1 << lg
    batch = (1 << 26) // n
    x = workloads.cgauss(n, batch, seed=5650 + lg)
    rows = np.unique(np.concatenate([np.arange(0, batch, max(1, batch // 7)), [batch - 1]]))
    ref = oracle.fft(x[rows].astype(np.complex128))
    got = run_1d(lib, x, 0)
    assert_rows(got[rows], ref, tol32(n), f"TMA-store rows N=2^{lg}")
    back = run_1d(lib, got, 1, inplace=True)
    assert_rows(back[rows], x[rows].astype(np.complex128), 2 * tol32(n), f"TMA-store rows inverse N=2^{lg}")
    monkeypatch.setenv("GBFFT_ROWTMAS", "0")
    plain = run_1d(hooks_lib, x, 0)
    assert np.array_equal(plain, got), f"N=2^{lg}: TMA-store and plain row pass differ"


# --- full-size large transforms (config 3a) ----------------------------------------
@pytest.mark.parametrize("lg,batch", [(24, 1), (26, 1), (24, 2)])
def test_fourstep_full_size(lib, lg, batch):
    n = 1 << lg
    x = workloads.uniform(n, batch, workloads.seed_for(2))
    got = run_1d(lib, x, 0)
    ref = oracle.fft(x.astype(np.complex128))
    assert_rows(got, ref, tol32(n), f"N=2^{lg}")


@pytest.mark.parametrize("lg", [27, 28])
def test_maximum_lengths_by_properties(lib, lg):
    """2^27 and 2^28 (the largest 1-D lengths) through properties that hold at
    any size: a delta transforms to a constant, a single tone to one bin of
    height N, Parseval, and the inverse round trip."""
    n = 1 << lg
    p = CPlan(lib, lib.fft_plan_create(n, 1, 0, 0))
    x = torch.zeros(n, dtype=torch.complex64, device="cuda")
    x[5] = 1.0
    X = p.run(x, 0)
    k = torch.arange(n, device="cuda", dtype=torch.float64)
    ph = torch.exp(-2j * torch.pi * torch.remainder(5 * k, n) / n)
    assert float(torch.linalg.norm(X.to(torch.complex128) - ph) / np.sqrt(n)) <= tol32(n)
    m = 12345
    tone = torch.exp(2j * torch.pi * torch.remainder(m * k, n) / n).to(torch.complex64)
    T = p.run(tone, 0).to(torch.complex128)
    spike = torch.zeros(n, dtype=torch.complex128, device="cuda")
    spike[m] = n
    assert float(torch.linalg.norm(T - spike) / n) <= tol32(n)
    del tone, T, spike, ph
    g = torch.Generator(device="cuda").manual_seed(lg)
    r = torch.complex(torch.randn(n, device="cuda", generator=g), torch.randn(n, device="cuda", generator=g))
    R = p.run(r, 0)
    e_in = float(torch.sum(torch.abs(r.to(torch.complex128)) ** 2))
    e_out = float(torch.sum(torch.abs(R.to(torch.complex128)) ** 2))
    assert abs(e_out - n * e_in) <= 2 * tol32(n) * n * e_in
    back = p.run(R, 1)
    assert float(torch.linalg.norm((back - r).to(torch.complex128)) / torch.linalg.norm(r.to(torch.complex128))) \
        <= 2 * tol32(n)


# --- 2-D -----------------------------------------------------------------------
def run_2d(lib, x: np.ndarray, d: int) -> np.ndarray:
    batch, ny, nx = x.shape
    p = CPlan(lib, lib.fft_plan_create_2d(ny, nx, batch, d, 0))
    xt = torch.from_numpy(x).cuda()
    out = p.run(xt, d)
    torch.cuda.synchronize()
    return out.cpu().numpy()


# (sides of 2^10..2^12 on both axes: the transposed two-pass plan)
@pytest.mark.parametrize("ny,nx,batch", [(2, 2, 1), (8, 32, 2), (64, 16, 1), (256, 512, 1), (32, 4096, 1),
                                         (4096, 64, 1), (1024, 1024, 1), (2048, 16, 3), (16384, 8, 1),
                                         (8192, 2, 2), (1024, 1024, 3), (2048, 1024, 2), (1024, 4096, 1),
                                         (4096, 4096, 1)])
@pytest.mark.parametrize("d", ["fwd", "inv"])
def test_2d(lib, ny, nx, batch, d):
    x = workloads.cgauss(ny * nx, batch, seed=ny * 31 + nx).reshape(batch, ny, nx)
    got = run_2d(lib, x, DIRS[d])
    ref = oracle.fft2(x.astype(np.complex128), oracle.FORWARD if d == "fwd" else oracle.INVERSE)
    tol = tol32(ny * nx)
    for b in range(batch):
        assert oracle.rel_l2(got[b], ref[b]) <= tol, f"2-D {ny}x{nx} {d}"


@pytest.mark.parametrize("ny,nx,tr", [(256, 512, "1"), (512, 8192, "1"), (1024, 1024, "0"), (2048, 1024, "0")])
def test_2d_transposed_switch(hooks_lib, monkeypatch, ny, nx, tr):
    """The transposed two-pass 2-D plan forced where it is not the default,
    and the rows + column passes forced where it is (test build)."""
    monkeypatch.setenv("GBFFT_2D_TRANSPOSE", tr)
    x = workloads.cgauss(ny * nx, 2, seed=ny + 3 * nx).reshape(2, ny, nx)
    got = run_2d(hooks_lib, x, 0)
    ref = oracle.fft2(x.astype(np.complex128))
    for b in range(2):
        assert oracle.rel_l2(got[b], ref[b]) <= tol32(ny * nx), f"{ny}x{nx} transposed={tr}"


def test_2d_transposed_in_place(lib):
    ny, nx, batch = 2048, 1024, 3
    x = workloads.cgauss(ny * nx, batch, seed=91).reshape(batch, ny, nx)
    p = CPlan(lib, lib.fft_plan_create_2d(ny, nx, batch, 1, 0))
    xt = torch.from_numpy(x).cuda()
    out = p.run(xt, 1, out=xt)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = oracle.fft2(x.astype(np.complex128), oracle.INVERSE)
    for b in range(batch):
        assert oracle.rel_l2(got[b], ref[b]) <= tol32(ny * nx)


def test_2d_one_column_pass_forced(hooks_lib, monkeypatch):
    monkeypatch.setenv("GBFFT_2D_ONE_COLUMN_PASS", "1")
    x = workloads.cgauss(4096 * 32, 2, seed=77).reshape(2, 4096, 32)
    got = run_2d(hooks_lib, x, 0)
    ref = oracle.fft2(x.astype(np.complex128))
    for b in range(2):
        assert oracle.rel_l2(got[b], ref[b]) <= tol32(4096 * 32)


@pytest.mark.parametrize("ny,nx,batch", [(4096, 64, 2), (256, 512, 1), (2048, 16, 3)])
def test_2d_tensor_tma_columns(hooks_lib, monkeypatch, ny, nx, batch):
    """Column passes staged by tensor-TMA boxes (opt-in for 2-D plans)."""
    monkeypatch.setenv("GBFFT_COLTMA", "1")
    x = workloads.cgauss(ny * nx, batch, seed=ny + nx + 7).reshape(batch, ny, nx)
    got = run_2d(hooks_lib, x, 1)
    ref = oracle.fft2(x.astype(np.complex128), oracle.INVERSE)
    for b in range(batch):
        assert oracle.rel_l2(got[b], ref[b]) <= tol32(ny * nx)


def test_2d_sar_full_size(lib):
    """8192 x 8192 speckle + 64 scatterers of amplitude 100 (config 3b)."""
    x = workloads.sar_image(8192, 8192, seed=workloads.seed_for(2, 1))
    got = run_2d(lib, x[None], 0)[0]
    ref = oracle.fft2(x.astype(np.complex128))
    assert oracle.rel_l2(got, ref) <= tol32(8192 * 8192)


# --- error paths that need a device pointer ---------------------------------------
def test_misaligned_pointer_rejected(lib):
    p = CPlan(lib, lib.fft_plan_create(64, 1, 0, 0))
    buf = torch.zeros(200, dtype=torch.uint8, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.fft_exec(p.h, ctypes.c_void_p(buf.data_ptr() + 4), ctypes.c_void_p(buf.data_ptr() + 4), s)
    assert rc == -2


def test_missing_workspace(lib):
    h = ctypes.c_void_p(lib.fft_plan_create(1 << 16, 1, 0, 0))
    assert lib.fft_plan_workspace_bytes(h) == (1 << 16) * 8
    x = torch.zeros(1 << 16, dtype=torch.complex64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.fft_exec(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), s) == -3
    assert lib.fft_plan_set_workspace(h, None) == 0       # library-owned workspace
    assert lib.fft_exec(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), s) == 0
    lib.fft_destroy(h)


def test_product_library_ignores_planner_variables(lib, hooks_lib, monkeypatch):
    """Planner overrides in the environment change plans only in the test
    build: libgbfft.so builds its default plan whatever the variables say."""
    monkeypatch.setenv("GBFFT_PASSES", "3")
    monkeypatch.setenv("GBFFT_FORCE_SPLIT", "9")
    configs = {}
    for name, L in (("product", lib), ("test build", hooks_lib)):
        h = ctypes.c_void_p(L.fft_plan_create(1 << 20, 1, 0, 0))
        assert h.value
        c = _lib.FftPlanConfig()
        assert L.fft_plan_get_config(h, ctypes.byref(c)) == 0
        configs[name] = (c.npass, c.lg1)
        L.fft_destroy(h)
    assert configs["test build"][0] == 3
    assert configs["product"][0] == 2 and configs["product"][1] != 9
