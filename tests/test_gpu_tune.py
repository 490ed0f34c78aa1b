"""Plan configurations and the native autotuner."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1707_07263_gb300 import _lib, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    return _lib.load()


def run_cfg(lib, x: np.ndarray, cfg: dict) -> np.ndarray:
    batch, n = x.shape
    c = _lib.FftPlanConfig.from_dict(cfg)
    h = ctypes.c_void_p(lib.fft_plan_create_config(n, batch, 0, 0, ctypes.byref(c)))
    assert h.value, (cfg, _lib.ERRORS.get(lib.fft_last_error()))
    got_cfg = _lib.FftPlanConfig()
    assert lib.fft_plan_get_config(h, ctypes.byref(got_cfg)) == 0
    ws = lib.fft_plan_workspace_bytes(h)
    wsb = torch.empty(max(ws, 1), dtype=torch.uint8, device="cuda")
    if ws:
        assert lib.fft_plan_set_workspace(h, ctypes.c_void_p(wsb.data_ptr())) == 0
    xt = torch.from_numpy(x).cuda()
    out = torch.empty_like(xt)
    assert lib.fft_exec(h, ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    torch.cuda.synchronize()
    lib.fft_destroy(h)
    return out.cpu().numpy(), got_cfg.as_dict()


@pytest.mark.parametrize("lg,cfg", [
    (13, {"npass": 1, "tma": 1}),
    (14, {"npass": 1, "tma": 1}),
    (8, {"npass": 1, "tma": 1}),
    (11, {"npass": 1, "tma": 0}),
    (14, {"npass": 2, "lg1": 7, "c1": 16, "c2": 16}),
    (12, {"npass": 2, "lg1": 5, "c1": 4, "c2": 16}),
    (10, {"npass": 2, "lg1": 3, "c1": 16, "c2": 8}),
    (20, {"npass": 2, "lg1": 9, "c1": 16, "c2": 8}),
    (20, {"npass": 3, "lg1": 7, "lg2": 7, "c1": 16, "c2": 8, "c3": 16}),
    (18, {"npass": 3, "lg1": 6, "lg2": 6}),
    (16, {"npass": 2, "lg1": 8, "c1": 16, "c2": 8, "tma": 1}),
    (20, {"npass": 2, "lg1": 8, "c1": 32, "c2": 4, "tma": 1}),
    (21, {"npass": 3, "lg1": 7, "lg2": 7, "c1": 32, "c2": 16, "c3": 16, "tma": 1}),
    (12, {"npass": 1, "halves": 2}),
    (13, {"npass": 1, "halves": 2}),
    (14, {"npass": 1, "halves": 2}),
    (12, {"npass": 1, "tma": 2}),
    (13, {"npass": 1, "tma": 2}),
    (14, {"npass": 1, "tma": 2}),
    (12, {"npass": 1, "tma": 3}),
    (13, {"npass": 1, "tma": 3}),
    (14, {"npass": 1, "tma": 3}),
    (14, {"npass": 1, "tma": 0}),
])
def test_explicit_configs(lib, lg, cfg):
    n = 1 << lg
    x = workloads.cgauss(n, 3, seed=8000 + lg)
    got, used = run_cfg(lib, x, cfg)
    for k, v in cfg.items():
        assert used[k] == v, (k, used)
    ref = oracle.transform(x.astype(np.complex128))
    assert oracle.rel_l2_rows(got, ref).max() <= 5e-7 * lg


@pytest.mark.parametrize("lg", [13, 14])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_two_cta_split_directions(lib, lg, d):
    n = 1 << lg
    x = workloads.uniform(n, 5, seed=8200 + lg + d)
    c = _lib.FftPlanConfig.from_dict({"npass": 1, "halves": 2})
    h = ctypes.c_void_p(lib.fft_plan_create_config(n, 5, d, 0, ctypes.byref(c)))
    assert h.value
    xt = torch.from_numpy(x).cuda()
    out = torch.empty_like(xt)
    assert lib.fft_exec(h, ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    torch.cuda.synchronize()
    lib.fft_destroy(h)
    x64 = x.astype(np.complex128)
    ref = {1: oracle.fft(x64, oracle.INVERSE), 2: oracle.fft(x64, oracle.ADJOINT),
           3: oracle.fft(x64, oracle.FORWARD) / n}[d]
    assert oracle.rel_l2_rows(out.cpu().numpy(), ref).max() <= 5e-7 * lg


@pytest.mark.parametrize("lg,batch,d", [(14, 333, 0), (14, 457, 1), (13, 700, 2), (12, 1337, 3)])
def test_prefetching_persistent_kernel_loops(lib, lg, batch, d):
    """Persistent single pass with the L2 prefetch (tma = 2): more transforms
    than resident CTAs, so every CTA loops and prefetches; every direction."""
    n = 1 << lg
    x = workloads.cgauss(n, batch, seed=8300 + lg + d)
    c = _lib.FftPlanConfig.from_dict({"npass": 1, "tma": 2})
    h = ctypes.c_void_p(lib.fft_plan_create_config(n, batch, d, 0, ctypes.byref(c)))
    assert h.value
    got_cfg = _lib.FftPlanConfig()
    assert lib.fft_plan_get_config(h, ctypes.byref(got_cfg)) == 0 and got_cfg.tma == 2
    xt = torch.from_numpy(x).cuda()
    out = torch.empty_like(xt)
    assert lib.fft_exec(h, ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    torch.cuda.synchronize()
    lib.fft_destroy(h)
    x64 = x.astype(np.complex128)
    ref = {0: oracle.fft(x64), 1: oracle.fft(x64, oracle.INVERSE), 2: oracle.fft(x64, oracle.ADJOINT),
           3: oracle.fft(x64, oracle.FORWARD) / n}[d]
    assert oracle.rel_l2_rows(out.cpu().numpy(), ref).max() <= 5e-7 * lg


def test_unsupported_config_is_rejected(lib):
    # a row pass of length 2^3 has no compiled kernel
    c = _lib.FftPlanConfig.from_dict({"npass": 2, "lg1": 7})
    assert lib.fft_plan_create_config(1 << 10, 1, 0, 0, ctypes.byref(c)) is None
    assert lib.fft_last_error() == -6


@pytest.mark.parametrize("lg,batch", [(12, 64), (17, 4)])
def test_autotune_returns_a_working_config(lib, lg, batch, tmp_path, monkeypatch):
    monkeypatch.setenv("GBFFT_TUNE_CACHE", str(tmp_path / "tune.json"))
    from paper_1707_07263_gb300 import tune
    n = 1 << lg
    cfg = tune.tuned_config(n, batch, 0)
    assert cfg["npass"] in (1, 2, 3)
    assert (tmp_path / "tune.json").exists()
    x = workloads.cgauss(n, batch, seed=8100 + lg)
    got, _ = run_cfg(lib, x, cfg)
    assert oracle.rel_l2_rows(got, oracle.transform(x.astype(np.complex128))).max() <= 5e-7 * lg
    # the cached answer is reused
    assert tune.tuned_config(n, batch, 0) == cfg


@pytest.mark.parametrize("lg", [12, 13, 14])
@pytest.mark.parametrize("d", [0, 1, 2, 3])
def test_staged_persistent_kernel_loops(lib, lg, d):
    """tma = 3 (the next transform bulk-copied into the exchange buffer once
    the last pass has read it): several transforms per CTA (batch well above
    the resident grid), every direction, each transform against the oracle;
    an 8-byte-aligned input takes the non-staged kernel and gives the same
    result."""
    n = 1 << lg
    batch = 1100 if lg == 14 else 2100
    x = workloads.cgauss(n, batch, seed=8600 + lg + 17 * d)
    c = _lib.FftPlanConfig.from_dict({"npass": 1, "tma": 3})
    h = ctypes.c_void_p(lib.fft_plan_create_config(n, batch, d, 0, ctypes.byref(c)))
    assert h.value, _lib.ERRORS.get(lib.fft_last_error())
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    buf = torch.zeros(n * batch + 1, dtype=torch.complex64, device="cuda")
    xt = buf[:-1]
    xt.copy_(torch.from_numpy(x.reshape(-1)))
    assert xt.data_ptr() % 16 == 0
    out = torch.empty_like(xt)
    assert lib.fft_exec(h, ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(out.data_ptr()), s) == 0
    x8 = buf[1:]
    x8.copy_(torch.from_numpy(x.reshape(-1)))
    assert x8.data_ptr() % 16 == 8
    out8 = torch.empty_like(x8)
    assert lib.fft_exec(h, ctypes.c_void_p(x8.data_ptr()), ctypes.c_void_p(out8.data_ptr()), s) == 0
    torch.cuda.synchronize()
    assert lib.fft_status(h, s) == 0
    lib.fft_destroy(h)
    x64 = x.astype(np.complex128)
    ref = {0: oracle.fft(x64), 1: oracle.fft(x64, oracle.INVERSE), 2: oracle.fft(x64, oracle.ADJOINT),
           3: oracle.fft(x64) / n}[d]
    got = out.cpu().numpy().reshape(batch, n)
    assert oracle.rel_l2_rows(got, ref).max() <= 5e-7 * lg
    got8 = out8.cpu().numpy().reshape(batch, n)
    assert oracle.rel_l2_rows(got8, ref).max() <= 5e-7 * lg


RADIX_CASES = [(8, lg) for lg in range(5, 14)] + [(4, lg) for lg in range(5, 13)]


@pytest.mark.parametrize("radix,lg", RADIX_CASES)
def test_smaller_radix_single_pass(lib, radix, lg):
    """One on-chip pass with radix-8 or radix-4 Stockham passes (8 / 4 points
    per thread, so 2x / 4x the threads of the radix-16 kernel): every compiled
    length, a batch of two full tiles plus a ragged one, every direction
    through one plan, and one call in place; each transform against the
    oracle.  The plan reports the radix it was built with."""
    n = 1 << lg
    cols = (4096 >> lg) if lg < 12 else 1
    batch = 2 * cols + max(1, cols // 3)
    x = workloads.cgauss(n, batch, seed=8700 + 16 * lg + radix)
    c = _lib.FftPlanConfig.from_dict({"npass": 1, "tma": 0, "radix": radix})
    h = ctypes.c_void_p(lib.fft_plan_create_config(n, batch, 0, 0, ctypes.byref(c)))
    assert h.value, _lib.ERRORS.get(lib.fft_last_error())
    got_cfg = _lib.FftPlanConfig()
    assert lib.fft_plan_get_config(h, ctypes.byref(got_cfg)) == 0
    assert got_cfg.radix == radix and got_cfg.npass == 1 and got_cfg.tma == 0
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    xt = torch.from_numpy(x).cuda()
    x64 = x.astype(np.complex128)
    refs = {0: oracle.fft(x64), 1: oracle.fft(x64, oracle.INVERSE), 2: oracle.fft(x64, oracle.ADJOINT),
            3: oracle.fft(x64) / n}
    for d in range(4):
        out = torch.empty_like(xt)
        assert lib.fft_exec_dir(h, ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(out.data_ptr()), d, s) == 0
        torch.cuda.synchronize()
        err = oracle.rel_l2_rows(out.cpu().numpy(), refs[d]).max()
        assert err <= 5e-7 * lg, (radix, lg, d, err)
    y = xt.clone()
    assert lib.fft_exec_dir(h, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(y.data_ptr()), 1, s) == 0
    torch.cuda.synchronize()
    assert oracle.rel_l2_rows(y.cpu().numpy(), refs[1]).max() <= 5e-7 * lg
    lib.fft_destroy(h)


@pytest.mark.parametrize("lg", [9, 12])
def test_smaller_radix_agrees_with_radix16(lib, lg):
    """The three schedules compute the same transform: outputs of the radix-4,
    radix-8 and radix-16 single passes agree with each other to the FP32
    bound on a larger batch (many CTAs)."""
    n = 1 << lg
    batch = (1 << 20) // n + 7
    x = workloads.cgauss(n, batch, seed=8800 + lg)
    outs = {}
    for r in (16, 8, 4):
        got, used = run_cfg(lib, x, {"npass": 1, "tma": 0, "radix": r})
        assert used["radix"] == r
        outs[r] = got.reshape(batch, n).astype(np.complex128)
    ref = oracle.fft(x.astype(np.complex128)[:64])
    for r in (16, 8, 4):
        assert oracle.rel_l2_rows(outs[r][:64], ref).max() <= 5e-7 * lg
        assert oracle.rel_l2_rows(outs[r], outs[16]).max() <= 1e-6 * lg


@pytest.mark.parametrize("lg,radix", [(4, 16), (5, 8), (6, 8), (7, 16), (12, 16)])
def test_planner_default_radix(lib, lg, radix):
    """Left open by the configuration, one on-chip FP32 pass takes radix-8
    passes at 2^5 and 2^6 (measured faster there) and radix 16 elsewhere; the
    plan's description reports it, and the result matches the oracle."""
    n = 1 << lg
    batch = 77
    h = ctypes.c_void_p(lib.fft_plan_create(n, batch, 0, 0))
    assert h.value
    c = _lib.FftPlanConfig()
    assert lib.fft_plan_get_config(h, ctypes.byref(c)) == 0 and c.radix == radix
    buf = ctypes.create_string_buffer(512)
    lib.fft_plan_describe(h, buf, 512)
    assert f"radix={radix}" in buf.value.decode()
    x = workloads.cgauss(n, batch, seed=8900 + lg)
    xt = torch.from_numpy(x).cuda()
    out = torch.empty_like(xt)
    assert lib.fft_exec(h, ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    torch.cuda.synchronize()
    lib.fft_destroy(h)
    assert oracle.rel_l2_rows(out.cpu().numpy(), oracle.fft(x.astype(np.complex128))).max() <= 5e-7 * max(lg, 1)
