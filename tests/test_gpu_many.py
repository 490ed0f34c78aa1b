"""Uneven-length batches in one persistent launch (fft_plan_create_many):
parity against the oracle per transform, CUDA-graph capture and replay, and
the bounded inter-CTA wait turning a missing producer into FFT_ERR_TIMEOUT."""
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


class ManyPlan:
    def __init__(self, lib, lengths, d=0):
        arr = (ctypes.c_int64 * len(lengths))(*[int(v) for v in lengths])
        h = lib.fft_plan_create_many(arr, len(lengths), d, 0)
        assert h, _lib.ERRORS.get(lib.fft_last_error())
        self.lib, self.h = lib, ctypes.c_void_p(h)
        ws = lib.fft_plan_workspace_bytes(self.h)
        self.ws = torch.empty(max(ws, 256), dtype=torch.uint8, device="cuda")
        if ws:
            assert lib.fft_plan_set_workspace(self.h, ctypes.c_void_p(self.ws.data_ptr())) == 0

    def run(self, x, d, out=None, stream=None):
        out = torch.empty_like(x) if out is None else out
        s = (stream or torch.cuda.current_stream()).cuda_stream
        rc = self.lib.fft_exec_dir(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), d,
                                   ctypes.c_void_p(s))
        assert rc == 0, _lib.ERRORS.get(rc, rc)
        return out

    def status(self):
        return self.lib.fft_status(self.h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))

    def __del__(self):
        self.lib.fft_destroy(self.h)


def oracle_many(x, lengths, d):
    outs, o = [], 0
    for n in lengths:
        seg = x[o:o + n].astype(np.complex128)
        if d == 3:
            outs.append(oracle.transform(seg, oracle.FORWARD) / n)
        else:
            outs.append(oracle.transform(seg, d))
        o += n
    return outs


def check(got, refs, lengths, what):
    o = 0
    for n, ref in zip(lengths, refs):
        err = oracle.rel_l2(got[o:o + n], ref)
        assert err <= 5e-7 * max(1, np.log2(n)), f"{what}: length {n} at {o}: {err:.3e}"
        o += n


@pytest.mark.parametrize("d", [0, 1, 2, 3])
def test_many_every_length(lib, d):
    # every supported length, twice, in a shuffled order
    lengths = [1 << e for e in list(range(1, 17)) * 2]
    rng = np.random.Generator(np.random.PCG64(5))
    rng.shuffle(lengths)
    x = workloads.packed_cgauss(lengths, seed=300 + d)
    p = ManyPlan(lib, lengths, d)
    got = p.run(torch.from_numpy(x).cuda(), d).cpu().numpy()
    check(got, oracle_many(x, lengths, d), lengths, f"dir {d}")
    assert p.status() == 0


def test_many_config5_shape(lib):
    """Lengths drawn like the uneven-batch workload (exponent uniform over
    8..16), 256 transforms, every transform checked."""
    lengths = workloads.uneven_lengths(256, seed=workloads.seed_for(4)).tolist()
    x = workloads.packed_cgauss(lengths, seed=workloads.seed_for(4, 2))
    p = ManyPlan(lib, lengths, 0)
    got = p.run(torch.from_numpy(x).cuda(), 0).cpu().numpy()
    check(got, oracle_many(x, lengths, 0), lengths, "cfg5-shaped")


def test_many_in_place_and_graph_replay(lib):
    lengths = workloads.uneven_lengths(64, seed=17).tolist()
    p = ManyPlan(lib, lengths, 0)
    x1 = workloads.packed_cgauss(lengths, seed=18)
    x2 = workloads.packed_cgauss(lengths, seed=19)
    buf = torch.from_numpy(x1).cuda()
    out = torch.empty_like(buf)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        p.run(buf, 0, out, stream=s)      # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        p.run(buf, 0, out, stream=s)
    for x in (x1, x2):
        buf.copy_(torch.from_numpy(x))
        g.replay()
        torch.cuda.synchronize()
        check(out.cpu().numpy(), oracle_many(x, lengths, 0), lengths, "graph replay")
    # in place
    buf.copy_(torch.from_numpy(x2))
    p.run(buf, 0, buf)
    torch.cuda.synchronize()
    check(buf.cpu().numpy(), oracle_many(x2, lengths, 0), lengths, "in place")


def test_many_bounded_wait_reports_timeout(lib, monkeypatch):
    """A row tile told to wait for a column tile that never comes gives up
    after its budget and reports FFT_ERR_TIMEOUT instead of hanging.  The
    missing producer is planted by the test build of the library
    (libgbfft_testhooks.so; the product library has no such switch)."""
    from paper_1707_07263_gb300 import build_lib
    flib = _lib.load(build_lib.TEST_LIB)
    monkeypatch.setenv("GBFFT_FAULT_MISSING_PRODUCER", "1")
    lengths = [1 << 14, 1 << 10, 1 << 16]
    x = torch.from_numpy(workloads.packed_cgauss(lengths, seed=3)).cuda()
    p = ManyPlan(flib, lengths, 0)
    p.run(x, 0)
    torch.cuda.synchronize()
    assert p.status() == -5
    p_product = ManyPlan(lib, lengths, 0)   # the product library ignores the switch
    p_product.run(x, 0)
    assert p_product.status() == 0
    monkeypatch.delenv("GBFFT_FAULT_MISSING_PRODUCER")
    p2 = ManyPlan(flib, lengths, 0)     # a fresh plan is unaffected
    p2.run(x, 0)
    assert p2.status() == 0


def test_many_config5_full_shape_forward_and_graph_gradient(lib):
    """The uneven-batch workload at its stated shape: 4096 transforms with
    lengths 2^e, e uniform over 8..16.  The forward result of every transform
    is checked against the oracle; then the benchmark's graph-captured step
    (forward, loss gradient 2 w^2 X, adjoint backward) is replayed and the
    gradient of every transform is checked against the oracle gradient
    2 F^H (w^2 F x) of L = sum |w X|^2."""
    lengths = workloads.uneven_lengths(4096, seed=workloads.seed_for(4)).tolist()
    total = int(sum(lengths))
    xh = workloads.packed_cgauss(lengths, seed=workloads.seed_for(4, 2))
    wh = workloads.real_weights(total, seed=workloads.seed_for(4, 1))
    p = ManyPlan(lib, lengths, 0)
    x = torch.from_numpy(xh).cuda()
    X = p.run(x, 0)
    torch.cuda.synchronize()
    assert p.status() == 0
    check(X.cpu().numpy(), oracle_many(xh, lengths, 0), lengths, "cfg5 forward, 4096 transforms")

    w2 = torch.from_numpy(2.0 * wh.astype(np.float32) ** 2).cuda()
    G = torch.empty_like(x)
    gx = torch.empty_like(x)
    s = torch.cuda.Stream()

    def step():
        p.run(x, 0, X, stream=s)
        torch.mul(X, w2, out=G)
        p.run(G, 2, gx, stream=s)

    with torch.cuda.stream(s):
        step()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        step()
    gx.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert p.status() == 0
    got = gx.cpu().numpy()
    o = 0
    for n in lengths:
        ref = oracle.spectral_loss_grad(xh[o:o + n].astype(np.complex128), wh[o:o + n].astype(np.float64))
        err = oracle.rel_l2(got[o:o + n], ref)
        assert err <= 1e-6 * np.log2(n), f"gradient, length {n} at {o}: {err:.3e}"
        o += n


@pytest.mark.parametrize("cfg", [{"gap": 1, "ctas_per_sm": 2, "lg1": [7, 8, 7, 8]},
                                 {"gap": 8, "ctas_per_sm": 3, "lg1": [7, 8, 8, 8]},
                                 {"gap": 3, "ctas_per_sm": 9, "lg1": [0, 0, 0, 0]}])
def test_many_explicit_configs(lib, cfg):
    """Every split the configuration offers, short and long gaps, fewer
    resident CTAs (and a count above the occupancy limit, which is lowered),
    against the oracle for every transform and direction."""
    lengths = [1 << e for e in (13, 14, 15, 16, 9, 14, 13, 12, 16, 15, 1)] * 3
    arr = (ctypes.c_int64 * len(lengths))(*lengths)
    c = _lib.FftManyConfig.from_dict(cfg)
    for d in (0, 1):
        h = lib.fft_plan_create_many_config(arr, len(lengths), d, 0, ctypes.byref(c))
        assert h, _lib.ERRORS.get(lib.fft_last_error())
        got_cfg = _lib.FftManyConfig()
        assert lib.fft_plan_get_many_config(ctypes.c_void_p(h), ctypes.byref(got_cfg)) == 0
        res = got_cfg.as_dict()
        assert 1 <= res["ctas_per_sm"] <= min(max(cfg["ctas_per_sm"], 1), 4)
        for i, v in enumerate(cfg["lg1"]):
            assert res["lg1"][i] == (v if v > 0 else (7, 7, 8, 8)[i])
        lib.fft_destroy(ctypes.c_void_p(h))
        p = ManyPlanCfg(lib, lengths, d, c)
        x = workloads.packed_cgauss(lengths, seed=800 + d)
        got = p.run(torch.from_numpy(x).cuda(), d).cpu().numpy()
        check(got, oracle_many(x, lengths, d), lengths, f"config {cfg} dir {d}")
        assert p.status() == 0


class ManyPlanCfg(ManyPlan):
    def __init__(self, lib, lengths, d, cfg):
        arr = (ctypes.c_int64 * len(lengths))(*[int(v) for v in lengths])
        h = lib.fft_plan_create_many_config(arr, len(lengths), d, 0, ctypes.byref(cfg))
        assert h, _lib.ERRORS.get(lib.fft_last_error())
        self.lib, self.h = lib, ctypes.c_void_p(h)
        ws = lib.fft_plan_workspace_bytes(self.h)
        self.ws = torch.empty(max(ws, 256), dtype=torch.uint8, device="cuda")
        if ws:
            assert lib.fft_plan_set_workspace(self.h, ctypes.c_void_p(self.ws.data_ptr())) == 0


def test_many_autotuned_plan_matches_oracle(lib, tmp_path, monkeypatch):
    """The native search over uneven-batch configurations returns a valid
    configuration, the tuned plan (built through the per-GPU cache) matches
    the oracle on every transform, and the result is cached."""
    monkeypatch.setenv("GBFFT_TUNE_CACHE", str(tmp_path / "tune.json"))
    from paper_1707_07263_gb300 import api, tune
    lengths = workloads.uneven_lengths(512, seed=workloads.seed_for(4, 7)).tolist()
    cfg = tune.tuned_many_config(lengths, torch.device("cuda", 0))
    assert set(cfg) == {"gap", "ctas_per_sm", "lg1"} and 1 <= cfg["gap"] <= 16
    assert (tmp_path / "tune.json").exists()
    assert tune.tuned_many_config(lengths, torch.device("cuda", 0)) == cfg     # from the cache now
    x = workloads.packed_cgauss(lengths, seed=901)
    xt = torch.from_numpy(x).cuda()
    got = api.fft_many(xt, lengths, tuned=True).cpu().numpy()
    check(got, oracle_many(x, lengths, 0), lengths, f"tuned {cfg}")
    back = api.fft_many(torch.from_numpy(got).cuda(), lengths, inverse=True, tuned=True).cpu().numpy()
    assert oracle.rel_l2(back, x) <= 2 * 5e-7 * 16
