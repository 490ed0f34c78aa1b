"""Host-resident batches: the direct mode (kernels read and write page-locked
host memory) and the copy pipeline (uploads, transforms and downloads
overlapped on three streams) both equal the oracle, including ragged last
chunks, single chunks, multi-pass plans and the inverse; shared streams keep
successive pipelines ordered; fft_pointer_usable classifies pointers."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1707_07263_gb300 as gb
from paper_1707_07263_gb300 import _lib as L
from paper_1707_07263_gb300 import workloads

pytestmark = pytest.mark.gpu


def _pinned(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def _ref(x, inverse):
    return oracle.transform(x.astype(np.complex128), oracle.INVERSE if inverse else oracle.FORWARD)


@pytest.mark.parametrize("lg,batch,chunk", [(4, 37, 5), (10, 9, 4), (12, 6, 6), (12, 5, 16), (16, 3, 1)])
@pytest.mark.parametrize("inverse", [False, True])
def test_copy_pipeline_matches_oracle(lg, batch, chunk, inverse):
    n = 1 << lg
    x = workloads.cgauss(n, batch, seed=3100 + lg * 7 + batch)
    p = gb.HostPipeline(n, batch, gb.FFT_INVERSE if inverse else gb.FFT_FORWARD, chunk=chunk, direct=False)
    out = torch.empty(batch, n, dtype=torch.complex64).pin_memory()
    p(_pinned(x), out)
    torch.cuda.synchronize()
    assert p.last_mode == "copy"
    assert oracle.rel_l2_rows(out.numpy(), _ref(x, inverse)).max() <= 2e-7 * lg


@pytest.mark.parametrize("lg,batch", [(1, 5), (6, 100), (10, 33), (13, 7), (14, 3), (16, 2), (20, 1)])
@pytest.mark.parametrize("inverse", [False, True])
def test_direct_matches_oracle(lg, batch, inverse):
    """Kernels on page-locked host buffers; one-pass lengths pick direct by
    default, multi-pass lengths (2^16, 2^20) take it when asked."""
    n = 1 << lg
    x = workloads.cgauss(n, batch, seed=3200 + lg * 7 + batch)
    p = gb.HostPipeline(n, batch, gb.FFT_INVERSE if inverse else gb.FFT_FORWARD, direct=True if lg > 14 else None)
    out = torch.empty(batch, n, dtype=torch.complex64).pin_memory()
    p(_pinned(x), out)
    torch.cuda.synchronize()
    assert p.last_mode == "direct"
    assert oracle.rel_l2_rows(out.numpy(), _ref(x, inverse)).max() <= 2e-7 * lg


def test_direct_equals_device_bitwise():
    """The same kernel on host or device memory computes the same bits."""
    n, batch = 4096, 64
    x = workloads.cgauss(n, batch, seed=3333)
    xd = torch.from_numpy(x).cuda()
    dev = gb.fft(xd).cpu()
    out = torch.empty(batch, n, dtype=torch.complex64).pin_memory()
    gb.HostPipeline(n, batch)(_pinned(x), out)
    torch.cuda.synchronize()
    assert torch.equal(out, dev)


def test_pageable_host_falls_back_to_copies():
    n, batch = 1024, 8
    x = workloads.cgauss(n, batch, seed=3401)
    p = gb.HostPipeline(n, batch)
    xin = torch.from_numpy(x.copy())            # pageable
    out = torch.empty(batch, n, dtype=torch.complex64)
    assert not p.usable(xin)
    p(xin, out)
    torch.cuda.synchronize()
    assert p.last_mode == "copy"
    assert oracle.rel_l2_rows(out.numpy(), _ref(x, False)).max() <= 2e-6
    with pytest.raises(ValueError):
        gb.HostPipeline(n, batch, direct=True)(xin, out)


def test_pipelines_sharing_streams():
    """Two pipelines on one stream triple, run back to back without a join in
    between (one direct, one copying), into separate output buffers."""
    n1, b1, n2, b2 = 256, 40, 4096, 7
    x1 = workloads.cgauss(n1, b1, seed=3301)
    x2 = workloads.cgauss(n2, b2, seed=3302)
    p1 = gb.HostPipeline(n1, b1, gb.FFT_FORWARD, chunk=3)
    p2 = gb.HostPipeline(n2, b2, gb.FFT_INVERSE, chunk=2, streams=p1.streams, direct=False)
    h1, h2 = _pinned(x1), _pinned(x2)
    o1 = torch.empty_like(h1).pin_memory()
    o2 = torch.empty_like(h2).pin_memory()
    for _ in range(2):
        p1(h1, o1, join=False)
        p2(h2, o2)
        torch.cuda.synchronize()
    assert (p1.last_mode, p2.last_mode) == ("direct", "copy")
    assert oracle.rel_l2_rows(o1.numpy(), _ref(x1, False)).max() <= 2e-6
    assert oracle.rel_l2_rows(o2.numpy(), _ref(x2, True)).max() <= 3e-6


def test_pointer_usable():
    lib = L.load()
    d = torch.zeros(1024, dtype=torch.complex64, device="cuda")
    h = torch.zeros(1024, dtype=torch.complex64).pin_memory()
    g = torch.zeros(1024, dtype=torch.complex64)
    nb = 1024 * 8
    assert lib.fft_pointer_usable(ctypes.c_void_p(d.data_ptr()), nb) == 1
    assert lib.fft_pointer_usable(ctypes.c_void_p(h.data_ptr()), nb) == 1
    assert lib.fft_pointer_usable(ctypes.c_void_p(g.data_ptr()), nb) == 0
    assert lib.fft_pointer_usable(None, nb) < 0
    assert lib.fft_pointer_usable(ctypes.c_void_p(d.data_ptr()), 0) < 0


def test_host_pipeline_rejects_device_tensors():
    p = gb.HostPipeline(64, 2)
    x = torch.zeros(128, dtype=torch.complex64, device="cuda")
    with pytest.raises(TypeError):
        p(x, x)
