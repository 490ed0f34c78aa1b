"""The Python API's argument checks (raised before any launch) and its
empty-batch cases."""
from __future__ import annotations

import pytest
import torch

import paper_1707_07263_gb300 as gb

pytestmark = pytest.mark.gpu


def test_plan_rejects_wrong_sizes_before_launching():
    p = gb.get_plan("1d", (256,), 4)
    x = torch.zeros(256 * 4, dtype=torch.complex64, device="cuda")
    assert p.numel() == 1024
    with pytest.raises(ValueError):
        p(x[:1000])                                   # too few elements: would read past the end
    with pytest.raises(ValueError):
        p(x, out=torch.empty(512, dtype=torch.complex64, device="cuda"))
    with pytest.raises(ValueError):
        p(x, out=torch.empty(2048, dtype=torch.complex64, device="cuda")[::2])   # not contiguous
    with pytest.raises(TypeError):
        p(x.to(torch.complex128))
    with pytest.raises(TypeError):
        p(x.cpu())
    assert p(x).shape == x.shape
    p2 = gb.get_plan("2d", (16, 32), 2)
    assert p2.numel() == 16 * 32 * 2
    with pytest.raises(ValueError):
        p2(torch.zeros(16 * 32, dtype=torch.complex64, device="cuda"))
    pr = gb.get_plan("r2c", (64,), 1)
    with pytest.raises(TypeError):
        pr(torch.zeros(64, dtype=torch.complex64, device="cuda"))
    torch.cuda.synchronize()


def test_empty_batches():
    for f in (gb.fft, gb.ifft):
        x = torch.empty(0, 64, dtype=torch.complex64, device="cuda", requires_grad=True)
        y = f(x)
        assert y.shape == (0, 64)
        y.abs().sum().backward()
        assert x.grad.shape == (0, 64)
    x2 = torch.empty(0, 8, 8, dtype=torch.complex64, device="cuda")
    assert gb.fft2(x2).shape == (0, 8, 8) and gb.ifft2(x2).shape == (0, 8, 8)
    assert gb.fft_many(torch.empty(0, dtype=torch.complex64, device="cuda"), []).shape == (0,)
    r = gb.rfft(torch.empty(0, 16, dtype=torch.float32, device="cuda"))
    assert r.shape == (0, 9) and r.dtype == torch.complex64
    assert gb.irfft(r).shape == (0, 16)
    torch.cuda.synchronize()
