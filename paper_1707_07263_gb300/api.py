"""PyTorch-facing API: plans over the C ABI plus autograd Functions.

PyTorch supplies device memory and streams only.  Every transform, inverse
and adjoint runs in libgbfft's CUDA kernels; if the library or a GPU is
missing these calls raise instead of computing anything another way.

Conventions (paper Sec. 2.1): ``fft`` is Eq. 1 with W_N = exp(-2*pi*i/N),
``ifft`` is Eq. 2 (with 1/N), natural-order outputs.  Gradients follow
PyTorch's complex convention: for y = F x the backward pass returns F^H g,
which is the adjoint transform (conjugate direction, no 1/N, Eq. 4); for
y = F^{-1} x it returns (1/N) F g.
"""
from __future__ import annotations

import ctypes
import threading

import torch

from . import _lib as L

FORWARD, INVERSE, ADJOINT = L.FFT_FORWARD, L.FFT_INVERSE, L.FFT_ADJOINT
PREC = {
    "fp32": L.FFT_PREC_FP32,
    "tc_bf16": L.FFT_PREC_TC_BF16,
    "tc_fp16": L.FFT_PREC_TC_FP16,
    "tc_bf16_split": L.FFT_PREC_TC_BF16_SPLIT,
    "tc_fp16_split": L.FFT_PREC_TC_FP16_SPLIT,
    "fp64": L.FFT_PREC_FP64,
}


def _prec_code(prec) -> int:
    if isinstance(prec, int):
        return prec
    return PREC[prec]


def _stream_handle(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Plan:
    """Owns one library plan and (for four-step plans) its torch-allocated
    workspace.  ``kind`` is "1d", "2d", "many" or "r2c" (real data)."""

    def __init__(self, kind: str, shape, batch: int = 1, dir: int = FORWARD, prec="fp32",
                 device=None, lengths=None, config: dict | None = None):
        self.lib = L.load()
        self.kind = kind
        self.shape = tuple(shape)
        self.batch = int(batch)
        self.dir = int(dir)
        self.prec = _prec_code(prec)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            if kind == "1d" and config is not None:
                cfg = L.FftPlanConfig.from_dict(config)
                h = self.lib.fft_plan_create_config(int(shape[0]), self.batch, self.dir, self.prec, ctypes.byref(cfg))
            elif kind == "1d":
                h = self.lib.fft_plan_create(int(shape[0]), self.batch, self.dir, self.prec)
            elif kind == "2d":
                h = self.lib.fft_plan_create_2d(int(shape[0]), int(shape[1]), self.batch, self.dir, self.prec)
            elif kind == "r2c":
                h = self.lib.fft_plan_create_r2c(int(shape[0]), self.batch, self.prec)
            elif kind == "many":
                arr = (ctypes.c_int64 * len(lengths))(*[int(v) for v in lengths])
                self.lengths = [int(v) for v in lengths]
                if config is not None:
                    mc = L.FftManyConfig.from_dict(config)
                    h = self.lib.fft_plan_create_many_config(arr, len(lengths), self.dir, self.prec, ctypes.byref(mc))
                else:
                    h = self.lib.fft_plan_create_many(arr, len(lengths), self.dir, self.prec)
            else:
                raise ValueError(kind)
            if not h:
                raise L.GbfftError(self.lib.fft_last_error(), f"plan {kind} {shape} batch={batch} prec={prec}")
            self.handle = ctypes.c_void_p(h)
            self.ws_bytes = int(self.lib.fft_plan_workspace_bytes(self.handle))
            self.workspace = None
            if self.ws_bytes:
                # the workspace belongs to torch; the library only borrows it
                self.workspace = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
                ptr = self.workspace.data_ptr()
                ptr = (ptr + 255) & ~255
                L.check(self.lib.fft_plan_set_workspace(self.handle, ctypes.c_void_p(ptr)), "set_workspace")

    @property
    def launches(self) -> int:
        return int(self.lib.fft_plan_launches(self.handle))

    def many_config(self) -> dict:
        """Resolved configuration of an uneven-batch plan."""
        c = L.FftManyConfig()
        L.check(self.lib.fft_plan_get_many_config(self.handle, ctypes.byref(c)), "fft_plan_get_many_config")
        return c.as_dict()

    def describe(self) -> str:
        buf = ctypes.create_string_buffer(512)
        self.lib.fft_plan_describe(self.handle, buf, 512)
        return buf.value.decode()

    def exec_ptr(self, in_ptr: int, out_ptr: int, dir: int | None = None, stream=None) -> None:
        d = self.dir if dir is None else int(dir)
        rc = self.lib.fft_exec_dir(self.handle, ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr), d,
                                   ctypes.c_void_p(_stream_handle(stream)))
        L.check(rc, "fft_exec")

    def numel(self) -> int:
        """Complex elements one execution reads and writes."""
        if self.kind == "many":
            return sum(self.lengths)
        m = self.batch
        for d in self.shape:
            m *= int(d)
        return m

    def __call__(self, x: torch.Tensor, out: torch.Tensor | None = None, dir: int | None = None,
                 stream=None) -> torch.Tensor:
        if self.kind == "r2c":
            raise TypeError("real plans run through rfft / irfft")
        want = torch.complex128 if self.prec == L.FFT_PREC_FP64 else torch.complex64
        if x.dtype != want or not x.is_cuda or x.device != self.device:
            raise TypeError(f"expected a {want} tensor on {self.device}")
        if x.numel() != self.numel():
            raise ValueError(f"expected {self.numel()} elements, got {x.numel()}")
        x = x.contiguous()
        if out is None:
            out = torch.empty_like(x)
        elif (out.dtype != want or out.device != self.device or out.numel() != x.numel()
              or not out.is_contiguous()):
            raise ValueError("out must be a contiguous tensor of the input's dtype, device and size")
        self.exec_ptr(x.data_ptr(), out.data_ptr(), dir, stream)
        return out

    def exec_filter_ptr(self, in_ptr: int, out_ptr: int, filt_ptr: int, stream=None, dir: int = FORWARD) -> None:
        """Range compression IFFT(H * FFT(row)) of every row, or with
        dir=ADJOINT its adjoint IFFT(conj(H) * FFT(row)) (fft_exec_filter_dir)."""
        rc = self.lib.fft_exec_filter_dir(self.handle, ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr),
                                          ctypes.c_void_p(filt_ptr), int(dir), ctypes.c_void_p(_stream_handle(stream)))
        L.check(rc, "fft_exec_filter_dir")

    def status(self, stream=None) -> int:
        return int(self.lib.fft_status(self.handle, ctypes.c_void_p(_stream_handle(stream))))

    def close(self) -> None:
        if getattr(self, "handle", None):
            self.lib.fft_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_cache: dict = {}
_cache_lock = threading.Lock()


def get_plan(kind: str, shape, batch: int, prec="fp32", device=None, lengths=None, tuned: bool = False) -> Plan:
    """Cached plan (twiddle tables are built once per shape/precision/device).
    tuned=True builds 1-D and uneven-batch plans from the autotuner's cached
    configuration (tuning the shape first if it has never been tuned on this
    GPU model)."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    key = (kind, tuple(shape), int(batch), _prec_code(prec), dev.index,
           tuple(lengths) if lengths is not None else None, bool(tuned and kind in ("1d", "many")))
    with _cache_lock:
        p = _cache.get(key)
        if p is None:
            config = None
            n0 = int(shape[0])
            tunable = n0 > 1 and (n0 & (n0 - 1)) == 0 and _prec_code(prec) != L.FFT_PREC_FP64
            if tuned and kind == "1d" and tunable:   # mixed-radix and FP64 plans take no configuration
                from . import tune
                config = tune.tuned_config(int(shape[0]), int(batch), _prec_code(prec), dev)
            elif tuned and kind == "many" and _prec_code(prec) == L.FFT_PREC_FP32:
                from . import tune
                config = tune.tuned_many_config(lengths, dev)
            p = Plan(kind, shape, batch, FORWARD, prec, dev, lengths, config=config)
            _cache[key] = p
        return p


def clear_plan_cache() -> None:
    with _cache_lock:
        for p in _cache.values():
            p.close()
        _cache.clear()


def _check_input(x: torch.Tensor, min_dims: int = 1, allow_fp64: bool = False) -> None:
    ok = (torch.complex64, torch.complex128) if allow_fp64 else (torch.complex64,)
    if not isinstance(x, torch.Tensor) or x.dtype not in ok or not x.is_cuda:
        raise TypeError("expected a complex64 CUDA tensor" + (" (or complex128)" if allow_fp64 else ""))
    if x.dim() < min_dims:
        raise ValueError(f"expected at least {min_dims} dimension(s)")


class _FFT1d(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, dir, prec):
        n = x.shape[-1]
        ctx.dir = dir
        ctx.plan = None
        if x.numel() == 0 and n > 0:   # no rows: nothing to transform
            return torch.empty_like(x)
        plan = get_plan("1d", (n,), x.numel() // n if n else 0, prec, x.device)
        ctx.plan = plan
        return plan(x, dir=dir)

    @staticmethod
    def backward(ctx, g):
        if ctx.plan is None:
            return torch.zeros_like(g), None, None
        return ctx.plan(g.contiguous(), dir=ctx.dir ^ ADJOINT), None, None


class _FFT2d(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, dir, prec):
        ny, nx = x.shape[-2], x.shape[-1]
        ctx.dir = dir
        ctx.plan = None
        if x.numel() == 0 and ny * nx > 0:
            return torch.empty_like(x)
        plan = get_plan("2d", (ny, nx), x.numel() // (ny * nx) if ny * nx else 0, prec, x.device)
        ctx.plan = plan
        return plan(x, dir=dir)

    @staticmethod
    def backward(ctx, g):
        if ctx.plan is None:
            return torch.zeros_like(g), None, None
        return ctx.plan(g.contiguous(), dir=ctx.dir ^ ADJOINT), None, None


class _FFTMany(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, lengths, dir, prec, tuned):
        plan = get_plan("many", (int(sum(lengths)),), len(lengths), prec, x.device, lengths=tuple(lengths),
                        tuned=tuned)
        ctx.plan, ctx.dir = plan, dir
        return plan(x, dir=dir)

    @staticmethod
    def backward(ctx, g):
        return ctx.plan(g.contiguous(), dir=ctx.dir ^ ADJOINT), None, None, None, None


def _prec_for(x: torch.Tensor, prec):
    if x.dtype == torch.complex128:
        if prec not in (None, "fp64", L.FFT_PREC_FP64):
            raise ValueError("complex128 tensors run in FP64")
        return "fp64"
    return "fp32" if prec is None else prec


def fft(x: torch.Tensor, prec=None) -> torch.Tensor:
    """Eq. 1 over the last dimension.  complex64 runs in FP32 (or a
    tensor-core precision): powers of two 2..2^28 and products 2^a 3^b 5^c 7^d
    up to 14336^2 (two passes above 14336).  complex128 runs in FP64: the same
    7-smooth lengths up to 7168^2 (powers of two up to 2^24; two passes above
    7168)."""
    _check_input(x, allow_fp64=True)
    return _FFT1d.apply(x, FORWARD, _prec_for(x, prec))


def ifft(x: torch.Tensor, prec=None) -> torch.Tensor:
    """Eq. 2 over the last dimension (same lengths and precisions as fft)."""
    _check_input(x, allow_fp64=True)
    return _FFT1d.apply(x, INVERSE, _prec_for(x, prec))


def fft2(x: torch.Tensor, prec=None) -> torch.Tensor:
    """2-D transform over the last two dimensions (rows, then columns).
    complex64: power-of-two sides up to 2^14 (any precision), or 7-smooth
    sides up to 14336 in FP32; complex128: 7-smooth sides up to 7168 in FP64."""
    _check_input(x, 2, allow_fp64=True)
    return _FFT2d.apply(x, FORWARD, _prec_for(x, prec))


def ifft2(x: torch.Tensor, prec=None) -> torch.Tensor:
    """Eq. 2 in two dimensions (same sides and precisions as fft2)."""
    _check_input(x, 2, allow_fp64=True)
    return _FFT2d.apply(x, INVERSE, _prec_for(x, prec))


def fft_many(packed: torch.Tensor, lengths, inverse: bool = False, prec="fp32", tuned: bool = False) -> torch.Tensor:
    """Transforms of uneven power-of-two lengths packed back to back in a 1-D
    complex64 tensor (transform i starts at sum(lengths[:i])).  tuned=True
    builds the plan from the autotuner's configuration for this length list on
    this GPU model (cached per GPU model; tuned once, on first use)."""
    _check_input(packed)
    lengths = [int(v) for v in lengths]
    if packed.numel() != sum(lengths):
        raise ValueError("packed size does not match the sum of the lengths")
    if not lengths:
        return packed.reshape(-1).clone()
    return _FFTMany.apply(packed.reshape(-1), lengths, INVERSE if inverse else FORWARD, prec, bool(tuned))


def _run_filter(x: torch.Tensor, H: torch.Tensor, dir: int = FORWARD) -> torch.Tensor:
    n = x.shape[-1]
    batch = x.numel() // n if n else 0
    out = torch.empty_like(x)
    if batch == 0:
        return out
    p = get_plan("1d", (n,), batch, "fp32", x.device)
    p.exec_filter_ptr(x.data_ptr(), out.data_ptr(), H.data_ptr(), dir=dir)
    return out


class _RangeCompress(torch.autograd.Function):
    """y = F^{-1} diag(H) F x per row.  Its adjoint is F^{-1} diag(conj H) F:
    the backward pass is one library call, the same fused kernels with the
    filter conjugated as it is loaded (no gradient for H)."""

    @staticmethod
    def forward(ctx, x, H):
        ctx.save_for_backward(H)
        return _run_filter(x, H)

    @staticmethod
    def backward(ctx, g):
        (H,) = ctx.saved_tensors
        return _run_filter(g.contiguous(), H, ADJOINT), None


def range_compress(x: torch.Tensor, H: torch.Tensor) -> torch.Tensor:
    """SAR range compression (fast convolution) over the last dimension:
    IFFT(H * FFT(row)) for every row, with one fused kernel per tile for
    rows of up to 2^14 points (Eq. 1, pointwise product, Eq. 2).  x: complex64
    CUDA tensor (..., n); H: complex64 CUDA tensor of n filter values in
    natural frequency order.  Differentiable in x."""
    _check_input(x)
    if H.dtype != torch.complex64 or not H.is_cuda or H.shape != x.shape[-1:]:
        raise TypeError("H must be a complex64 CUDA tensor of shape (n,)")
    if H.device != x.device:
        raise ValueError("x and H must be on the same device")
    return _RangeCompress.apply(x.contiguous(), H.detach().contiguous())


def _run_real(x: torch.Tensor, n: int, dir: int) -> torch.Tensor:
    """Through a cached real plan: real-to-complex (dir FORWARD, float32 rows
    of n -> complex64 rows of n/2 + 1; float64 -> complex128 in FP64) or
    complex-to-real (dir INVERSE), and their adjoints (ADJOINT: complex rows ->
    real rows; INVERSE | ADJOINT: real rows -> complex rows)."""
    rows = x.shape[:-1]
    batch = 1
    for d in rows:
        batch *= int(d)
    fp64 = x.dtype in (torch.float64, torch.complex128)
    if dir in (FORWARD, INVERSE | ADJOINT):
        out = torch.empty(rows + (n // 2 + 1,), dtype=torch.complex128 if fp64 else torch.complex64, device=x.device)
    else:
        out = torch.empty(rows + (n,), dtype=torch.float64 if fp64 else torch.float32, device=x.device)
    if batch == 0:
        return out
    p = get_plan("r2c", (n,), batch, "fp64" if fp64 else "fp32", x.device)
    p.exec_ptr(x.data_ptr(), out.data_ptr(), dir)
    return out


class _RFFT(torch.autograd.Function):
    """X = rfft(x).  For real x the gradient is Re(sum_k g_k W^{-nk}) over the
    kept outputs: the adjoint of the real-to-complex transform, one library
    call (FFT_ADJOINT on the real plan)."""

    @staticmethod
    def forward(ctx, x):
        ctx.n = x.shape[-1]
        return _run_real(x, ctx.n, FORWARD)

    @staticmethod
    def backward(ctx, g):
        return _run_real(g.contiguous(), ctx.n, ADJOINT)


class _IRFFT(torch.autograd.Function):
    """x = irfft(X, n).  The gradient is the adjoint of the complex-to-real
    transform: Eq. 1 of g with the interior bins times 2/n (each stands for
    itself and its conjugate partner) and bins 0, n/2 times 1/n, one library
    call (FFT_INVERSE | FFT_ADJOINT on the real plan)."""

    @staticmethod
    def forward(ctx, X, n):
        ctx.n = n
        return _run_real(X, n, INVERSE)

    @staticmethod
    def backward(ctx, g):
        return _run_real(g.contiguous(), ctx.n, INVERSE | ADJOINT), None


def rfft(x: torch.Tensor) -> torch.Tensor:
    """Eq. 1 of real rows (last dimension): the n/2 + 1 non-redundant
    outputs.  float32 CUDA tensor (n a power of two >= 4; one fused kernel for
    n <= 2^15) -> complex64, or float64 (FP64; any even n >= 4 whose half is
    a 7-smooth FP64 length) -> complex128.  Differentiable."""
    if not isinstance(x, torch.Tensor) or x.dtype not in (torch.float32, torch.float64) or not x.is_cuda:
        raise TypeError("expected a float32 or float64 CUDA tensor")
    return _RFFT.apply(x.contiguous())


def irfft(X: torch.Tensor, n: int | None = None) -> torch.Tensor:
    """Eq. 2 (with 1/n) of the Hermitian extension of X[0..n/2] (last
    dimension): real rows of length n (default 2 * (X.shape[-1] - 1)); the
    imaginary parts of X[0] and X[n/2] are ignored.  complex64 -> float32,
    complex128 -> float64 (FP64).  Differentiable."""
    _check_input(X, allow_fp64=True)
    if n is None:
        n = 2 * (X.shape[-1] - 1)
    if X.shape[-1] != n // 2 + 1:
        raise ValueError(f"irfft: {X.shape[-1]} values for length {n}")
    return _IRFFT.apply(X.contiguous(), int(n))


class HostPipeline:
    """Transforms of data that lives in (pinned) HOST memory, end to end.

    The paper's GPU times include moving the data to and from the device, the
    part it finds limiting (Sec. 3, Sec. 4).  Two ways across the host link:

    direct  the plan runs on the host buffers themselves: its kernels read the
            input and write the output over the link (page-locked memory that
            the library reports usable, fft_pointer_usable).  One launch per
            pass, no device buffer for the data and no copy engine.
    copy    the batch is cut into chunks and three CUDA streams overlap the
            upload of chunk i+1, the transform of chunk i and the download of
            chunk i-1, events ordering each chunk's steps; two device buffers
            per stage, allocated on first use.  A batch that fits one chunk
            runs its three steps in order on the transform stream (nothing to
            overlap, no events).

    direct=None picks direct for one-pass plans when both buffers are usable
    and copy otherwise; True / False force one (True raises if a buffer is not
    usable).  n: transform length; batch: transforms per call; chunk:
    transforms per chunk of the copy mode (default: about 64 MiB); streams: an
    optional (upload, transform, download) stream triple shared by several
    pipelines so that they overlap one another.
    """

    def __init__(self, n: int, batch: int, dir: int = FORWARD, prec="fp32", device=None, chunk: int | None = None,
                 streams=None, direct: bool | None = None):
        self.n, self.batch, self.dir, self.prec = int(n), int(batch), int(dir), prec
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.lib = L.load()
        if chunk is None:
            chunk = max(1, (64 << 20) // (8 * self.n))
        self.chunk = int(min(max(1, chunk), self.batch))
        self.nchunks = (self.batch + self.chunk - 1) // self.chunk
        self.want_direct = direct
        self.full_plan = None
        if direct is not False:
            self.full_plan = get_plan("1d", (self.n,), self.batch, prec, self.device)
            if direct is None and self.full_plan.launches != 1:
                self.full_plan = None
        self.plan = self.tail_plan = None
        self.dev_in = self.dev_out = None
        if streams is None:
            streams = tuple(torch.cuda.Stream(self.device) for _ in range(3))
        self.streams = tuple(streams)
        self.s_h2d, self.s_fft, self.s_d2h = self.streams
        self.last_mode = None

    def usable(self, t: torch.Tensor) -> bool:
        """True if the library's kernels can address t's storage directly."""
        with torch.cuda.device(self.device):
            rc = int(self.lib.fft_pointer_usable(ctypes.c_void_p(t.data_ptr()), t.numel() * t.element_size()))
        if rc < 0:
            raise L.GbfftError(rc, "fft_pointer_usable")
        return rc == 1

    def _copy_setup(self):
        if self.plan is not None:
            return
        self.plan = get_plan("1d", (self.n,), self.chunk, self.prec, self.device)
        tail = self.batch - (self.nchunks - 1) * self.chunk
        if tail != self.chunk:
            self.tail_plan = get_plan("1d", (self.n,), tail, self.prec, self.device)
        el = self.chunk * self.n
        self.dev_in = [torch.empty(el, dtype=torch.complex64, device=self.device) for _ in range(2)]
        self.dev_out = [torch.empty(el, dtype=torch.complex64, device=self.device) for _ in range(2)]

    def __call__(self, x_host: torch.Tensor, out_host: torch.Tensor, join: bool = True) -> torch.Tensor:
        """x_host, out_host: contiguous complex64 host tensors of batch*n
        elements (pin them for asynchronous copies or the direct mode).
        Returns out_host once the work is queued; synchronise the current
        stream before reading it.  join=False leaves the current stream
        unordered after the last step (the caller joins the download stream
        itself, e.g. after the last of several pipelines on shared streams)."""
        if x_host.is_cuda or out_host.is_cuda:
            raise TypeError("HostPipeline takes host tensors")
        if x_host.dtype != torch.complex64 or out_host.dtype != torch.complex64:
            raise TypeError("expected complex64 tensors")
        if x_host.numel() != self.batch * self.n or out_host.numel() != self.batch * self.n:
            raise ValueError("expected batch*n elements")
        xf, of = x_host.reshape(-1), out_host.reshape(-1)
        cur = torch.cuda.current_stream(self.device)
        direct = self.full_plan is not None and self.usable(xf) and self.usable(of)
        if self.want_direct and not direct:
            raise ValueError("direct mode needs page-locked host buffers the GPU can address")
        if direct:
            # one launch sequence on the transform stream; the download stream
            # (which join=False callers join) is ordered after it
            self.last_mode = "direct"
            self.s_fft.wait_stream(cur)
            self.full_plan.exec_ptr(xf.data_ptr(), of.data_ptr(), self.dir, self.s_fft)
            self.s_d2h.wait_stream(self.s_fft)
            if join:
                cur.wait_stream(self.s_d2h)
            return out_host
        self.last_mode = "copy"
        self._copy_setup()
        if self.nchunks == 1:
            # nothing to overlap: upload, transform and download in order on
            # the transform stream, with no cross-stream events
            m = self.batch * self.n
            s = self.s_fft
            s.wait_stream(cur)
            with torch.cuda.stream(s):
                self.dev_in[0][:m].copy_(xf, non_blocking=True)
                self.plan.exec_ptr(self.dev_in[0].data_ptr(), self.dev_out[0].data_ptr(), self.dir, s)
                of.copy_(self.dev_out[0][:m], non_blocking=True)
            self.s_d2h.wait_stream(s)
            if join:
                cur.wait_stream(self.s_d2h)
            return out_host
        for s in self.streams:
            s.wait_stream(cur)
        uploaded = [None, None]
        transformed = [None, None]
        downloaded = [None, None]
        for i in range(self.nchunks):
            b = i % 2
            lo = i * self.chunk * self.n
            m = min(self.chunk, self.batch - i * self.chunk) * self.n
            plan = self.plan if m == self.chunk * self.n else self.tail_plan
            with torch.cuda.stream(self.s_h2d):
                if transformed[b] is not None:
                    self.s_h2d.wait_event(transformed[b])      # dev_in[b] free again
                self.dev_in[b][:m].copy_(xf[lo:lo + m], non_blocking=True)
                uploaded[b] = torch.cuda.Event()
                uploaded[b].record(self.s_h2d)
            with torch.cuda.stream(self.s_fft):
                self.s_fft.wait_event(uploaded[b])
                if downloaded[b] is not None:
                    self.s_fft.wait_event(downloaded[b])       # dev_out[b] free again
                plan.exec_ptr(self.dev_in[b].data_ptr(), self.dev_out[b].data_ptr(), self.dir, self.s_fft)
                transformed[b] = torch.cuda.Event()
                transformed[b].record(self.s_fft)
            with torch.cuda.stream(self.s_d2h):
                self.s_d2h.wait_event(transformed[b])
                of[lo:lo + m].copy_(self.dev_out[b][:m], non_blocking=True)
                downloaded[b] = torch.cuda.Event()
                downloaded[b].record(self.s_d2h)
        if join:
            cur.wait_stream(self.s_d2h)
        return out_host


def fft_host(x_host: torch.Tensor, out_host: torch.Tensor | None = None, inverse: bool = False,
             chunk: int | None = None, direct: bool | None = None) -> torch.Tensor:
    """Eq. 1 (or Eq. 2) over the last dimension of a HOST complex64 tensor,
    through a HostPipeline (direct on page-locked buffers for one-pass plans,
    else pipelined copies).  Synchronous: returns when the result is in
    out_host."""
    n = x_host.shape[-1]
    batch = x_host.numel() // n
    if out_host is None:
        out_host = torch.empty(x_host.shape, dtype=x_host.dtype, pin_memory=torch.cuda.is_available())
    pipe = HostPipeline(n, batch, INVERSE if inverse else FORWARD, chunk=chunk, direct=direct)
    pipe(x_host.contiguous(), out_host)
    torch.cuda.synchronize(pipe.device)
    return out_host
