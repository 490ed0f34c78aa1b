"""Autotune cache: the fastest plan configuration per (GPU, n, batch, prec).

The search itself is native (fft_autotune in the library times every
candidate configuration with CUDA events); this module only stores its
answers in a JSON file so a shape is tuned once per GPU model.  The file is
$GBFFT_TUNE_CACHE, else ~/.cache/gbfft/tune.json; when a shape is missing
there, the results shipped with the package (tune_shipped.json, measured on
GB300) are used before tuning anew.

Uneven batches (fft_plan_create_many) are cached the same way, keyed by the
GPU model and a digest of the length list.

Command line (tunes shapes and writes them to a cache file):
    python -m paper_1707_07263_gb300.tune --out FILE [--many-uneven COUNT] n:batch [n:batch ...]
"""
from __future__ import annotations

import ctypes
import json
import os
import threading

import torch

from . import _lib as L

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("GBFFT_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "gbfft",
                                                                "tune.json")


SHIPPED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_shipped.json")


def _load(path: str | None = None) -> dict:
    try:
        with open(path or cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d: dict) -> None:
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def key(n: int, batch: int, prec: int, device) -> str:
    name = torch.cuda.get_device_name(device).replace(" ", "_")
    return f"{name}|n={n}|batch={batch}|prec={prec}"


def autotune(n: int, batch: int, prec: int = 0, device=None, iters: int = 10, stream=None) -> tuple[dict, float]:
    """Run the native search now on scratch buffers; returns (config, microseconds)."""
    lib = L.load()
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    x = torch.randn(n * batch, dtype=torch.complex64, device=dev)
    y = torch.empty_like(x)
    ws = torch.empty(n * batch * 8 + 256, dtype=torch.uint8, device=dev)
    wsp = (ws.data_ptr() + 255) & ~255
    best = L.FftPlanConfig()
    us = ctypes.c_float(0.0)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    rc = lib.fft_autotune(n, batch, prec, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                          ctypes.c_void_p(wsp), n * batch * 8, ctypes.c_void_p(s.cuda_stream), iters,
                          ctypes.byref(best), ctypes.byref(us))
    L.check(rc, "fft_autotune")
    return best.as_dict(), float(us.value)


def tuned_config(n: int, batch: int, prec: int = 0, device=None, retune: bool = False) -> dict:
    """Cached configuration for the shape, tuning it first if needed."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    k = key(n, batch, prec, dev)
    with _lock:
        cache = _load()
        if k in cache and not retune:
            return cache[k]["config"]
        shipped = _load(SHIPPED)
        if k in shipped and not retune:
            return shipped[k]["config"]
        cfg, us = autotune(n, batch, prec, dev)
        cache = _load()
        cache[k] = {"config": cfg, "us": us}
        _store(cache)
        return cfg


def many_key(lengths, device) -> str:
    """Cache key of an uneven batch: GPU model, count and a digest of the
    length multiset (the plan depends on the multiset and on the order)."""
    import hashlib
    name = torch.cuda.get_device_name(device).replace(" ", "_")
    h = hashlib.sha256(",".join(str(int(v)) for v in lengths).encode()).hexdigest()[:16]
    return f"{name}|many|count={len(lengths)}|lengths={h}"


def autotune_many(lengths, device=None, iters: int = 5, stream=None) -> tuple[dict, float]:
    """Run the native uneven-batch search now on scratch buffers."""
    lib = L.load()
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    lens = [int(v) for v in lengths]
    total = sum(lens)
    x = torch.randn(total, dtype=torch.complex64, device=dev)
    y = torch.empty_like(x)
    ws = torch.empty(total * 8 + 256, dtype=torch.uint8, device=dev)
    wsp = (ws.data_ptr() + 255) & ~255
    arr = (ctypes.c_int64 * len(lens))(*lens)
    best = L.FftManyConfig()
    us = ctypes.c_float(0.0)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    rc = lib.fft_autotune_many(arr, len(lens), 0, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                               ctypes.c_void_p(wsp), total * 8, ctypes.c_void_p(s.cuda_stream), iters,
                               ctypes.byref(best), ctypes.byref(us))
    L.check(rc, "fft_autotune_many")
    return best.as_dict(), float(us.value)


def tuned_many_config(lengths, device=None, retune: bool = False) -> dict:
    """Cached configuration for an uneven batch, tuning it first if needed."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    k = many_key(lengths, dev)
    with _lock:
        cache = _load()
        if k in cache and not retune:
            return cache[k]["config"]
        shipped = _load(SHIPPED)
        if k in shipped and not retune:
            return shipped[k]["config"]
        cfg, us = autotune_many(lengths, dev)
        cache = _load()
        cache[k] = {"config": cfg, "us": us}
        _store(cache)
        return cfg


def main(argv=None) -> None:
    import argparse
    ap = argparse.ArgumentParser(description="tune plan configurations and store them")
    ap.add_argument("--out", required=True, help="cache file to write (merged with its contents)")
    ap.add_argument("--iters", type=int, default=10)
    ap.add_argument("--many-uneven", type=int, default=0,
                    help="also tune the uneven batch of this many lengths 2^8..2^16 drawn like the benchmark's")
    ap.add_argument("shapes", nargs="*", help="n:batch pairs")
    args = ap.parse_args(argv)
    dev = torch.device("cuda", torch.cuda.current_device())
    out = _load(args.out)
    if args.many_uneven:
        from . import workloads
        lengths = workloads.uneven_lengths(args.many_uneven, seed=workloads.seed_for(4)).tolist()
        cfg, us = autotune_many(lengths, dev)
        out[many_key(lengths, dev)] = {"config": cfg, "us": us}
        print(f"many {args.many_uneven}: {cfg} {us:.1f} us", flush=True)
    for sh in args.shapes:
        n, b = (int(v) for v in sh.split(":"))
        cfg, us = autotune(n, b, 0, dev, iters=args.iters)
        out[key(n, b, 0, dev)] = {"config": cfg, "us": us}
        print(f"{sh}: {cfg} {us:.1f} us", flush=True)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
