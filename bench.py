"""Benchmark: batched 1-D complex64 FFTs on GB300 through libgbfft.

Default workload (one "step"): for each N in {2^10, 2^12, 2^14}, a forward and
an inverse transform of batch = 2^26 / N transforms (2^26 complex64 points,
512 MiB per direction, larger than the 126 MB L2, so no L2 flush is needed
between launches), inputs CN(0,1) from a fixed seed.  Metric: GFLOP/s with
the conventional 5 N log2 N flops per complex transform.

Also printed on the same JSON line:
  roofline      the dominant kernel's algorithmic HBM bytes (16 B per point:
                one complex64 read + one write) / its CUDA-event launch time,
                against the measured copy bandwidth;
  cpu_baseline  the FP64 oracle (test infrastructure) timed on the host cores
                on a bounded sample of the same workload;
  e2e           the same metric through the public API (HostPipeline) on
                page-locked HOST buffers, every step's data crossing the host
                link both ways inside the timed region: the copy-engine
                pipeline (uploads, transforms and downloads overlapped on
                three streams), with the direct mode (kernels reading and
                writing the host buffers) and the link's own ceiling
                (concurrent copies up and down) beside it;
  clocks        nvidia-smi samples taken during the timed region;
  cfg1_latency, cfg3_large, cfg4_precision, cfg5_uneven
                per-size results of the other configurations, measured on
                the same GPU after the timed step (not part of it): time,
                GFLOP/s, the algorithmic HBM fraction (16 B per point
                whatever the pass count) beside the per-launch one, sampled
                oracle errors, and whether the 70 % target at 2^20 and the
                split-tensor-core-beats-FP32 target are met.

``--impl reference`` times the oracle instead (the deliberately slow CPU
baseline) and prints the same line with "impl": "reference".
Other workloads for measurement only: --workload large | tc | many | range | real | mixed | fp64 |
passes | radix.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

TOTAL = 1 << 26
HBM_FALLBACK = 6800.0
METRIC = "GFLOP/s (5N log2N) and % of HBM roofline per FFT size; split-TC vs plain FP32 at stated err"


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", HBM_FALLBACK)), "measured"
    return HBM_FALLBACK, "fallback"


# The sources the benchmark's kernels are compiled from (the single-pass
# register, prefetching and TMA-staged kernels and what they include).  The
# DRAM traffic recorded in profiles/traffic.json is valid only while these
# files are unchanged.
BENCH_KERNEL_SOURCES = ("fft_common.cuh", "tile_fft.cuh", "tile_fft_tma.cuh", "tma_util.cuh", "tile_registry.h",
                        "tile_inst_jj.cu", "tile_inst_pf.cu", "tile_inst_tma.cu")


def source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1707_07263_gb300", "csrc")
    for name in BENCH_KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def single_kernel_name(lib, h) -> str:
    """The kernel a one-launch plan runs, from its configuration."""
    from paper_1707_07263_gb300 import _lib
    c = _lib.FftPlanConfig()
    _lib.check(lib.fft_plan_get_config(h, ctypes.byref(c)))
    if c.halves == 2:
        return "tile_fft_dif2_kernel"
    return {1: "tile_fft_tma_kernel", 2: "tile_fft_pf_kernel", 3: "tile_fft_pfs_kernel"}.get(c.tma, "tile_fft_kernel")


def ncu_traffic(kernel_key: str):
    """DRAM bytes per launch of `kernel_key` from the committed ncu summary, or
    None when the kernels changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("source_hash") != source_hash():
        return None
    e = d.get("kernels", {}).get(kernel_key)
    return None if e is None else float(e["dram_bytes_per_launch"])


def smi_gpu_id(local: int) -> str:
    """nvidia-smi's name for CUDA device `local`: its UUID (indices differ
    from CUDA's when CUDA_VISIBLE_DEVICES remaps devices), else the index."""
    try:
        import torch
        u = str(torch.cuda.get_device_properties(local).uuid)
        if u:
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        pass
    return str(local)


class ClockSampler:
    """nvidia-smi samples during the timed region (clocks and throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: str):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.lines:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(value: float, dist, device) -> float:
    """The largest of every rank's value (the job takes as long as its
    slowest rank); the value itself without a process group."""
    if not dist:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl != "reference" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


# ------------------------------------------------------------------------------------
# workloads
# ------------------------------------------------------------------------------------
def workload_cfg2():
    """(name, list of (label, n, batch, dir)) for the default step."""
    items = []
    for lg in (10, 12, 14):
        n = 1 << lg
        items.append((f"fwd_2^{lg}", n, TOTAL // n, 0))
        items.append((f"inv_2^{lg}", n, TOTAL // n, 1))
    desc = ("batched 1D complex64 FFT, N in {2^10, 2^12, 2^14}, batch = 2^26/N, CN(0,1) inputs, "
            "forward + inverse per size (single-kernel on-chip path, FP32)")
    return desc, items


def workload_large():
    items = [("fwd_2^24", 1 << 24, 1, 0), ("fwd_2^26", 1 << 26, 1, 0)]
    return "1D complex64 FFT via the four-step split, N = 2^24 and 2^26, batch 1, U[-1,1]", items


def _describe(lib, h) -> str:
    buf = ctypes.create_string_buffer(512)
    lib.fft_plan_describe(h, buf, 512)
    return buf.value.decode()


def flops(n, batch):
    return 5.0 * n * np.log2(n) * batch


# ------------------------------------------------------------------------------------
# CPU baseline (oracle)
# ------------------------------------------------------------------------------------
def oracle_sample(items, budget_s: float):
    """Time the FP64 oracle on a bounded sample: for each (n, dir) item, as many
    whole transforms as fit the per-item share of the budget (at least one)."""
    import oracle
    from paper_1707_07263_gb300 import workloads
    oracle.build()
    share = budget_s / max(1, len(items))
    total_flop, total_t, desc = 0.0, 0.0, []
    for label, n, batch, d in items:
        x = workloads.cgauss(n, 1, seed=7).astype(np.complex128)
        rows, t = 0, 0.0
        while rows < batch and (t < share or rows == 0):
            t0 = time.perf_counter()
            oracle.fft(x, oracle.FORWARD if d == 0 else oracle.INVERSE)
            t += time.perf_counter() - t0
            rows += 1
        total_flop += flops(n, rows)
        total_t += t
        desc.append(f"{rows}x{label}")
    return total_flop / total_t / 1e9, ", ".join(desc), total_t


def oracle_sample_all_cores(items, budget_s: float):
    """The same oracle on every host core, one thread per transform (the
    C oracle runs with the GIL released), for about budget_s seconds of wall
    time.  Returns (GFLOP/s, threads, sample description)."""
    import concurrent.futures
    import oracle
    from paper_1707_07263_gb300 import workloads
    oracle.build()
    threads = os.cpu_count() or 1
    xs = {n: workloads.cgauss(n, 1, seed=7).astype(np.complex128) for _, n, _, _ in items}
    share = budget_s / max(1, len(items))
    total_flop, total_t, desc = 0.0, 0.0, []
    for label, n, batch, d in items:
        direction = oracle.FORWARD if d == 0 else oracle.INVERSE
        t0 = time.perf_counter()
        oracle.fft(xs[n], direction)
        t1 = max(time.perf_counter() - t0, 1e-6)
        # every thread loops over its own transforms, so that the wall time
        # measures the C oracle rather than task dispatch
        per_thread = max(1, min(batch // threads, int(share / t1)))

        def work(_):
            for _ in range(per_thread):
                oracle.fft(xs[n], direction)

        with concurrent.futures.ThreadPoolExecutor(max_workers=threads) as ex:
            t0 = time.perf_counter()
            list(ex.map(work, range(threads)))
            t = time.perf_counter() - t0
        rows = per_thread * threads
        total_flop += flops(n, rows)
        total_t += t
        desc.append(f"{rows}x{label}")
    return total_flop / total_t / 1e9, threads, ", ".join(desc)


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


# ------------------------------------------------------------------------------------
# the other configurations, measured beside the headline (not part of its step)
# ------------------------------------------------------------------------------------
def measure_other_configs(torch, lib, dev, stream, peak, iters, warmup):
    """Per-size results of the other configurations on the same GPU, outside
    the headline's timed region: CUDA events on `stream`, `warmup` untimed and
    `iters` timed executions, data resident in HBM, inputs larger than L2
    where the configuration's size allows.  hbm_frac_algorithmic counts the
    algorithmic 16 bytes per point (one complex64 read and one write) however
    many passes the plan makes; hbm_frac_per_launch counts them once per
    launch.  Errors are relative L2 against the FP64 oracle on sampled rows."""
    import oracle
    from paper_1707_07263_gb300 import _lib, api, tune, workloads
    sh = ctypes.c_void_p(stream.cuda_stream)
    out = {}

    def make(n, batch, prec=0, tuned=True, two_d=None):
        if two_d:
            h = lib.fft_plan_create_2d(two_d[0], two_d[1], 1, 0, 0)
        elif tuned and prec == 0:
            c = _lib.FftPlanConfig.from_dict(tune.tuned_config(n, batch, 0, dev))
            h = lib.fft_plan_create_config(n, batch, 0, 0, ctypes.byref(c))
        else:
            h = lib.fft_plan_create(n, batch, 0, prec)
        if not h:
            return None, None
        h = ctypes.c_void_p(h)
        ws = lib.fft_plan_workspace_bytes(h)
        wsb = torch.empty(ws, dtype=torch.uint8, device=dev) if ws else None
        if ws:
            _lib.check(lib.fft_plan_set_workspace(h, ctypes.c_void_p(wsb.data_ptr())))
        return h, wsb

    def timed(h, x, y, d=0, n_iter=iters):
        def one():
            _lib.check(lib.fft_exec_dir(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), d, sh))
        return _time_fn(torch, one, n_iter, warmup, stream)

    def entry(n_points, lg_sum, ms, launches):
        gbs = 16.0 * n_points / (ms * 1e-3) / 1e9
        return {"us": round(ms * 1e3, 2), "gflops": round(5.0 * n_points * lg_sum / (ms * 1e-3) / 1e9, 1),
                "hbm_gbs_algorithmic": round(gbs, 1), "hbm_frac_algorithmic": round(gbs / peak, 4),
                "hbm_frac_per_launch": round(gbs * launches / peak, 4), "launches": launches}

    # cfg1: one 4096-point transform (latency, not bandwidth)
    n = 4096
    x1 = torch.from_numpy(workloads.uniform(n, 1, workloads.seed_for(0)).reshape(-1)).to(dev)
    y1 = torch.empty_like(x1)
    h, _ = make(n, 1)
    ms = timed(h, x1, y1, 0, max(200, iters))
    ref = oracle.dft(x1.cpu().numpy().astype(np.complex128))
    out["cfg1_latency"] = {"n": n, "batch": 1, "us_per_transform": round(ms * 1e3, 2),
                           "gflops": round(flops(n, 1) / (ms * 1e-3) / 1e9, 2),
                           "rel_l2": float(f"{oracle.rel_l2(y1.cpu().numpy(), ref):.3e}"),
                           "note": "one CTA: launch-latency bound, roofline fraction not meaningful"}
    lib.fft_destroy(h)

    # cfg3: four-step 1-D (U[-1,1]) and the 8192 x 8192 SAR image
    xu = torch.from_numpy(workloads.uniform(TOTAL, 1, workloads.seed_for(2)).reshape(-1)).to(dev)
    y = torch.empty_like(xu)
    res3 = {}
    for lg, batch in ((20, 64), (24, 4), (26, 1)):
        nn = 1 << lg
        h, wsb = make(nn, batch)
        ms = timed(h, xu, y)
        res3[f"2^{lg}x{batch}"] = entry(TOTAL, lg, ms, lib.fft_plan_launches(h))
        lib.fft_destroy(h)
        del wsb
    del xu
    img = torch.from_numpy(workloads.sar_image(8192, 8192, seed=workloads.seed_for(2, 1)).reshape(-1)).to(dev)
    h, wsb = make(0, 1, two_d=(8192, 8192))
    ms = timed(h, img, y)
    res3["8192x8192"] = entry(TOTAL, 26, ms, lib.fft_plan_launches(h))
    lib.fft_destroy(h)
    del wsb, img
    f20 = res3["2^20x64"]["hbm_frac_algorithmic"]
    out["cfg3_large"] = {"sizes": res3,
                         "target_70pct_hbm_at_2p20": {"hbm_frac_algorithmic": f20, "met": bool(f20 >= 0.70)}}

    # cfg4: FP32 against the tensor-core radix-16 variants, CN(0,1)
    precs = [("fp32", 0), ("tc_bf16", 1), ("tc_fp16", 2), ("tc_bf16_split", 3), ("tc_fp16_split", 4)]
    res4 = {}
    for lg in (12, 16, 20):
        nn = 1 << lg
        batch = TOTAL // nn
        xh = workloads.cgauss(nn, batch, seed=workloads.seed_for(3) + lg)
        x = torch.from_numpy(xh.reshape(-1)).to(dev)
        rows = 2
        ref = oracle.fft(xh[:rows].astype(np.complex128))
        del xh
        for name, pc in precs:
            h, wsb = make(nn, batch, pc)
            if h is None:
                res4[f"2^{lg}/{name}"] = {"unsupported": True}
                continue
            ms = timed(h, x, y)
            e = entry(TOTAL, lg, ms, lib.fft_plan_launches(h))
            got = y[: rows * nn].cpu().numpy().reshape(rows, nn)
            e["rel_l2_max_sampled"] = float(f"{float(oracle.rel_l2_rows(got, ref).max()):.3e}")
            res4[f"2^{lg}/{name}"] = e
            lib.fft_destroy(h)
            del wsb
        del x
    best = {}
    for lg in (12, 16, 20):
        t32 = res4[f"2^{lg}/fp32"]["us"]
        split = [(res4[f"2^{lg}/{k}"]["us"], k) for k in ("tc_fp16_split", "tc_bf16_split")
                 if "us" in res4.get(f"2^{lg}/{k}", {}) and res4[f"2^{lg}/{k}"]["rel_l2_max_sampled"] <= 1e-5]
        best[f"2^{lg}"] = {"fp32_us": t32, "best_split_us": min(split)[0] if split else None,
                           "split_faster_at_1e-5": bool(split and min(split)[0] < t32)}
    out["cfg4_precision"] = {"variants": res4, "split_tc_vs_fp32": best}

    # cfg5: 4096 uneven lengths, forward and the graph-captured gradient step
    lengths = workloads.uneven_lengths(4096, seed=workloads.seed_for(4)).tolist()
    total = int(sum(lengths))
    xh = workloads.packed_cgauss(lengths, seed=workloads.seed_for(4, 2))
    wh = workloads.real_weights(total, seed=workloads.seed_for(4, 1))
    x = torch.from_numpy(xh).to(dev)
    w2 = torch.from_numpy(2.0 * wh.astype(np.float32) ** 2).to(dev)
    mcfg = tune.tuned_many_config(lengths, dev)   # the autotuner's configuration (shipped or cached)
    pm = api.Plan("many", (total,), len(lengths), 0, "fp32", dev, lengths=lengths, config=mcfg)
    X, G, gx = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x)

    def step():
        pm.exec_ptr(x.data_ptr(), X.data_ptr(), 0, stream)
        torch.mul(X, w2, out=G)
        pm.exec_ptr(G.data_ptr(), gx.data_ptr(), 2, stream)

    with torch.cuda.stream(stream):
        step()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        step()
    ms_step = _time_fn(torch, g.replay, iters, warmup, stream)
    ms_fwd = _time_fn(torch, lambda: pm.exec_ptr(x.data_ptr(), X.data_ptr(), 0, stream), iters, warmup, stream)
    pd = api.Plan("many", (total,), len(lengths), 0, "fp32", dev, lengths=lengths)   # planner defaults
    ms_fwd_default = _time_fn(torch, lambda: pd.exec_ptr(x.data_ptr(), G.data_ptr(), 0, stream), iters, warmup,
                              stream)
    default_cfg = pd.many_config()
    pd.close()
    fl = sum(flops(nn, 1) for nn in lengths)
    gxh = gx.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum(lengths)])
    errs = [oracle.rel_l2(gxh[offs[i]:offs[i + 1]],
                          oracle.spectral_loss_grad(xh[offs[i]:offs[i + 1]].astype(np.complex128),
                                                    wh[offs[i]:offs[i + 1]].astype(np.float64)))
            for i in range(0, len(lengths), 97)]
    gbs = 16.0 * total / (ms_fwd * 1e-3) / 1e9
    out["cfg5_uneven"] = {"transforms": len(lengths), "points": total, "forward_us": round(ms_fwd * 1e3, 1),
                          "gflops_fwd": round(fl / (ms_fwd * 1e-3) / 1e9, 1),
                          "hbm_frac_algorithmic_fwd": round(gbs / peak, 4),
                          "graph_step_us": round(ms_step * 1e3, 1),
                          "gflops_fwd_plus_bwd": round(2 * fl / (ms_step * 1e-3) / 1e9, 1),
                          "grad_rel_l2_max_sampled": float(f"{max(errs):.3e}"), "grad_samples": len(errs),
                          "step": "graph-captured: forward (one launch), 2 w^2 X (torch), adjoint (one launch)",
                          "plan_config": pm.many_config(),
                          "forward_us_planner_default": round(ms_fwd_default * 1e3, 1),
                          "planner_default_config": default_cfg}
    pm.close()
    return out


# ------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------
def run_gpu(args):
    import torch
    from paper_1707_07263_gb300 import _lib
    from paper_1707_07263_gb300 import workloads

    world, rank, local, dist = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = _lib.load()

    if args.workload == "cfg2":
        desc, items = workload_cfg2()
    elif args.workload == "large":
        desc, items = workload_large()
    else:
        raise SystemExit(f"unknown workload {args.workload}")

    stream = torch.cuda.Stream(device=dev)
    sh = ctypes.c_void_p(stream.cuda_stream)

    # one plan per (n, batch); inputs resident in HBM before timing
    plans, bufs = {}, {}
    tuned = {}
    for label, n, batch, d in items:
        key = (n, batch)
        if key not in plans:
            if args.tuned:
                # autotuner (native search, cached per GPU model); untimed set-up
                from paper_1707_07263_gb300 import tune
                cfg = tune.tuned_config(n, batch, 0, dev)
                tuned[f"2^{int(np.log2(n))}"] = cfg
                c = _lib.FftPlanConfig.from_dict(cfg)
                h = lib.fft_plan_create_config(n, batch, 0, 0, ctypes.byref(c))
            else:
                h = lib.fft_plan_create(n, batch, 0, 0)
            if not h:
                raise RuntimeError(f"plan {n}x{batch}: {_lib.ERRORS.get(lib.fft_last_error())}")
            h = ctypes.c_void_p(h)
            ws = lib.fft_plan_workspace_bytes(h)
            wsbuf = torch.empty(ws, dtype=torch.uint8, device=dev) if ws else None
            if ws:
                _lib.check(lib.fft_plan_set_workspace(h, ctypes.c_void_p(wsbuf.data_ptr())))
            plans[key] = (h, wsbuf)
    maxel = max(n * b for _, n, b, _ in items)
    x_host = workloads.cgauss(maxel, 1, seed=workloads.seed_for(1) + rank).reshape(-1)
    xin = torch.from_numpy(x_host).to(dev)
    xout = torch.empty_like(xin)
    launches_per_step = sum(lib.fft_plan_launches(plans[(n, b)][0]) for _, n, b, _ in items)

    def exec_item(i, src, dst):
        label, n, batch, d = items[i]
        rc = lib.fft_exec_dir(plans[(n, batch)][0], ctypes.c_void_p(src.data_ptr()),
                              ctypes.c_void_p(dst.data_ptr()), d, sh)
        if rc:
            raise RuntimeError(f"exec {label}: {_lib.ERRORS.get(rc)}")

    def one_step(ev=None):
        for i in range(len(items)):
            if ev is not None:
                ev[i][0].record(stream)
            exec_item(i, xin, xout)
            if ev is not None:
                ev[i][1].record(stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_step()
    torch.cuda.synchronize()

    K = args.steps
    evs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in items]
           for _ in range(K)]
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(smi_gpu_id(local)) as clk:
        t0e.record(stream)
        with torch.cuda.stream(stream):
            for k in range(K):
                one_step(evs[k])
        t1e.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms_total = t0e.elapsed_time(t1e)
    per_item_ms = [float(np.mean([evs[k][i][0].elapsed_time(evs[k][i][1]) for k in range(K)]))
                   for i in range(len(items))]
    ms_total = max_over_ranks(ms_total, dist, dev)
    ms_step = ms_total / K
    step_flop = sum(flops(n, b) for _, n, b, _ in items)
    value = step_flop * world / (ms_step * 1e-3) / 1e9

    # ---- roofline of the dominant kernel ----
    peak, peak_kind = measured_peaks()
    dom = int(np.argmax(per_item_ms))
    label, n, batch, d = items[dom]
    nl = lib.fft_plan_launches(plans[(n, batch)][0])
    # each launch of every plan kind reads and writes the whole array once
    bytes_launch = 16.0 * n * batch
    # average per-launch duration of the dominant plan's kernels
    achieved = bytes_launch / (per_item_ms[dom] / nl * 1e-3) / 1e9
    lg = int(np.log2(n))
    kname = single_kernel_name(lib, plans[(n, batch)][0]) if nl == 1 else "multi-pass"
    traffic = ncu_traffic(f"{kname}_lg{lg}") if nl == 1 else None
    per_size = {}
    for i, (lab, nn, bb, dd) in enumerate(items):
        gbs = 16.0 * nn * bb / (per_item_ms[i] * 1e-3) / 1e9
        per_size[lab] = {"us": round(per_item_ms[i] * 1e3, 2),
                         "gflops": round(flops(nn, bb) / (per_item_ms[i] * 1e-3) / 1e9, 1),
                         "hbm_gbs": round(gbs, 1), "hbm_frac": round(gbs / peak, 4)}

    # ---- the other configurations (per size, outside the timed step) ----
    others = {}
    if rank == 0 and not args.no_extra:
        others = measure_other_configs(torch, lib, dev, stream, peak, max(10, K // 2), args.warmup)

    # ---- end to end through the public API with pinned host buffers ----
    e2e = None
    if not args.no_e2e:
        from paper_1707_07263_gb300 import api
        host_in = torch.from_numpy(x_host).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        h2d = d2h = 0

        def time_e2e(direct):
            """One pipeline per (length, direction), sharing three streams so
            that successive items overlap; direct=None is the API default
            (kernels on the page-locked buffers for one-pass lengths), False
            the copy-engine pipeline."""
            nonlocal h2d, d2h
            pipes = []
            streams = None
            for lab, nn, bb, dd in items:
                pp = api.HostPipeline(nn, bb, dd, device=dev, streams=streams, direct=direct)
                streams = pp.streams
                pipes.append(pp)

            def e2e_step():
                nonlocal h2d, d2h
                h2d = d2h = 0
                with torch.cuda.stream(stream):
                    for i, (lab, nn, bb, dd) in enumerate(items):
                        m = nn * bb
                        pipes[i](host_in[:m], host_out[:m], join=(i == len(items) - 1))
                        h2d += m * 8
                        d2h += m * 8

            for _ in range(max(1, min(args.warmup, 2))):
                e2e_step()
            torch.cuda.synchronize()
            ke = max(1, min(K, 5))
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for _ in range(ke):
                e2e_step()
            a1.record(stream)
            torch.cuda.synchronize()
            ms = max_over_ranks(a0.elapsed_time(a1) / ke, dist, dev)
            return ms, sorted({pp.last_mode for pp in pipes})

        # streaming calls on shared streams: the copy pipeline overlaps the
        # next item's upload with this one's download and is the faster mode
        e_ms, modes = time_e2e(False)
        d_ms, dmodes = time_e2e(None)

        # the host link's own ceiling: the copy engines moving the same bytes
        # up and down at once (one 512 MiB buffer each way, two streams)
        dscratch = torch.empty_like(xin)
        su, sd = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        nbytes = xin.numel() * 8

        def link_copy():
            for s_ in (su, sd):
                s_.wait_stream(stream)
            with torch.cuda.stream(su):
                dscratch.copy_(host_in, non_blocking=True)
            with torch.cuda.stream(sd):
                host_out.copy_(xin, non_blocking=True)
            stream.wait_stream(su)
            stream.wait_stream(sd)

        with torch.cuda.stream(stream):
            link_copy()
            torch.cuda.synchronize()
            l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            l0.record(stream)
            for _ in range(3):
                link_copy()
            l1.record(stream)
            torch.cuda.synchronize()
        link_peak = 2 * nbytes / (l0.elapsed_time(l1) / 3 * 1e-3) / 1e9
        del dscratch
        link_gbs = (h2d + d2h) / (e_ms * 1e-3) / 1e9
        e2e = {"value": round(step_flop * world / (e_ms * 1e-3) / 1e9, 2), "unit": "GFLOP/s",
               "ms_per_step": round(e_ms, 3), "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "api": "paper_1707_07263_gb300.api.HostPipeline(direct=False) -> fft_exec_dir, page-locked host "
                      "tensors, 64 MiB chunks, upload/transform/download on three shared streams",
               "modes": modes,
               "host_link": {"achieved_gbs": round(link_gbs, 1), "copy_engine_peak_gbs": round(link_peak, 1),
                             "frac": round(link_gbs / link_peak, 4),
                             "peak_source": "measured live: concurrent 512 MiB H2D + D2H copies"},
               "direct": {"value": round(step_flop * world / (d_ms * 1e-3) / 1e9, 2),
                          "ms_per_step": round(d_ms, 3), "modes": dmodes,
                          "mode": "HostPipeline default: kernels read and write the page-locked host tensors"}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, sample, secs = oracle_sample(items, args.cpu_budget)
        cpu = {"value": round(v, 4), "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
               "sample": f"FP64 recursive radix-2 oracle, 1 thread, {sample} ({secs:.1f} s)",
               "cpu_model": cpu_model(), "cpu_count": os.cpu_count()}
        va, thr, sample_a = oracle_sample_all_cores(items, args.cpu_budget / 2)
        cpu["all_cores"] = {"value": round(va, 4), "unit": "GFLOP/s", "threads": thr,
                            "sample": f"one transform per thread, {sample_a}"}

    line = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "GFLOP/s",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": desc, "points_per_transform_batch": TOTAL, "sizes": [n for _, n, _, _ in items],
                   "l2": "inputs and outputs (512 MiB each) larger than L2; no flush",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "frac_of_nominal_7900": round(achieved / 7900.0, 4),
                     "hbm_passes": round(traffic / bytes_launch, 3) if traffic else None,
                     "kernel": f"{kname} (L=2^{lg}, {label})",
                     "algorithmic_bytes_per_launch": bytes_launch,
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback"},
        "per_size": per_size,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk.summary(),
        "gpu_launches": int(launches_per_step * K),
        "plans": {f"2^{int(np.log2(n))}": _describe(lib, plans[(n, b)][0]) for _, n, b, _ in items},
        "autotuned": tuned if args.tuned else None,
    }
    line.update(others)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ------------------------------------------------------------------------------------
def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    desc, items = workload_cfg2() if args.workload == "cfg2" else workload_large()
    import oracle
    from paper_1707_07263_gb300 import workloads
    oracle.build()
    # one step = one transform of each (size, direction) item: a bounded sample
    xs = {n: workloads.cgauss(n, 1, seed=workloads.seed_for(1)).astype(np.complex128) for _, n, _, _ in items}

    def step():
        for _, n, _, d in items:
            oracle.fft(xs[n], oracle.FORWARD if d == 0 else oracle.INVERSE)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    secs = time.perf_counter() - t0
    step_flop = sum(flops(n, 1) for _, n, _, _ in items)
    ms = secs / args.steps * 1e3
    v = step_flop / (ms * 1e-3) / 1e9
    sample = "one transform per (size, direction) per step: " + ", ".join(l for l, _, _, _ in items)
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "sizes": [n for _, n, _, _ in items]},
            "cpu_baseline": {"value": round(v, 4), "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(v, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_case(args):
    """One plan (2^lg points, batch 2^26/2^lg unless --batch) run warmup + iters
    times: the small, self-contained case used for ncu captures."""
    import torch
    from paper_1707_07263_gb300 import _lib
    lib = _lib.load()
    n = args.case_n or (1 << args.case)
    fp64 = args.prec == _lib.FFT_PREC_FP64
    batch = args.batch or max(1, (TOTAL // 2 if fp64 else TOTAL) // n)
    if args.real:
        h = lib.fft_plan_create_r2c(n, batch, args.prec)
    elif args.tma >= 0:
        c = _lib.FftPlanConfig.from_dict({"tma": args.tma})
        h = lib.fft_plan_create_config(n, batch, args.dir, args.prec, ctypes.byref(c))
    else:
        h = lib.fft_plan_create(n, batch, args.dir, args.prec)
    if not h:
        raise RuntimeError(_lib.ERRORS.get(lib.fft_last_error()))
    h = ctypes.c_void_p(h)
    ws = lib.fft_plan_workspace_bytes(h)
    wsb = torch.empty(ws, dtype=torch.uint8, device="cuda") if ws else None
    if ws:
        _lib.check(lib.fft_plan_set_workspace(h, ctypes.c_void_p(wsb.data_ptr())))
    if args.real:
        # real rows of n floats and rows of n/2 + 1 complex values; --dir picks the direction
        xr = torch.randn(n * batch, dtype=torch.float32, device="cuda")
        xc = torch.randn((n // 2 + 1) * batch, dtype=torch.complex64, device="cuda")
        x, y = (xr, xc) if args.dir == 0 else (xc, xr)
    else:
        x = torch.randn(n * batch, dtype=torch.complex128 if fp64 else torch.complex64, device="cuda")
        y = torch.empty_like(x)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if args.real:
        def one():
            _lib.check(lib.fft_exec_dir(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), args.dir, s))
    elif args.filter:
        # range compression with a random filter (fft_exec_filter)
        H = torch.randn(n, dtype=torch.complex64, device="cuda")

        def one():
            _lib.check(lib.fft_exec_filter(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                           ctypes.c_void_p(H.data_ptr()), s))
    else:
        def one():
            _lib.check(lib.fft_exec(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), s))
    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        one()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    buf = ctypes.create_string_buffer(512)
    lib.fft_plan_describe(h, buf, 512)
    # algorithmic bytes per transform: one read and one write of every value
    bytes_pt = (4.0 * n + 8.0 * (n // 2 + 1)) if args.real else (32.0 if fp64 else 16.0) * n
    print(json.dumps({"case": f"{n} x {batch}", "us": round(ms * 1e3, 2),
                      "hbm_gbs_per_launch": round(bytes_pt * batch * lib.fft_plan_launches(h) / (ms * 1e-3) / 1e9, 1),
                      "plan": buf.value.decode()}))
    lib.fft_destroy(h)


# ------------------------------------------------------------------------------------
# measurement-only workloads (not the contract line): tc, large, many
# ------------------------------------------------------------------------------------
def _time_fn(torch, fn, iters, warmup, stream):
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(iters):
            fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / iters


def run_measure(args):
    import torch
    import oracle
    from paper_1707_07263_gb300 import _lib, api, workloads
    lib = _lib.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream()
    sh = ctypes.c_void_p(stream.cuda_stream)
    peak, _ = measured_peaks()
    res = []

    def plan(n, batch, prec):
        h = lib.fft_plan_create(n, batch, 0, prec)
        if not h:
            return None, None
        h = ctypes.c_void_p(h)
        ws = lib.fft_plan_workspace_bytes(h)
        wsb = torch.empty(max(ws, 1), dtype=torch.uint8, device=dev)
        if ws:
            _lib.check(lib.fft_plan_set_workspace(h, ctypes.c_void_p(wsb.data_ptr())))
        return h, wsb

    def run_plan(h, x, y, d=0):
        _lib.check(lib.fft_exec_dir(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), d, sh))

    if args.workload == "tc":
        precs = [("fp32", 0), ("tc_bf16", 1), ("tc_fp16", 2), ("tc_bf16_split", 3), ("tc_fp16_split", 4)]
        for lg in (12, 16, 20):
            n = 1 << lg
            batch = TOTAL // n
            xh = workloads.cgauss(n, batch, seed=workloads.seed_for(3) + lg)
            x = torch.from_numpy(xh.reshape(-1)).to(dev)
            y = torch.empty_like(x)
            rows = 2
            ref = oracle.fft(xh[:rows].astype(np.complex128))
            for name, pc in precs:
                h, wsb = plan(n, batch, pc)
                if h is None:
                    res.append({"n": n, "prec": name, "unsupported": True})
                    continue
                ms = _time_fn(torch, lambda: run_plan(h, x, y), args.steps, args.warmup, stream)
                got = y[: rows * n].cpu().numpy().reshape(rows, n)
                err = float(oracle.rel_l2_rows(got, ref).max())
                nl = lib.fft_plan_launches(h)
                res.append({"n": n, "batch": batch, "prec": name, "us": round(ms * 1e3, 1),
                            "gflops": round(flops(n, batch) / (ms * 1e-3) / 1e9, 1),
                            "hbm_gbs_per_launch": round(16.0 * n * batch * nl / (ms * 1e-3) / 1e9, 1),
                            "hbm_frac_per_launch": round(16.0 * n * batch * nl / (ms * 1e-3) / 1e9 / peak, 4),
                            "launches": nl, "rel_l2_max": float(f"{err:.3e}")})
                lib.fft_destroy(h)
        desc = "precision variants: batched N in {2^12, 2^16, 2^20}, batch 2^26/N, CN(0,1); FP32 vs TC radix-16"
    elif args.workload == "large":
        x = torch.from_numpy(workloads.uniform(1 << 26, 1, workloads.seed_for(2)).reshape(-1)).to(dev)
        y = torch.empty_like(x)
        for lg in (20, 22, 24, 26):
            n = 1 << lg
            batch = TOTAL // n
            h, wsb = plan(n, batch, 0)
            ms = _time_fn(torch, lambda: run_plan(h, x, y), args.steps, args.warmup, stream)
            buf = ctypes.create_string_buffer(512)
            lib.fft_plan_describe(h, buf, 512)
            nl = lib.fft_plan_launches(h)
            res.append({"n": n, "batch": batch, "us": round(ms * 1e3, 1),
                        "gflops": round(flops(n, batch) / (ms * 1e-3) / 1e9, 1),
                        "hbm_frac_algorithmic": round(16.0 * n * batch / (ms * 1e-3) / 1e9 / peak, 4),
                        "hbm_frac_per_launch": round(16.0 * n * batch * nl / (ms * 1e-3) / 1e9 / peak, 4),
                        "plan": buf.value.decode()})
            lib.fft_destroy(h)
        img = torch.from_numpy(workloads.sar_image(8192, 8192, seed=workloads.seed_for(2, 1)).reshape(-1)).to(dev)
        h2 = ctypes.c_void_p(lib.fft_plan_create_2d(8192, 8192, 1, 0, 0))
        ws2 = torch.empty(max(1, lib.fft_plan_workspace_bytes(h2)), dtype=torch.uint8, device=dev)
        if lib.fft_plan_workspace_bytes(h2):
            _lib.check(lib.fft_plan_set_workspace(h2, ctypes.c_void_p(ws2.data_ptr())))
        ms = _time_fn(torch, lambda: run_plan(h2, img, y), args.steps, args.warmup, stream)
        nl2 = lib.fft_plan_launches(h2)
        res.append({"n": "8192x8192", "us": round(ms * 1e3, 1),
                    "gflops": round(flops(1 << 26, 1) / (ms * 1e-3) / 1e9, 1),
                    "hbm_frac_algorithmic": round(16.0 * (1 << 26) / (ms * 1e-3) / 1e9 / peak, 4),
                    "hbm_frac_per_launch": round(16.0 * (1 << 26) * nl2 / (ms * 1e-3) / 1e9 / peak, 4),
                    "launches": nl2})
        lib.fft_destroy(h2)
        desc = "large transforms: four-step 1-D N = 2^20..2^26 (2^26 points per launch), 2-D 8192x8192 SAR image"
    elif args.workload == "many":
        lengths = workloads.uneven_lengths(4096, seed=workloads.seed_for(4)).tolist()
        total = int(sum(lengths))
        xh = workloads.packed_cgauss(lengths, seed=workloads.seed_for(4, 2))
        wh = workloads.real_weights(total, seed=workloads.seed_for(4, 1))
        x = torch.from_numpy(xh).to(dev)
        w2 = torch.from_numpy(2.0 * wh.astype(np.float32) ** 2).to(dev)
        p = api.get_plan("many", (total,), len(lengths), "fp32", dev, lengths=tuple(lengths), tuned=True)
        X = torch.empty_like(x)
        G = torch.empty_like(x)
        gx = torch.empty_like(x)

        def step():
            p.exec_ptr(x.data_ptr(), X.data_ptr(), 0, stream)          # forward, one persistent launch
            torch.mul(X, w2, out=G)                                     # dL/dX* = 2 w^2 X
            p.exec_ptr(G.data_ptr(), gx.data_ptr(), 2, stream)          # backward: adjoint F^H

        with torch.cuda.stream(stream):
            step()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            step()
        ms = _time_fn(torch, g.replay, args.steps, args.warmup, stream)
        ms_fwd = _time_fn(torch, lambda: p.exec_ptr(x.data_ptr(), X.data_ptr(), 0, stream), args.steps,
                          args.warmup, stream)
        fl = sum(flops(n, 1) for n in lengths)
        # gradient check on a sample of transforms against the oracle
        gxh = gx.cpu().numpy()
        offs = np.concatenate([[0], np.cumsum(lengths)])
        errs = []
        for i in range(0, len(lengths), 97):
            a, b = offs[i], offs[i + 1]
            ref = oracle.spectral_loss_grad(xh[a:b].astype(np.complex128), wh[a:b].astype(np.float64))
            errs.append(oracle.rel_l2(gxh[a:b], ref))
        res.append({"transforms": len(lengths), "points": total, "graph_step_us": round(ms * 1e3, 1),
                    "forward_us": round(ms_fwd * 1e3, 1),
                    "gflops_fwd_plus_bwd": round(2 * fl / (ms * 1e-3) / 1e9, 1),
                    "gflops_fwd": round(fl / (ms_fwd * 1e-3) / 1e9, 1),
                    "hbm_frac_fwd": round(16.0 * total / (ms_fwd * 1e-3) / 1e9 / peak, 4),
                    "grad_rel_l2_max_sampled": float(f"{max(errs):.3e}"), "grad_samples": len(errs)})
        desc = ("uneven batch: 4096 transforms, lengths 2^e with e uniform over 8..16, CN(0,1); "
                "graph-captured forward + loss gradient + adjoint backward")
    elif args.workload == "range":
        # SAR range compression: 2^26 / N range lines of N samples, each the
        # echoes of a linear-FM pulse of N/4 samples; closed-form matched filter
        for lg in (12, 13, 14, 16, 20):
            n = 1 << lg
            batch = TOTAL // n
            P = n // 4
            xh = workloads.range_lines(n, batch, P, n_targets=2, seed=workloads.seed_for(6) + lg)
            Hh = workloads.range_filter(n, P)
            x = torch.from_numpy(xh.reshape(-1)).to(dev)
            H = torch.from_numpy(Hh).to(dev)
            y = torch.empty_like(x)
            X = torch.empty_like(x)
            p = api.Plan("1d", (n,), batch, device=dev)
            fused = _time_fn(torch, lambda: p.exec_filter_ptr(x.data_ptr(), y.data_ptr(), H.data_ptr(), stream),
                             args.steps, args.warmup, stream)
            X2 = X.view(batch, n)

            def unfused():
                p.exec_ptr(x.data_ptr(), X.data_ptr(), 0, stream)
                with torch.cuda.stream(stream):
                    torch.mul(X2, H, out=X2)
                p.exec_ptr(X.data_ptr(), y.data_ptr(), 1, stream)

            sep = _time_fn(torch, unfused, args.steps, args.warmup, stream)

            def cufft():
                with torch.cuda.stream(stream):
                    torch.fft.ifft(torch.fft.fft(x.view(batch, n)) * H)

            cu = _time_fn(torch, cufft, args.steps, args.warmup, stream)
            p.exec_filter_ptr(x.data_ptr(), y.data_ptr(), H.data_ptr(), stream)
            torch.cuda.synchronize()
            rows = [0, batch // 2, batch - 1]
            ref = oracle.range_compress(xh[rows].astype(np.complex128), Hh.astype(np.complex128))
            got = y.view(batch, n)[rows].cpu().numpy().astype(np.complex128)
            scale = np.abs(Hh).max() * np.sqrt(np.sum(np.abs(xh[rows].astype(np.complex128)) ** 2, axis=-1))
            err = float(np.max(np.sqrt(np.sum(np.abs(got - ref) ** 2, axis=-1)) / scale))
            fl = (10.0 * n * lg + 6.0 * n) * batch
            nl = p.launches
            res.append({"n": n, "lines": batch, "pulse": P, "fused_us": round(fused * 1e3, 1),
                        "unfused_us": round(sep * 1e3, 1), "cufft_torch_us": round(cu * 1e3, 1),
                        "gflops": round(fl / (fused * 1e-3) / 1e9, 1),
                        "hbm_frac_algorithmic": round(16.0 * n * batch / (fused * 1e-3) / 1e9 / peak, 4),
                        "launches": 1 if nl == 1 else 2 * nl,
                        "err_sampled": float(f"{err:.3e}")})
            del p
        desc = ("SAR range compression IFFT(H * FFT(line)): 2^26/N lines of N samples, LFM echoes + CN(0,1) "
                "noise, closed-form matched filter; fused = fft_exec_filter, unfused = FFT, torch multiply, "
                "IFFT; cufft_torch = torch.fft (context)")
    elif args.workload == "real":
        # real-data transforms: 2^26 reals per launch, N reals per row
        for lg in (12, 13, 14, 15, 16, 20):
            n = 1 << lg
            batch = TOTAL // n
            xh = workloads.uniform(n, batch, seed=workloads.seed_for(7) + lg).real.astype(np.float32)
            x = torch.from_numpy(xh).to(dev)
            X = torch.empty(batch, n // 2 + 1, dtype=torch.complex64, device=dev)
            y = torch.empty_like(x)
            p = api.Plan("r2c", (n,), batch, device=dev)
            fwd = _time_fn(torch, lambda: p.exec_ptr(x.data_ptr(), X.data_ptr(), 0, stream), args.steps,
                           args.warmup, stream)
            inv = _time_fn(torch, lambda: p.exec_ptr(X.data_ptr(), y.data_ptr(), 1, stream), args.steps,
                           args.warmup, stream)

            def cufft():
                with torch.cuda.stream(stream):
                    torch.fft.rfft(x)

            cu = _time_fn(torch, cufft, args.steps, args.warmup, stream)

            def cufft_inv():
                with torch.cuda.stream(stream):
                    torch.fft.irfft(X, n)

            cui = _time_fn(torch, cufft_inv, args.steps, args.warmup, stream)
            p.exec_ptr(x.data_ptr(), X.data_ptr(), 0, stream)
            torch.cuda.synchronize()
            rows = [0, batch // 2, batch - 1]
            err = float(oracle.rel_l2_rows(X[rows].cpu().numpy(), oracle.rfft(xh[rows].astype(np.float64))).max())
            # algorithmic bytes: N reals in (4 B each) and N/2 + 1 complex out (8 B each)
            byt = (4.0 * n + 8.0 * (n // 2 + 1)) * batch
            res.append({"n": n, "rows": batch, "rfft_us": round(fwd * 1e3, 1), "irfft_us": round(inv * 1e3, 1),
                        "cufft_torch_rfft_us": round(cu * 1e3, 1), "cufft_torch_irfft_us": round(cui * 1e3, 1),
                        "gflops_rfft": round(2.5 * n * lg * batch / (fwd * 1e-3) / 1e9, 1),
                        "hbm_frac_rfft": round(byt / (fwd * 1e-3) / 1e9 / peak, 4),
                        "hbm_frac_irfft": round(byt / (inv * 1e-3) / 1e9 / peak, 4),
                        "launches": p.launches, "err_sampled": float(f"{err:.3e}")})
            del p
        desc = ("real-data transforms: 2^26 U[-1,1] reals per launch in rows of N; rfft -> N/2+1 complex, irfft "
                "back; GFLOP/s counts 2.5 N log2 N per real row; cufft_torch = torch.fft.rfft (context)")
    elif args.workload == "mixed":
        # lengths that are not powers of two: ~2^26 points per launch
        for n in (1000, 3000, 5000, 6000, 10000, 12000):
            batch = TOTAL // n
            x = torch.from_numpy(workloads.cgauss(n, batch, seed=workloads.seed_for(8) + n).reshape(-1)).to(dev)
            y = torch.empty_like(x)
            h, wsb = plan(n, batch, 0)
            us = _time_fn(torch, lambda: run_plan(h, x, y), args.steps, args.warmup, stream) * 1e3

            def cufft():
                with torch.cuda.stream(stream):
                    torch.fft.fft(x.view(batch, n))

            cu = _time_fn(torch, cufft, args.steps, args.warmup, stream) * 1e3
            run_plan(h, x, y)
            torch.cuda.synchronize()
            rows = [0, batch - 1]
            xr = x.view(batch, n)[rows].cpu().numpy()
            err = float(oracle.rel_l2_rows(y.view(batch, n)[rows].cpu().numpy(),
                                           oracle.transform(xr.astype(np.complex128))).max())
            res.append({"n": n, "batch": batch, "us": round(us, 1), "cufft_torch_us": round(cu, 1),
                        "gflops": round(5.0 * n * np.log2(n) * batch / (us * 1e-6) / 1e9, 1),
                        "hbm_frac": round(16.0 * n * batch / (us * 1e-6) / 1e9 / peak, 4),
                        "err_sampled": float(f"{err:.3e}")})
            lib.fft_destroy(h)
        desc = ("mixed-radix lengths (2^a 3^b 5^c 7^d, one on-chip pass): ~2^26 CN(0,1) points per launch; "
                "cufft_torch = torch.fft (context)")
    elif args.workload == "fp64":
        # complex128 transforms in FP64: 2^25 points per launch (512 MiB each way)
        for n in (1024, 4096, 1000, 5000):
            batch = (1 << 25) // n
            g = np.random.Generator(np.random.PCG64(workloads.seed_for(9) + n))
            xh = g.normal(0, np.sqrt(0.5), (batch, n)) + 1j * g.normal(0, np.sqrt(0.5), (batch, n))
            x = torch.from_numpy(xh.reshape(-1)).to(dev)
            y = torch.empty_like(x)
            h = ctypes.c_void_p(lib.fft_plan_create(n, batch, 0, _lib.FFT_PREC_FP64))
            us = _time_fn(torch, lambda: run_plan(h, x, y), args.steps, args.warmup, stream) * 1e3

            def cufft():
                with torch.cuda.stream(stream):
                    torch.fft.fft(x.view(batch, n))

            cu = _time_fn(torch, cufft, args.steps, args.warmup, stream) * 1e3
            run_plan(h, x, y)
            torch.cuda.synchronize()
            rows = [0, batch - 1]
            err = float(oracle.rel_l2_rows(y.view(batch, n)[rows].cpu().numpy(), oracle.transform(xh[rows])).max())
            res.append({"n": n, "batch": batch, "us": round(us, 1), "cufft_torch_us": round(cu, 1),
                        "gflops_fp64": round(5.0 * n * np.log2(n) * batch / (us * 1e-6) / 1e9, 1),
                        "hbm_frac": round(32.0 * n * batch / (us * 1e-6) / 1e9 / peak, 4),
                        "err_sampled": float(f"{err:.3e}")})
            lib.fft_destroy(h)
        desc = ("FP64 (complex128) transforms, one on-chip pass: 2^25 CN(0,1) points per launch; HBM fraction "
                "counts 32 B per point; cufft_torch = torch.fft on complex128 (context)")
    elif args.workload == "passes":
        # two strided mixed-radix passes: FP64 lengths beyond one pass (2^25 points per launch) and
        # FP32 mixed-radix lengths beyond 14336 (~2^26 points), 1-D and 2-D
        cases = [(1 << 13, None, 5), (1 << 16, None, 5), (1 << 20, None, 5), (1 << 24, None, 5), (10000, None, 5),
                 (10 ** 6, None, 5), (1024, 1024, 5), (15000, None, 0), (16000, None, 0), (10 ** 6, None, 0),
                 (1000, 1000, 0)]
        for n, ny, prec in cases:
            fp64 = prec == _lib.FFT_PREC_FP64
            pts = (1 << 25) if fp64 else TOTAL
            img = n * (ny or 1)
            batch = max(1, pts // img)
            gen = workloads.cgauss128 if fp64 else workloads.cgauss
            xh = gen(img, batch, seed=workloads.seed_for(10) + img)
            x = torch.from_numpy(xh.reshape(-1)).to(dev)
            y = torch.empty_like(x)
            if ny:
                h = ctypes.c_void_p(lib.fft_plan_create_2d(ny, n, batch, 0, prec))
                wsb = None
            else:
                h, wsb = plan(n, batch, prec)
            us = _time_fn(torch, lambda: run_plan(h, x, y), args.steps, args.warmup, stream) * 1e3
            shape = (batch, ny, n) if ny else (batch, n)

            def cufft():
                with torch.cuda.stream(stream):
                    (torch.fft.fft2 if ny else torch.fft.fft)(x.view(*shape))

            cu = _time_fn(torch, cufft, args.steps, args.warmup, stream) * 1e3
            run_plan(h, x, y)
            torch.cuda.synchronize()
            if ny:
                err = None
                if n & (n - 1) == 0 and ny & (ny - 1) == 0:
                    got = y.view(*shape)[:1].cpu().numpy()
                    err = float(oracle.rel_l2(got, oracle.fft2(xh.reshape(shape)[:1].astype(np.complex128))))
            else:
                ks = np.array([0, 1, n // 3, n - 1])
                got = y.view(*shape)[[0, batch - 1]][:, ks].cpu().numpy()
                err = float(oracle.rel_l2_rows(got, oracle.dft_bins(xh[[0, batch - 1]].astype(np.complex128),
                                                                    ks)).max())
            N = img
            res.append({"n": n, "ny": ny, "batch": batch, "prec": "fp64" if fp64 else "fp32", "us": round(us, 1),
                        "cufft_torch_us": round(cu, 1),
                        "gflops": round(5.0 * N * np.log2(N) * batch / (us * 1e-6) / 1e9, 1),
                        "hbm_frac": round((32.0 if fp64 else 16.0) * N * batch / (us * 1e-6) / 1e9 / peak, 4),
                        "err_sampled": None if err is None else float(f"{err:.3e}")})
            lib.fft_destroy(h)
            del wsb
        desc = ("two strided mixed-radix passes (four-step N = N1 N2, or rows then columns): FP64 complex128 "
                "2^25 points per launch, FP32 ~2^26; errors at sampled outputs (term-by-term oracle sums) or "
                "whole images; cufft_torch = torch.fft (context)")
    elif args.workload == "radix":
        # the autotuner's radix dimension for one on-chip pass: radix-16 / 8 / 4 passes (16 / 8 / 4 points
        # per thread) on the register path, the planner default, and what fft_autotune picks, 2^26 points
        for lg in range(5, 15):
            n = 1 << lg
            batch = TOTAL // n
            xh = workloads.cgauss(n, batch, seed=workloads.seed_for(1) + lg)
            x = torch.from_numpy(xh.reshape(-1)).to(dev)
            y = torch.empty_like(x)
            ref = oracle.fft(xh[[0, batch - 1]].astype(np.complex128))
            row = {"n": n, "batch": batch}
            cands = [("default", None)] + [(f"radix{r}", {"npass": 1, "tma": 0, "radix": r}) for r in (16, 8, 4)]
            for name, cfg in cands:
                if cfg is None:
                    h = lib.fft_plan_create(n, batch, 0, 0)
                else:
                    c = _lib.FftPlanConfig.from_dict(cfg)
                    h = lib.fft_plan_create_config(n, batch, 0, 0, ctypes.byref(c))
                if not h:
                    row[name] = None
                    continue
                h = ctypes.c_void_p(h)
                us = _time_fn(torch, lambda: run_plan(h, x, y), args.steps, args.warmup, stream) * 1e3
                got = y.view(batch, n)[[0, batch - 1]].cpu().numpy()
                err = float(oracle.rel_l2_rows(got, ref).max())
                row[name] = {"us": round(us, 1), "hbm_frac": round(16.0 * n * batch / (us * 1e-6) / 1e9 / peak, 4),
                             "rel_l2_max": float(f"{err:.3e}")}
                lib.fft_destroy(h)
            best = _lib.FftPlanConfig()
            best_us = ctypes.c_float(0.0)
            _lib.check(lib.fft_autotune(n, batch, 0, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                        None, 0, sh, args.steps, ctypes.byref(best), ctypes.byref(best_us)))
            row["autotune"] = {"config": best.as_dict(), "us": round(float(best_us.value), 1)}
            res.append(row)
        desc = ("one on-chip pass, N = 2^5..2^14, batch 2^26/N, CN(0,1): register-path kernels with radix-16 / 8 / 4 "
                "passes (points per thread = radix), the planner default and the autotuner's pick (fft_autotune "
                "over every candidate, no workspace: single-pass candidates only); sampled rows against the oracle")
    print(json.dumps({"workload": args.workload, "desc": desc, "results": res,
                      "peak_hbm_gbs": peak}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gbfft", choices=["gbfft", "reference"])
    ap.add_argument("--workload", default="cfg2", choices=["cfg2", "large", "tc", "many", "range", "real", "mixed", "fp64",
                                                          "passes", "radix"])
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle time for cpu_baseline")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the per-size results of configurations 1, 3, 4, 5")
    ap.add_argument("--case", type=int, default=0, help="run one plan of 2^CASE points (profiling case)")
    ap.add_argument("--tuned", type=int, default=1, help="1: plans from the autotuner (default), 0: planner defaults")
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--dir", type=int, default=0)
    ap.add_argument("--prec", type=int, default=0)
    ap.add_argument("--filter", action="store_true", help="with --case: range compression instead of the FFT")
    ap.add_argument("--case-n", type=int, default=0, help="profiling case of any supported length n")
    ap.add_argument("--real", action="store_true", help="with --case/--case-n: a real-data plan (--dir 0 r2c, 1 c2r)")
    ap.add_argument("--tma", type=int, default=-1, help="with --case: the configuration's tma field (-1: planner default)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.case or args.case_n:
        run_case(args)
    elif args.workload != "cfg2" and args.impl != "reference":
        run_measure(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
