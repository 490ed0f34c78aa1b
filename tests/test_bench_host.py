"""The benchmark's host-side bookkeeping on CPU: the clock record it attaches
to every line, and the rule that recorded DRAM traffic is reported only while
the kernel sources it was captured from are unchanged."""
from __future__ import annotations

import json
import os
import shutil

import bench


def test_clock_summary():
    s = bench.ClockSampler("0")
    assert s.summary() is None
    s.lines = [
        "0, 2070, 2070, 910.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    got = s.summary()
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    s.lines = ["0, 1500, 2070, 700, 0x8, Active, Not Active, Active, Not Active"]
    assert s.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_traffic_only_for_unchanged_sources(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1707_07263_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in bench.BENCH_KERNEL_SOURCES:
        shutil.copy(os.path.join(bench.ROOT, "paper_1707_07263_gb300", "csrc", name), csrc / name)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("tile_fft_pf_kernel_lg14") is None            # no record
    (tmp_path / "profiles").mkdir()
    rec = {"source_hash": bench.source_hash(),
           "kernels": {"tile_fft_pf_kernel_lg14": {"dram_bytes_per_launch": 1012296448}}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.ncu_traffic("tile_fft_pf_kernel_lg14") == 1012296448.0
    assert bench.ncu_traffic("some_other_kernel") is None
    with open(csrc / bench.BENCH_KERNEL_SOURCES[1], "a") as f:             # a kernel source changes
        f.write("\n")
    assert bench.ncu_traffic("tile_fft_pf_kernel_lg14") is None


def test_peaks_and_flops(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (bench.HBM_FALLBACK, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6785.9}))
    assert bench.measured_peaks() == (6785.9, "measured")
    assert bench.flops(1024, 3) == 5.0 * 1024 * 10 * 3
