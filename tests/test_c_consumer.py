"""The boundary from C: a plain C99 program includes include/gbfft.h,
compiles with every warning as an error, links against libgbfft.so and
exercises the calls that are answered on the host (argument rejection,
error strings, NULL safety).  No GPU is touched."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "gbfft.h"

static int fails = 0;
#define CHECK(c) do { if (!(c)) { fprintf(stderr, "failed: %s\n", #c); ++fails; } } while (0)

int main(void) {
    int64_t lengths[2] = {16, 3};
    fft_plan_config cfg;
    memset(&cfg, 0, sizeof cfg);
    CHECK(fft_plan_create(11, 1, FFT_FORWARD, FFT_PREC_FP32) == NULL);
    CHECK(fft_last_error() == FFT_ERR_INVALID_ARG);
    CHECK(fft_plan_create(1024, 0, FFT_FORWARD, FFT_PREC_FP32) == NULL);
    CHECK(fft_plan_create(1024, 1, 7, FFT_PREC_FP32) == NULL);
    CHECK(fft_plan_create_2d(11, 16, 1, FFT_INVERSE, FFT_PREC_FP32) == NULL);
    CHECK(fft_plan_create_many(lengths, 2, FFT_FORWARD, FFT_PREC_FP32) == NULL);
    CHECK(fft_plan_create_r2c(12, 1, FFT_PREC_FP32) == NULL);
    CHECK(fft_plan_create_config(11, 1, FFT_FORWARD, FFT_PREC_FP32, &cfg) == NULL);
    CHECK(fft_last_error() == FFT_ERR_INVALID_ARG);
    CHECK(fft_exec(NULL, NULL, NULL, NULL) == FFT_ERR_INVALID_ARG);
    CHECK(fft_exec_dir(NULL, NULL, NULL, FFT_INVERSE | FFT_ADJOINT, NULL) == FFT_ERR_INVALID_ARG);
    CHECK(fft_exec_filter(NULL, NULL, NULL, NULL, NULL) == FFT_ERR_INVALID_ARG);
    CHECK(fft_exec_filter_dir(NULL, NULL, NULL, NULL, FFT_ADJOINT, NULL) == FFT_ERR_INVALID_ARG);
    CHECK(fft_plan_workspace_bytes(NULL) == 0);
    CHECK(fft_plan_launches(NULL) == 0);
    CHECK(strcmp(fft_error_string(FFT_OK), "ok") == 0);
    CHECK(strcmp(fft_error_string(FFT_ERR_TIMEOUT), "unknown error") != 0);
    fft_destroy(NULL);
    printf("%d\n", fails);
    return fails != 0;
}
"""


def test_c_program_uses_the_boundary(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1707_07263_gb300 import build_lib
    lib = build_lib.build()
    src = tmp_path / "consumer.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "consumer"
    libdir = os.path.dirname(lib)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe), "-L", libdir, "-l:" + os.path.basename(lib),
                        "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stdout + run.stderr
    assert run.stdout.strip() == "0"
