"""Host-side check of the Stockham radix schedules that the tile kernels and
the stage-twiddle generator share (no GPU): the constexpr schedule functions
of csrc/tile_fft.cuh, compiled into a small host program, give for every
length 2^1..2^14 and every largest radix (16, 8, 4; 16 also with the
remainder pass last) the pass list of the Cooley-Tukey split written out here
(full-radix passes plus one remainder pass, the radices multiplying to L), and
a stage-twiddle table of lgr * Ns entries per twiddled pass, laid out pass
after pass.  The tile geometry of the compiled radix-8 / radix-4 single-pass
kernels (threads = transforms per CTA * L / points per thread <= 1024,
shared memory within 227 KB) is checked the same way."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <cstdio>
#include "tile_fft.cuh"
#include "tile_registry.h"
using namespace gbfft;

template <int LG, int LGM>
void geom() {
  using Cfg = TileCfg<LG, jj_cols(LG), false, false, 0, LGM>;
  std::printf("G %d %d %d %d %d %d\n", LG, LGM, jj_cols(LG), Cfg::P, Cfg::T, Cfg::SMEM_BYTES);
}
template <int LG, int LGM>
void geoms() {
  geom<LG, LGM>();
  if constexpr (LG < (LGM == 3 ? 13 : 12)) geoms<LG + 1, LGM>();
}

int main() {
  for (int lgm = 2; lgm <= 4; ++lgm)
    for (int rev = 0; rev <= (lgm == 4 ? 1 : 0); ++rev)
      for (int lg = 1; lg <= 14; ++lg) {
        std::printf("S %d %d %d %d %d", lg, lgm, rev, radix_nst(lg, lgm), stage_tw_size(lg, rev != 0, lgm));
        for (int s = 0; s < radix_nst(lg, lgm); ++s)
          std::printf(" %d:%d:%d", radix_lgr(lg, s, rev != 0, lgm), radix_lgns(lg, s, rev != 0, lgm),
                      stage_tw_off(lg, s, rev != 0, lgm));
        std::printf("\n");
      }
  geoms<5, 3>();
  geoms<5, 2>();
  return 0;
}
"""


def schedule(lg: int, rev: bool, lgm: int):
    rest = [lgm] * (lg // lgm)
    if lg % lgm:
        rest = rest + [lg % lgm] if rev else [lg % lgm] + rest
    return rest


@pytest.fixture(scope="module")
def output(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("sched")
    src = d / "sched.cu"
    src.write_text(PROGRAM)
    exe = d / "sched"
    csrc = os.path.join(ROOT, "paper_1707_07263_gb300", "csrc")
    subprocess.check_call([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode",
                           "arch=compute_103a,code=sm_103a", "-I", csrc, "-I", os.path.join(ROOT, "include"),
                           str(src), "-o", str(exe)])
    return subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()


def test_schedules_and_stage_table_layout(output):
    seen = 0
    for line in output:
        if not line.startswith("S "):
            continue
        f = line.split()
        lg, lgm, rev, nst, size = (int(v) for v in f[1:6])
        passes = [tuple(int(v) for v in p.split(":")) for p in f[6:]]
        want = schedule(lg, bool(rev), lgm)
        assert nst == len(want) and [p[0] for p in passes] == want, line
        lgns = off = 0
        for lgr, got_lgns, got_off in passes:
            assert (got_lgns, got_off) == (lgns, off), line
            if lgns > 0:
                off += lgr * (1 << lgns)     # rows e = 0..lgr-1 of Ns entries W_{Ns R}^{2^e k}
            lgns += lgr
        assert lgns == lg and size == off, line
        seen += 1
    assert seen == 4 * 14


def test_compiled_radix_kernels_fit_a_cta(output):
    rows = [tuple(int(v) for v in line.split()[1:]) for line in output if line.startswith("G ")]
    assert len(rows) == 9 + 8          # radix 8: 2^5..2^13, radix 4: 2^5..2^12
    for lg, lgm, cols, p, threads, smem in rows:
        assert p == 1 << lgm
        assert threads == cols * (1 << lg) // p <= 1024
        assert smem <= 227 * 1024
