"""The product path and the oracle stay apart: importing and using the
package's host side never loads `oracle`, the package's sources never import
it, and the oracle shares no source with the CUDA library."""
from __future__ import annotations

import ast
import glob
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1707_07263_gb300")


def test_package_sources_do_not_import_the_oracle():
    for path in glob.glob(os.path.join(PKG, "*.py")):
        with open(path) as f:
            tree = ast.parse(f.read())
        for node in ast.walk(tree):
            names = []
            if isinstance(node, ast.Import):
                names = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                names = [node.module or ""]
            assert not any(n == "oracle" or n.startswith("oracle.") for n in names), path


def test_importing_the_package_loads_no_oracle():
    code = ("import sys; import paper_1707_07263_gb300 as gb; import paper_1707_07263_gb300.api, "
            "paper_1707_07263_gb300.tune, paper_1707_07263_gb300.workloads, paper_1707_07263_gb300.build_lib; "
            "print('oracle' in sys.modules)")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "False"


def test_oracle_and_cuda_sources_share_nothing():
    csrc = os.path.join(PKG, "csrc")
    cuda_names = {os.path.basename(p) for p in glob.glob(os.path.join(csrc, "*"))}
    with open(os.path.join(ROOT, "oracle", "fft_oracle.c")) as f:
        src = f.read()
    includes = [ln.split()[1].strip('<>"') for ln in src.splitlines() if ln.startswith("#include")]
    assert includes and not any(os.path.basename(i) in cuda_names or "gbfft" in i for i in includes)
    assert set(os.listdir(os.path.join(ROOT, "oracle"))) & cuda_names == set()
