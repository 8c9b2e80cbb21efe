"""Host check of the library's modular-arithmetic helpers (he_arith.cuh) against exact 128-bit
arithmetic: the value ranges the kernels rely on (Shoup's product with the cheaper quotient
estimate in [0, 4q), 96-bit sums of residue products and their reduction). The device forms of
the same helpers are covered by the bit-exact GPU parity tests."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_arith_helpers_match_exact_arithmetic(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path / "arith_bounds"
    src = os.path.join(ROOT, "tests", "arith_bounds.cpp")
    inc = os.path.join(ROOT, "paper_2512_18646_gb300", "csrc")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", inc, "-o", str(exe), src], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
