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


def test_fp32_quotient_estimate_is_at_most_one_off():
    """The transforms' final reduction (reduce_fp32 in he_arith.cuh) estimates floor(v / q) for
    v < 2^9 q as trunc(fl32(fl32(v >> sh) * fl32(2^sh / q))), sh = max(0, bitlen(q) + 9 - 32), and
    corrects the remainder once: the estimate must be floor(v / q) or one off for every prime size
    the transforms' growing-range path takes (below 2^54), at the ends of each quotient interval
    (where rounding bites) and at random points. The fp32 steps are reproduced with numpy's
    round-to-nearest float32 arithmetic, as the device's __uint2float_rn / __fmul_rn round."""
    import numpy as np
    rng = np.random.default_rng(9)
    for bits in (20, 30, 40, 45, 50, 53):
        for _ in range(4):
            q = int(rng.integers(1 << (bits - 1), 1 << bits)) | 1
            sh = max(0, q.bit_length() + 9 - 32)
            frd = np.float32((2.0 ** sh) / q)
            vs = [int(v) for v in rng.integers(0, 512 * q, size=2000, dtype=np.uint64)] if 512 * q < 2 ** 63 else \
                [int(rng.integers(0, 2 ** 62)) % (512 * q) for _ in range(2000)]
            for t in range(0, 512, 7):  # both ends of quotient intervals
                vs += [t * q, t * q + 1, (t + 1) * q - 1, max(0, t * q - 1)]
            for v in vs:
                if v >= 512 * q:
                    continue
                hi = np.float32(v >> sh)
                est = int(np.float32(hi * frd))
                true = v // q
                assert abs(est - true) <= 1, (bits, q, v, est, true)
                r = v - est * q
                r = r + q if r < 0 else (r - q if r >= q else r)
                assert r == v % q
