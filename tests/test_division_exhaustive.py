"""The small-n_f epilogues' division (ps::div_rn_lean, the quotient of Eq. 2's
c2 = 2 n2 / (S_i + S_j)) against CUDA's correctly rounded __fdiv_rn.

division_exhaustive.cu compares the two bit for bit on every pair of FP32
significands in [1, 2) (2^46 pairs) and checks that rcp.approx scales exactly
with the exponent over the division's range of denominators; together they
cover every input of that range, since each step of the division scales
exactly with powers of two there.
"""
import os
import subprocess

import pytest

from paper_1705_08210_gb300 import build_lib

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "division_exhaustive.cu")


def _compile(out_path):
    cmd = [build_lib.nvcc()] + build_lib.ARCH + ["-O3", "-std=c++17", SRC, "-o", out_path]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr


def test_division_check_compiles(tmp_path):
    # cross-compiles for sm_103a without a GPU
    _compile(str(tmp_path / "division_exhaustive"))


@pytest.mark.gpu
def test_lean_division_exhaustive(tmp_path):
    exe = str(tmp_path / "division_exhaustive")
    _compile(exe)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("mismatches")][-1]
    rcp_bad, quot_bad, zero_bad = (int(v) for v in line.split()[1:])
    assert rcp_bad == 0, "rcp.approx is not exact under scaling by powers of two"
    assert zero_bad == 0, "0 / d is not +0"
    assert quot_bad == 0, f"{quot_bad} of 2^46 quotients differ from __fdiv_rn"
