"""The integer-pipe conversions the integrator and the rebuild use in place
of the GPU's FP64-pipe conversions (csrc/md_fpconv.cuh) give the same bits
as the CPU's IEEE-754 round-to-nearest-even conversions: FP32 -> FP64,
FP64 -> FP32 (ties, carries into the next binade, overflow to infinity,
flush-to-zero below FLT_MIN), k + 1/2 and the floor of a non-negative
double.  The header is compiled as plain C++ by the host compiler."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1408_4599_gb300", "csrc")


def test_integer_conversions_match_ieee(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "fpconv_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC,
                    os.path.join(HERE, "native", "fpconv_check.cpp"), "-o", exe], check=True)
    p = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stdout + p.stderr
