"""The transform's exact float <-> double conversions and near-plane test
(`csrc/ieee754.h`, integer operations on the IEEE 754 encodings) agree with
the C conversions and comparison: every subnormal float, a stride over all
float patterns, random doubles over every exponent, round-to-nearest-even
ties and their neighbours on the normal and subnormal grids, overflow, and
NaN, zeros and infinities for the comparison.  Host code only."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "native", "ieee754_check.cpp")
INC = os.path.join(ROOT, "paper_1004_1302_gb300", "csrc")


def test_conversions_match_the_c_library(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "ieee754_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-fno-fast-math", "-I", INC, SRC, "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok "), out.stdout
    assert int(out.stdout.split()[1]) > 50_000_000
