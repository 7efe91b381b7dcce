"""The library's numerics header (csrc/rs_numeric.cuh) compiled as host C++ (no GPU):

* df_to_fixed's short path gives the bits of its general path (each float part truncated
  toward zero at the scale, summed, a negative sum clamped to 0) on random bit patterns,
  normalised and non-normalised double-floats, zeros, subnormals and products;
* the double-float product, sum, quotient by an integer and cube root stay within 2^-44
  relative of long double (the scores' tolerance is 1e-12).

The device intrinsics are given their IEEE-754 meaning on the host (tests/numeric_host.cpp)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "numeric_host.cpp")
CSRC = os.path.join(ROOT, "paper_2508_01485_gb300", "csrc")
EXE = os.path.join(HERE, "_build", "numeric_host")


@pytest.fixture(scope="module")
def exe():
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    os.makedirs(os.path.dirname(EXE), exist_ok=True)
    tmp = EXE + ".%d.tmp" % os.getpid()
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-I", CSRC, "-o", tmp, SRC])
    os.replace(tmp, EXE)
    return EXE


def test_fixed_point_short_path_equals_general_path(exe):
    r = subprocess.run([exe, "6000000"], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches 0" in r.stdout
    cases, short = (int(x) for x in r.stdout.split()[1:4:2])
    assert cases > 5_900_000 and short > cases // 10       # the short path is exercised


def test_double_float_accuracy(exe):
    r = subprocess.run([exe, "accuracy", "1000000"], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
