"""The split state's FP64 <-> float-float conversions (csrc/ff_convert.h) against the FP64
arithmetic they replace, bit for bit, on the host: the header's integer paths are compiled
with the host compiler and checked on random and constructed words (every binade gap between
the two words of a pair, borrows from a power-of-two high word, exact ties, carries into the
next binade, zeros, subnormals, infinities, NaN). The device build compiles the same source."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_integer_conversions_match_fp64_arithmetic(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "ff_convert_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I",
                    os.path.join(ROOT, "paper_1505_02248_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "ff_convert_check.cpp"), "-o", exe], check=True)
    out = subprocess.run([exe, "2000000"], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok ")
