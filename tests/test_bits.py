"""The integer-operation float <-> double conversions and comparisons of
csrc/gc_bits.h (used by the kernels in place of FP64-unit conversions and
compares) agree bit for bit with the host's IEEE conversions (round to
nearest even) and comparisons: every float exponent and sign, every double
exponent, rounding ties and their neighbours at every float exponent, range
edges, zeros of both signs (tests/c/bits_check.cpp)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bit_conversions_match_ieee(tmp_path):
    if not shutil.which("g++"):
        pytest.skip("g++ not found")
    exe = tmp_path / "bits_check"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2203_11043_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "c", "bits_check.cpp"), "-o", str(exe)], check=True,
                   capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout
    assert "bits ok" in r.stdout
