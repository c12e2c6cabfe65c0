"""The integer FP32 <-> FP64 conversions of the Mixed2 storage form
(csrc/lb_fpconv.cuh) equal the IEEE conversions bit for bit: every binary32
pattern widened (and narrowed back), random binary64 patterns in and around
the FP32 range, and the rounding ties of every exponent.  Built with the host
compiler from the same header and run on the CPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_integer_conversions_match_ieee(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path / "fpconv_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2409_16781_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "fpconv_check.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe), "20000000"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "widen 0 roundtrip 0 random 0 edge 0" in r.stdout
