"""The batch pool's first-fit allocator (csrc/lb_pool.h, host code) against
a brute-force model of the pool on randomised allocate / release sequences:
first fit by address, failure only when no free run holds the request,
exact free-byte counts and full coalescing.  Built with the host compiler
from the same header and run on the CPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_pool_allocator_against_model(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path / "pool_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-Wall", "-Werror",
                    "-I", os.path.join(ROOT, "paper_2409_16781_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "pool_check.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe), "300"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "pool checks failed: 0" in r.stdout
