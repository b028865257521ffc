"""Host check of the exact fixed-point path's IEEE <-> 128-bit conversions (no GPU).

The conversions live in a header shared by host and device code; this test
builds tests/fixed_point_check.cpp against it with the host compiler and runs
it: exact round trips, nearest-even rounding against the compiler's own
conversions, subnormal results against integer rounding, carries into the
exponent and overflow.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_fixed_point_conversions(tmp_path):
    cxx = os.environ.get("CXX") or shutil.which("g++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "fixed_point_check"
    subprocess.check_call([cxx, "-std=c++17", "-O2", "-o", str(exe), os.path.join(HERE, "fixed_point_check.cpp")])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("ok")
