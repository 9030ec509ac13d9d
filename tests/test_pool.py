"""The serving engine's grid-pool allocator (host logic, no GPU): pool_check.cpp
drives it with random allocations and releases and compares every result with
a brute-force model of the live ranges (first fit, no overlap, exact
accounting, full coalescing)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_free_list_matches_brute_force_model(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path / "pool_check"
    subprocess.run([cxx, "-O1", "-std=c++17", "-Wall", "-Werror", os.path.join(HERE, "pool_check.cpp"), "-o",
                    str(exe)], check=True, capture_output=True, text=True, timeout=300)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-3000:]
    assert r.stdout.strip() == "ok"
