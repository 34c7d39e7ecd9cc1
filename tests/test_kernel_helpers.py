"""The find kernels' exact helpers (row masks, window test, triplet D^2
cut), compiled for the host and checked bit for bit against brute force and
against the D^2 definition; no GPU needed."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_kernel_helpers_on_host(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path / "kernel_helpers"
    subprocess.run([cxx, "-std=c++17", "-O2", "-ffp-contract=off",
                    "-I", os.path.join(ROOT, "paper_2412_13755_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "kernel_helpers_host.cpp"), "-o", str(exe)],
                   check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout[-2000:]
