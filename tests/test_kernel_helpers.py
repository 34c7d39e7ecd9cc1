"""Kernel helpers compiled for the host and checked without a GPU:
- the find kernels' exact helpers (row masks, window test, triplet D^2 cut),
  bit for bit against brute force and the D^2 definition;
- the float-float arithmetic of the fit and the merge, against long double
  within counted error bounds (TwoSum exact, each operation a few u^2, the
  Cholesky chi2 within 64 kappa u^2)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("program", ["kernel_helpers_host", "ff_host"])
def test_kernel_helpers_on_host(tmp_path, program):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path / program
    subprocess.run([cxx, "-std=c++17", "-O2", "-ffp-contract=off",
                    "-I", os.path.join(ROOT, "paper_2412_13755_gb300", "csrc"),
                    os.path.join(ROOT, "tests", program + ".cpp"), "-o", str(exe)],
                   check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout[-2000:]
