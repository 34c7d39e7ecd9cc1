"""Kernel helpers compiled for the host and checked without a GPU:
- the find kernels' exact helpers (row masks, window test, triplet D^2 cut),
  bit for bit against brute force and the D^2 definition;
- the float-float arithmetic of the fit and the merge, against long double
  within counted error bounds (TwoSum exact, each operation a few u^2, the
  Cholesky chi2 within 64 kappa u^2);
- the distortion-map voxel of each cluster, bit for bit against the oracle's
  binning (an integer decided by FP32 arithmetic on both sides), on a central
  event and on clusters placed on and around the bin edges."""
import os
import shutil
import subprocess

import numpy as np
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


def _grid(which):
    """The default grid, or a seeded random one (band counts that divide
    152, uneven y and |z| bins, edges inside and outside the acceptance)."""
    from paper_2412_13755_gb300 import synth
    if which == 0:
        return synth.FIELD_GRID
    rng = np.random.default_rng(500 + which)
    n_y, n_z = int(rng.integers(1, 9)), int(rng.integers(1, 12))
    u_lo = -synth.TAN_HALF_SECTOR * rng.uniform(0.5, 1.2)
    return dict(n_band=int(rng.choice([1, 2, 4, 8, 19, 38, 76, 152])), n_y=n_y, n_z=n_z, u_lo=u_lo,
                u_inv=n_y / (2 * abs(u_lo) * rng.uniform(0.8, 1.3)), z_inv=n_z / rng.uniform(150.0, 300.0))


@pytest.mark.parametrize("which", [0, 1, 2, 3])
def test_field_voxel_matches_oracle(tmp_path, orc, which):
    from paper_2412_13755_gb300 import synth
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path / "field_voxel_host"
    subprocess.run([cxx, "-std=c++17", "-O2", "-ffp-contract=off",
                    "-I", os.path.join(ROOT, "paper_2412_13755_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "field_voxel_host.cpp"), "-o", str(exe)], check=True)
    ev = synth.central_event(n_tracks=1000, seed=77)
    G = _grid(which)
    # clusters on the bin edges of y / x and |z| and up to two float steps
    # either side of them
    rng = np.random.default_rng(78)
    m = 4000
    r_e = rng.integers(0, 152, m).astype(np.uint16)
    x_e = synth.ROW_X[r_e]
    ye = ((G["u_lo"] + rng.integers(0, G["n_y"] + 1, m) / G["u_inv"]) * x_e).astype(np.float32)
    ye = ye + rng.integers(-2, 3, m).astype(np.float32) * np.spacing(np.abs(ye))
    ze = (rng.integers(0, G["n_z"] + 1, m) / G["z_inv"] * rng.choice([-1.0, 1.0], m)).astype(np.float32)
    ze = ze + rng.integers(-2, 3, m).astype(np.float32) * np.spacing(np.abs(ze))
    y = np.concatenate([ev.y, ye]).astype(np.float32)
    z = np.concatenate([ev.z, ze]).astype(np.float32)
    row = np.concatenate([ev.row, r_e])
    sec = np.concatenate([ev.sector_of_cluster(), rng.integers(0, 36, m).astype(np.int32)])
    want, _ = orc.voxel_of(y, z, row, sec, orc.field_grid(**G))
    inp, out = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(inp, "wb") as f:
        f.write(np.int64(len(y)).tobytes())
        f.write(np.array([G["n_band"], G["n_y"], G["n_z"]], np.int32).tobytes())
        f.write(np.array([G["u_lo"], G["u_inv"], G["z_inv"]], np.float32).tobytes())
        f.write(synth.ROW_X.astype(np.float32).tobytes())
        for a, dt in ((y, np.float32), (z, np.float32), (row, np.uint16), (sec, np.int32)):
            f.write(np.ascontiguousarray(a, dt).tobytes())
    r = subprocess.run([str(exe), str(inp), str(out)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    got = np.fromfile(out, np.int32)
    assert np.array_equal(got, want)
    # the edge clusters do fall on both sides of the edges
    iy = (want[ev.n:] // G["n_z"]) % G["n_y"]
    iz = want[ev.n:] % G["n_z"]
    assert len(np.unique(iy)) == G["n_y"] and len(np.unique(iz)) == G["n_z"]
