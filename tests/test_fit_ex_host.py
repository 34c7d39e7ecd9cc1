"""The Kalman-filter variants' per-track functions (tpc_fit_ex.cuh)
compiled by nvcc for the host and run on the CPU, against the FP64 oracle on
the same hit lists, on tracks generated through material: the inward fit
with material, the outward refit and the smoother.  Both sides compute in
FP64 from the same definitions, written independently; the bar is 1e-9 of
max(|p_i|, s_i) for parameters, chi2 to 1e-9 relative, ndf equal, and
covariances to 1e-7 of sqrt(C_ii C_jj) (1e-6 for the smoothed ones): the
covariance recursions subtract nearly equal terms (C - K H C, and the
smoother's C_s - C_p), so the two orders of summation part in the 8th
digit of the smallest terms (measured 3e-9 for the fit, 4e-8 smoothed).
The GPU is held to the same bars."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2412_13755_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
SCALE = np.array([1.0, 1.0, 0.1, 0.1, 0.1])
DIAG = [0, 5, 9, 12, 14]
IU = [(i, j) for i in range(5) for j in range(i, 5)]
TOL = 1e-9
TOL_COV = 1e-7
TOL_SMOOTH_COV = 1e-6


@pytest.fixture(scope="module")
def fit_ex_host(tmp_path_factory):
    nvcc = NVCC if os.path.exists(NVCC) else shutil.which("nvcc")
    if nvcc is None:
        pytest.skip("no nvcc")
    exe = tmp_path_factory.mktemp("fitex") / "fit_ex_host"
    subprocess.run([nvcc, "-std=c++17", "-O2", "-Xcompiler", "-ffp-contract=off",
                    "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "paper_2412_13755_gb300", "csrc"),
                    "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "fit_ex_host.cu"), "-o", str(exe)],
                   check=True, capture_output=True)
    return exe


def lib_params():
    pytest.importorskip("torch")
    from paper_2412_13755_gb300 import tpc
    return tpc.default_params()


def run_host(exe, tmp_path, ev, off, hits, x0, eloss, mass, direction, smooth):
    p = lib_params()
    prm = np.array([p.sigma_y2, p.sigma_z2, p.snp_max, p.bz, p.seed_snp_max, p.seed_qpt_max,
                    *list(p.prior), x0, eloss, mass], np.float32)
    inp, out = tmp_path / "in.bin", tmp_path / "out.bin"
    T = len(off) - 1
    with open(inp, "wb") as f:
        f.write(np.array([ev.n, ev.n_events * 36, T], np.int64).tobytes())
        for a, dt in ((ev.y, np.float32), (ev.z, np.float32), (ev.row, np.uint16),
                      (ev.evt_sector_off, np.int64), (off, np.int32), (hits[:off[-1]], np.int32)):
            f.write(np.ascontiguousarray(a, dt).tobytes())
        f.write(prm.tobytes())
        f.write(np.array([direction, 1 if smooth else 0], np.int32).tobytes())
    r = subprocess.run([str(exe), str(inp), str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    raw = np.fromfile(out, np.float64)
    tab = raw[:22 * T].reshape(T, 22)
    sm = raw[22 * T:].reshape(-1, 20) if smooth else None
    return tab[:, :5], tab[:, 5:20], tab[:, 20], tab[:, 21].astype(np.int32), sm


def orc_params(orc, x0, eloss, mass):
    # the library takes the material in FP32: the oracle gets the same values
    return orc.default_params(mat_x_x0=float(np.float32(x0)), mat_eloss=float(np.float32(eloss)),
                              mass=float(np.float32(mass)))


def compare(par, cov, chi2, ndf, opar, ocov, ochi2, ondf, tol=TOL):
    assert np.array_equal(ndf <= 0, ondf <= 0)
    ok = ondf > 0
    assert np.array_equal(ndf[ok], ondf[ok])
    rel = np.abs(par - opar) / np.maximum(np.abs(opar), SCALE)
    d = ocov[:, DIAG]
    cs = np.stack([np.sqrt(np.abs(d[:, i] * d[:, j])) for i, j in IU], 1)
    crel = np.abs(cov - ocov) / np.maximum(cs, 1e-300)
    chrel = np.abs(chi2 - ochi2) / np.maximum(ochi2, 1.0)
    print(f"{ok.sum()} tracks: params {rel[ok].max():.2e} cov {crel[ok].max():.2e} chi2 {chrel[ok].max():.2e}")
    assert rel[ok].max() <= tol and crel[ok].max() <= TOL_COV and chrel[ok].max() <= tol
    return ok


@pytest.mark.parametrize("direction", [0, 1])
def test_material_fit_on_host(orc, fit_ex_host, tmp_path, direction):
    ev = synth.material_tracks(600, seed=81)
    off, hits, _ = ev.truth_tracks(n_min=10)
    x0, el, m = synth.MAT_X_X0_ROW, 3e-5, synth.PION_MASS
    par, cov, chi2, ndf, _ = run_host(fit_ex_host, tmp_path, ev, off, hits, x0, el, m, direction, False)
    opar, ocov, ochi2, ondf = orc.fit_tracks(ev.y, ev.z, ev.row, ev.sector_of_cluster(), off, hits,
                                             params=orc_params(orc, x0, el, m), reverse=direction == 1)
    assert compare(par, cov, chi2, ndf, opar, ocov, ochi2, ondf).sum() > 400


def test_smoother_on_host(orc, fit_ex_host, tmp_path):
    ev = synth.material_tracks(400, seed=82)
    off, hits, _ = ev.truth_tracks(n_min=10)
    x0, el, m = synth.MAT_X_X0_ROW, 3e-5, synth.PION_MASS
    par, cov, chi2, ndf, sm = run_host(fit_ex_host, tmp_path, ev, off, hits, x0, el, m, 0, True)
    osm, ochi2, ondf = orc.smooth_tracks(ev.y, ev.z, ev.row, ev.sector_of_cluster(), off, hits,
                                         params=orc_params(orc, x0, el, m))
    ok = np.repeat(ondf > 0, np.diff(off))
    rel = np.abs(sm[:, :5] - osm[:, :5]) / np.maximum(np.abs(osm[:, :5]), SCALE)
    d = osm[:, 5 + np.array(DIAG)]
    cs = np.stack([np.sqrt(np.abs(d[:, i] * d[:, j])) for i, j in IU], 1)
    crel = np.abs(sm[:, 5:] - osm[:, 5:]) / np.maximum(cs, 1e-300)
    print(f"{ok.sum()} smoothed states: params {rel[ok].max():.2e} cov {crel[ok].max():.2e}")
    assert rel[ok].max() <= TOL and crel[ok].max() <= TOL_SMOOTH_COV
    assert np.all(sm[~ok] == 0)


def test_no_material_matches_plain_fit_on_host(orc, fit_ex_host, tmp_path):
    """Without material the variants' inward fit is the plain fit."""
    ev = synth.central_event(n_tracks=500, noise=0.0, seed=83)
    off, hits, _ = ev.truth_tracks()
    par, cov, chi2, ndf, _ = run_host(fit_ex_host, tmp_path, ev, off, hits, 0.0, 0.0, synth.PION_MASS, 0, False)
    opar, ocov, ochi2, ondf = orc.fit_tracks(ev.y, ev.z, ev.row, ev.sector_of_cluster(), off, hits)
    compare(par, cov, chi2, ndf, opar, ocov, ochi2, ondf)
