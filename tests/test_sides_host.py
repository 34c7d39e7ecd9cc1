"""The A/C-side association's per-pair functions (tpc_sides.cuh: the
junction test, the six-parameter fit with t0, the chi2 increase over the
two end fits of tpc_fit_ex.cuh) compiled by nvcc for the host and run on the
CPU over the pairs the FP64 oracle accepts on a membrane-crossing frame.
Both sides compute in FP64 from the same definitions, written
independently: t0, the six parameters and chi2 agree to 1e-9 relative
(of max(|p_i|, s_i) for parameters), the covariance to 1e-7 of
sqrt(C_ii C_jj) (the covariance recursion subtracts nearly equal terms),
and every accepted pair passes the junction gates as computed here."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2412_13755_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
SCALE = np.array([1.0, 1.0, 0.1, 0.1, 0.1, 0.01])
IU6 = [(i, j) for i in range(6) for j in range(i, 6)]
DIAG6 = [IU6.index((i, i)) for i in range(6)]


@pytest.fixture(scope="module")
def sides_host(tmp_path_factory):
    nvcc = NVCC if os.path.exists(NVCC) else shutil.which("nvcc")
    if nvcc is None:
        pytest.skip("no nvcc")
    exe = tmp_path_factory.mktemp("sides") / "sides_host"
    subprocess.run([nvcc, "-std=c++17", "-O2", "-Xcompiler", "-ffp-contract=off",
                    "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "paper_2412_13755_gb300", "csrc"),
                    "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "sides_host.cu"), "-o", str(exe)],
                   check=True, capture_output=True)
    return exe


def run_host(exe, tmp_path, ev, off, hits, pairs, sp):
    pytest.importorskip("torch")
    from paper_2412_13755_gb300 import tpc
    p = tpc.default_params()
    prm = np.array([p.sigma_y2, p.sigma_z2, p.snp_max, p.bz, p.seed_snp_max, p.seed_qpt_max,
                    *list(p.prior)], np.float32)
    inp, out = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(inp, "wb") as f:
        f.write(np.array([ev.n, ev.n_events * 36, len(off) - 1, len(pairs)], np.int64).tobytes())
        for a, dt in ((ev.y, np.float32), (ev.z, np.float32), (ev.row, np.uint16),
                      (ev.evt_sector_off, np.int64), (off, np.int32), (hits, np.int32),
                      (np.asarray(pairs).reshape(-1), np.int32)):
            f.write(np.ascontiguousarray(a, dt).tobytes())
        f.write(prm.tobytes())
        f.write(np.array([sp.t0_prior, sp.v_drift], np.float64).tobytes())
    subprocess.run([str(exe), str(inp), str(out)], check=True)
    return np.fromfile(out, np.float64).reshape(len(pairs), 34)


def test_pairs_agree_with_the_oracle(orc, sides_host, tmp_path):
    ev = synth.membrane_frame(n_collisions=6, n_tracks=1000, truth=True, seed=123)
    off, hits, ids, sides = ev.truth_segments()
    sp = orc.default_sides_params()
    r = orc.match_sides(ev.y, ev.z, ev.row, ev.evt_sector_off, ev.n_events, off, hits, sides=sp)
    p = r["partner"]
    rows_out = ev.row[hits[off[:-1]]]
    pairs = []
    for i in range(len(p)):
        if p[i] > i:
            a, b = i, int(p[i])
            if rows_out[a] > rows_out[b]:     # inner first
                a, b = b, a
            pairs.append((a, b))
    assert len(pairs) > 60
    h = run_host(sides_host, tmp_path, ev, off, hits, pairs, sp)
    assert np.all(h[:, 0] == 1.0)
    assert np.all(h[:, 1] <= sp.chi2_junction) and np.all(np.abs(h[:, 2]) <= sp.z_membrane)
    sel = np.array([a for a, _ in pairs])
    o6, oc, oc2, od = r["params6"][sel], r["cov6"][sel], r["chi2"][sel], r["dchi2"][sel]
    s = np.sqrt(oc[:, DIAG6])
    err_p = np.abs(h[:, 4:10] - o6) / np.maximum(np.abs(o6), s)
    sd = np.sqrt(np.abs(oc[:, [DIAG6[i] for i, _ in IU6]] * oc[:, [DIAG6[j] for _, j in IU6]]))
    err_c = np.abs(h[:, 10:31] - oc) / sd
    err_x = np.abs(h[:, 31] - oc2) / oc2
    err_d = np.abs(h[:, 32] - od) / np.maximum(np.abs(od), 1.0)
    print(f"{len(pairs)} pairs: params {err_p.max():.2e} cov {err_c.max():.2e} chi2 {err_x.max():.2e} "
          f"dchi2 {err_d.max():.2e}")
    assert err_p.max() < 1e-9 and err_x.max() < 1e-9 and err_d.max() < 1e-8
    assert err_c.max() < 1e-7
