"""The adjoint kernel's per-track function (adjoint_track in
tpc_adjoint.cuh: forward fit on corrected clusters with checkpoints and the
hand-written reverse sweep) compiled by nvcc for the host and run on the
CPU for every track, against the FP64 oracle's dual-number gradients, with
the GPU parity bars:
* alignment: chi2 within 1e-5 relative, d chi2 / d align within 1e-4
  norm-relative;
* distortion map (with an alignment): chi2 within 1e-5, d chi2 / d field
  within 1e-4 norm-relative, voxels without clusters exactly 0, and the
  field gradient summed per sector equal to the alignment gradient's shift
  components of the same run;
* a zero field gives the alignment run's chi2 and gradient exactly.
No GPU is needed; the program launches no kernel."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2412_13755_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
G = synth.FIELD_GRID


@pytest.fixture(scope="module")
def adjoint_host(tmp_path_factory):
    nvcc = NVCC if os.path.exists(NVCC) else shutil.which("nvcc")
    if nvcc is None:
        pytest.skip("no nvcc")
    exe = tmp_path_factory.mktemp("adj") / "adjoint_host"
    subprocess.run([nvcc, "-std=c++17", "-O2", "-Xcompiler", "-ffp-contract=off",
                    "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "paper_2412_13755_gb300", "csrc"),
                    "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "adjoint_host.cu"), "-o", str(exe)],
                   check=True, capture_output=True)
    return exe


@pytest.fixture(scope="module")
def sample():
    mis = synth.draw_misalignment(71)
    ev = synth.alignment_sample(n_tracks=400, seed=71, misalign=mis)
    off, hits, _ = ev.truth_tracks(n_min=10)
    return ev, off, hits, 0.5 * mis


def _run(exe, tmp_path, ev, off, hits, align, field=None):
    pytest.importorskip("torch")
    from paper_2412_13755_gb300 import tpc
    p = tpc.default_params()
    prm = np.array([p.sigma_y2, p.sigma_z2, p.snp_max, p.bz, p.seed_snp_max, p.seed_qpt_max,
                    p.fp64_ratio, p.fp64_det, *list(p.prior)], np.float32)
    nv = synth.n_voxels()
    fld = np.zeros((nv, 3)) if field is None else field
    inp, out = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(inp, "wb") as f:
        f.write(np.array([ev.n, ev.n_events * 36, len(off) - 1], np.int64).tobytes())
        for a, dt in ((ev.y, np.float32), (ev.z, np.float32), (ev.row, np.uint16),
                      (ev.evt_sector_off, np.int64), (off, np.int32), (hits[:off[-1]], np.int32),
                      (align, np.float64)):
            f.write(np.ascontiguousarray(a, dt).tobytes())
        f.write(np.array([field is not None, G["n_band"], G["n_y"], G["n_z"]], np.int32).tobytes())
        f.write(np.array([G["u_lo"], G["u_inv"], G["z_inv"]], np.float32).tobytes())
        f.write(np.ascontiguousarray(fld, np.float64).tobytes())
        f.write(prm.tobytes())
    r = subprocess.run([str(exe), str(inp), str(out)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    raw = np.fromfile(out, np.uint8)
    vals = raw[:-8].view(np.float64)
    status = raw[-8:].view(np.int32)
    assert status[0] == 0, status
    return vals[0], vals[1:217].copy(), vals[217:].reshape(nv, 3).copy()


def test_alignment_adjoint_on_host(orc, adjoint_host, tmp_path, sample):
    ev, off, hits, align = sample
    chi2, g, _ = _run(adjoint_host, tmp_path, ev, off, hits, align)
    o_chi2, o_g = orc.fit_adjoint(ev.y, ev.z, ev.row, ev.sector_of_cluster(), off, hits, align)
    rel_c = abs(chi2 - o_chi2) / o_chi2
    rel_g = np.linalg.norm(g - o_g) / np.linalg.norm(o_g)
    print(f"alignment: chi2 rel {rel_c:.2e}, gradient norm-rel {rel_g:.2e}")
    assert rel_c < 1e-5 and rel_g < 1e-4


def test_field_adjoint_on_host(orc, adjoint_host, tmp_path, sample):
    ev, off, hits, align = sample
    field = synth.draw_field(seed=72, sigma=0.02)
    chi2, g_al, g_f = _run(adjoint_host, tmp_path, ev, off, hits, align, field)
    o_chi2, o_g = orc.field_adjoint(ev.y, ev.z, ev.row, ev.sector_of_cluster(), off, hits,
                                    orc.field_grid(**G), field, align=align)
    rel_c = abs(chi2 - o_chi2) / o_chi2
    rel_g = np.linalg.norm(g_f - o_g) / np.linalg.norm(o_g)
    print(f"field: chi2 rel {rel_c:.2e}, field gradient norm-rel {rel_g:.2e}")
    assert rel_c < 1e-5 and rel_g < 1e-4
    empty = np.all(o_g == 0, axis=1)
    assert empty.any() and np.all(g_f[empty] == 0)
    per_sector = g_f.reshape(36, -1, 3).sum(axis=1)
    want = g_al.reshape(36, 6)[:, :3]
    np.testing.assert_allclose(per_sector, want, rtol=1e-9, atol=1e-9 * np.abs(want).max())


def test_zero_field_is_the_alignment_run(adjoint_host, tmp_path, sample):
    ev, off, hits, align = sample
    c_a, g_a, _ = _run(adjoint_host, tmp_path, ev, off, hits, align)
    c_f, g_f_al, g_f = _run(adjoint_host, tmp_path, ev, off, hits, align, np.zeros((synth.n_voxels(), 3)))
    assert c_f == c_a and np.array_equal(g_f_al, g_a)
