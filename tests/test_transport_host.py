"""The fit's device transport (kf_move<float> in tpc_dev.cuh, the helix move
with frame rotation and its analytic Jacobian) compiled by nvcc for the host
and run on the CPU, against the oracle's FP64 transport from the same FP32
start.  Random moves between pad-row planes of one sector and of
phi-adjacent sectors, in both directions:
* both refuse the same moves (|sin phi| reaching the limit);
* each parameter within 1e-5 of max(|p_in|, |p_out|, s) + |p_out - p_in|,
  s = (1 cm, 1 cm, 0.1, 0.1, 0.1): FP32 rounding of values and steps;
* each Jacobian row within 1e-5 of its largest entry (at least 1).
No GPU is needed; the program launches no kernel."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2412_13755_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
SCALE = np.array([1.0, 1.0, 0.1, 0.1, 0.1])


def _cases(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        s1 = int(rng.integers(0, 36))
        s2 = s1 if i % 2 == 0 else (s1 // 18) * 18 + (s1 % 18 + int(rng.choice([-1, 1]))) % 18
        r1, r2 = rng.integers(0, 152, 2)
        x1, x2 = synth.ROW_X[r1], synth.ROW_X[r2]
        p = np.array([rng.uniform(-0.8, 0.8) * x1 * synth.TAN_HALF_SECTOR, rng.uniform(-200, 200),
                      rng.uniform(-0.6, 0.6), rng.uniform(-1.2, 1.2), rng.uniform(-3, 3)])
        out.append((x1, p.astype(np.float32).astype(np.float64), x2, s1, s2))
    return out


def test_device_transport_matches_oracle(tmp_path, orc):
    if not os.path.exists(NVCC) and shutil.which("nvcc") is None:
        pytest.skip("no nvcc")
    nvcc = NVCC if os.path.exists(NVCC) else shutil.which("nvcc")
    exe = tmp_path / "transport_host"
    subprocess.run([nvcc, "-std=c++17", "-O2", "-Xcompiler", "-ffp-contract=off",
                    "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "paper_2412_13755_gb300", "csrc"),
                    "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "transport_host.cu"), "-o", str(exe)],
                   check=True, capture_output=True)
    cases = _cases(4000, 5)
    kb = np.float32(synth.KAPPA * synth.BZ)
    snp = np.float32(0.999)
    inp, out = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(inp, "wb") as f:
        f.write(np.int64(len(cases)).tobytes())
        for x1, p, x2, s1, s2 in cases:
            f.write(np.float64(x1).tobytes())
            f.write(p.tobytes())
            f.write(np.float64(x2).tobytes())
            f.write(np.array([s1, s2], np.int32).tobytes())
            f.write(np.array([kb, snp], np.float32).tobytes())
    r = subprocess.run([str(exe), str(inp), str(out)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    raw = np.fromfile(out, np.uint8).reshape(len(cases), 4 + 240)
    ok = raw[:, :4].copy().view(np.int32)[:, 0]
    vals = raw[:, 4:].copy().view(np.float64)
    prm = orc.default_params(snp_max=0.999)
    n_ok = n_rot = 0
    worst_p = worst_j = 0.0
    for i, (x1, p, x2, s1, s2) in enumerate(cases):
        o = orc.propagate(x1, s1, p, x2, s2, params=prm)
        assert (o is None) == (ok[i] == 0), i
        if o is None:
            continue
        po, J = o[0], o[1]
        scale = np.maximum(np.maximum(np.abs(p), np.abs(po)), SCALE) + np.abs(po - p)
        worst_p = max(worst_p, float(np.max(np.abs(vals[i, :5] - po) / scale)))
        row = np.maximum(np.abs(J).max(axis=1), 1.0)[:, None]
        worst_j = max(worst_j, float(np.max(np.abs(vals[i, 5:].reshape(5, 5) - J) / row)))
        n_ok += 1
        n_rot += s1 != s2
    print(f"{n_ok} moves ({n_rot} with rotation): parameters {worst_p:.2e}, Jacobian {worst_j:.2e}")
    assert n_ok > 3500 and n_rot > 1500
    assert worst_p <= 1e-5 and worst_j <= 1e-5
