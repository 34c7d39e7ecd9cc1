"""The field calibration driver (calib.calibrate_field) on a stand-in for
the tracker whose chi2 is an exact quadratic: it must reach the minimiser of
chi2 + lam |F|^2 over the masked components (closed form solved here), with
a monotonically falling objective, and leave the unmasked components at
their start.  CPU only; the GPU run on generated distortions is in
tests/test_zz_gpu_field.py."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2412_13755_gb300 import calib, tpc  # noqa: E402


class QuadTracker:
    def __init__(self, nv, rng):
        n = 3 * nv
        B = rng.normal(size=(n, n // 2))
        self.A = B @ B.T / n + np.diag(rng.uniform(0.1, 10.0, n))
        self.Fs = rng.normal(0, 0.05, n)
        self.device = torch.device("cpu")
        self.calls = 0

    def adjoint_field(self, trk_off, trk_hits, n_tracks, grid, field, align=None):
        self.calls += 1
        x = field.cpu().numpy().reshape(-1) - self.Fs
        chi2 = float(x @ self.A @ x) + 1000.0
        g = 2.0 * self.A @ x
        return torch.tensor([chi2], dtype=torch.float64), None, torch.from_numpy(g.reshape(-1, 3))


def test_lbfgs_reaches_the_regularised_minimum(monkeypatch):
    rng = np.random.default_rng(3)
    nv = 20
    monkeypatch.setattr(tpc, "tpc_field_voxels", lambda grid: nv)
    tr = QuadTracker(nv, rng)
    mask = np.ones((nv, 3), bool)
    mask[:, 0] = False                      # x components stay at zero
    lam = 0.5
    seen = []
    F, hist = calib.calibrate_field(tr, None, None, 0, None, iters=80, lam=lam, mask=mask,
                                    callback=lambda it, f_, obj: seen.append((it, obj)))
    assert all(b <= a + 1e-9 for a, b in zip(hist, hist[1:]))
    # the callback sees every accepted iterate, numbered from 1
    assert [it for it, _ in seen] == list(range(1, len(hist))) and [o for _, o in seen] == hist[1:]
    assert np.all(F[:, 0] == 0)
    # closed form on the free components: (A_ff + lam I) x = A_ff Fs_f (+ coupling to fixed x = 0)
    free = mask.reshape(-1)
    A = tr.A
    Aff = A[np.ix_(free, free)]
    rhs = A[free] @ tr.Fs
    x = np.linalg.solve(Aff + lam * np.eye(free.sum()), rhs)
    err = np.abs(F.reshape(-1)[free] - x).max()
    print(f"{tr.calls} objective calls, max error {err:.2e}")
    assert err < 1e-6
