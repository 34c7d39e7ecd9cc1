"""The autograd wrapper (TPCChi2) on a stand-in tracker whose chi2 is an
exact quadratic in the 216 corrections: one library call per forward (with
the gradient only when the corrections require one), none in backward, and the gradient
torch returns equals the quadratic's.  CPU only; the GPU run is in
tests/test_gpu_adjoint.py."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2412_13755_gb300.autograd import TPCChi2  # noqa: E402


class QuadTracker:
    def __init__(self, rng):
        B = rng.normal(size=(216, 216))
        self.A = B @ B.T / 216 + np.eye(216)
        self.calls = []

    def adjoint(self, trk_off, trk_hits, n_tracks, align, want_grad=True):
        self.calls.append(want_grad)
        x = align.numpy()
        chi2 = torch.tensor([float(x @ self.A @ x)], dtype=torch.float64)
        return chi2, (torch.from_numpy(2.0 * self.A @ x) if want_grad else None)


def test_one_call_per_step_and_the_gradient():
    rng = np.random.default_rng(5)
    tr = QuadTracker(rng)
    a = torch.from_numpy(rng.normal(0, 0.01, 216)).requires_grad_(True)
    loss = 2.5 * TPCChi2.apply(a, tr, None, None, 0)
    loss.backward()
    assert tr.calls == [True]
    np.testing.assert_allclose(a.grad.numpy(), 2.5 * 2.0 * tr.A @ a.detach().numpy(), rtol=1e-12)
    TPCChi2.apply(a.detach(), tr, None, None, 0)   # no gradient wanted: forward sweep alone
    assert tr.calls == [True, False]
    with pytest.raises(TypeError):
        TPCChi2.apply(a.float(), tr, None, None, 0)
