"""GPU alignment gradient (S6) against the oracle.

* chi2 total: GPU (FP32 fits, FP64 sum) vs FP64 oracle.
* gradient: the hand-written reverse sweep vs the oracle's exact gradient
  (dual numbers) and vs FP64 central finite differences of the oracle chi2.
* torch.autograd.Function wrapper: backward equals the library gradient.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2412_13755_gb300 import synth, tpc  # noqa: E402
from paper_2412_13755_gb300.autograd import TPCChi2  # noqa: E402
from gpu_util import to_dev  # noqa: E402


def _setup(n_tracks, seed):
    mis = synth.draw_misalignment(seed)
    ev = synth.alignment_sample(n_tracks=n_tracks, seed=seed, misalign=mis)
    off, hits, _ = ev.truth_tracks(n_min=10)
    tr = tpc.Tracker(ev.n, 1)
    y, z, row, eo = to_dev(ev)
    tr.load(y, z, row, eo, 1)
    tr._keep = (y, z, row, eo)
    return ev, off, hits, mis, tr


def test_adjoint_matches_oracle(orc):
    ev, off, hits, mis, tr = _setup(2000, 41)
    sec = ev.sector_of_cluster()
    align = 0.5 * mis
    d_off = torch.from_numpy(off).cuda()
    d_hits = torch.from_numpy(hits).cuda()
    a = torch.from_numpy(align).cuda()
    chi2, grad = tr.adjoint(d_off, d_hits, len(off) - 1, a)
    torch.cuda.synchronize()
    tr.check()
    o_chi2, o_grad = orc.fit_adjoint(ev.y, ev.z, ev.row, sec, off, hits, align)
    g = grad.cpu().numpy()
    rel_chi2 = abs(chi2.item() - o_chi2) / o_chi2
    rel_g = np.linalg.norm(g - o_grad) / np.linalg.norm(o_grad)
    print(f"chi2 rel {rel_chi2:.2e}  grad norm-rel {rel_g:.2e}  |g| {np.linalg.norm(o_grad):.3e}")
    assert rel_chi2 < 1e-5
    assert rel_g < 1e-4


def test_adjoint_matches_finite_differences(orc):
    ev, off, hits, mis, tr = _setup(300, 42)
    sec = ev.sector_of_cluster()
    align = 0.3 * mis
    a = torch.from_numpy(align).cuda()
    chi2, grad = tr.adjoint(torch.from_numpy(off).cuda(), torch.from_numpy(hits).cuda(),
                            len(off) - 1, a)
    g = grad.cpu().numpy()
    h = 1e-6
    fd = np.zeros(216)
    for i in range(216):
        ap, am = align.copy(), align.copy()
        ap[i] += h
        am[i] -= h
        fd[i] = (orc.fit_adjoint(ev.y, ev.z, ev.row, sec, off, hits, ap, want_grad=False)
                 - orc.fit_adjoint(ev.y, ev.z, ev.row, sec, off, hits, am, want_grad=False)) / (2 * h)
    touched = np.abs(fd) > 0
    rel = np.linalg.norm(g - fd) / np.linalg.norm(fd)
    print(f"grad vs FD norm-rel {rel:.2e}")
    assert rel < 1e-4
    assert np.all(g[~touched] == 0)


def test_autograd_function():
    ev, off, hits, mis, tr = _setup(500, 43)
    d_off = torch.from_numpy(off).cuda()
    d_hits = torch.from_numpy(hits).cuda()
    a = torch.from_numpy(0.2 * mis).cuda().requires_grad_(True)
    loss = TPCChi2.apply(a, tr, d_off, d_hits, len(off) - 1)
    loss.backward()
    _, g = tr.adjoint(d_off, d_hits, len(off) - 1, a.detach())
    assert torch.allclose(a.grad, g, rtol=1e-12, atol=0)
    loss2 = 3.0 * TPCChi2.apply(a, tr, d_off, d_hits, len(off) - 1)
    a.grad = None
    loss2.backward()
    assert torch.allclose(a.grad, 3.0 * g)
