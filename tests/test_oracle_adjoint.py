"""Pins of the oracle's alignment gradient (S6).

The gradient of the total chi2 with respect to the 216 per-sector rigid-body
corrections, computed by forward-mode dual numbers through the FP64 fit, is
compared with FP64 central finite differences of the same total chi2
(h = 1e-6 cm / rad), parameter by parameter.  The Gauss-Newton matrix must be
symmetric positive semi-definite with the 12 rigid-body null modes (a common
transform of all sectors on one side leaves every chi2 unchanged).
"""
import numpy as np

from paper_2412_13755_gb300 import synth


def _sample(n_tracks=300, seed=31):
    mis = synth.draw_misalignment(seed)
    ev = synth.alignment_sample(n_tracks=n_tracks, seed=seed, misalign=mis)
    off, hits, _ = ev.truth_tracks(n_min=10)
    return ev, ev.sector_of_cluster(), off, hits, mis


def test_gradient_matches_central_differences(orc):
    ev, sec, off, hits, mis = _sample()
    align = mis * 0.5  # partially corrected: a generic point with a large gradient
    chi2, g = orc.fit_adjoint(ev.y, ev.z, ev.row, sec, off, hits, align)
    assert np.isfinite(chi2) and np.abs(g).max() > 1.0
    h = 1e-6
    fd = np.zeros(216)
    for i in range(216):
        ap, am = align.copy(), align.copy()
        ap[i] += h
        am[i] -= h
        fp = orc.fit_adjoint(ev.y, ev.z, ev.row, sec, off, hits, ap, want_grad=False)
        fm = orc.fit_adjoint(ev.y, ev.z, ev.row, sec, off, hits, am, want_grad=False)
        fd[i] = (fp - fm) / (2 * h)
    scale = np.abs(g).max()
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-6 * scale)


def test_chi2_matches_fit_sum(orc):
    ev, sec, off, hits, mis = _sample(n_tracks=200, seed=32)
    chi2 = orc.fit_adjoint(ev.y, ev.z, ev.row, sec, off, hits, mis, want_grad=False)
    par, cov, c2, ndf = orc.fit_tracks(ev.y, ev.z, ev.row, sec, off, hits, align=mis)
    assert abs(chi2 - c2[ndf > 0].sum()) <= 1e-9 * chi2


def test_gauss_newton_null_modes(orc):
    ev, sec, off, hits, mis = _sample(n_tracks=600, seed=33)
    gn = orc.gauss_newton(ev.y, ev.z, ev.row, sec, off, hits, mis)
    assert np.allclose(gn, gn.T, rtol=1e-9, atol=1e-9 * np.abs(gn).max())
    ev_ = np.linalg.eigvalsh(gn)
    assert ev_.min() > -1e-9 * ev_.max()
    # an infinitesimal common translation of all A-side sectors in the global
    # frame is a null direction: build it from the sector frames
    v = np.zeros(216)
    for s in range(18):
        a = synth.sector_alpha(s)
        v[s * 6 + 0] = np.cos(a)       # global X shift seen in the local frame
        v[s * 6 + 1] = -np.sin(a)
    assert v @ gn @ v <= 1e-6 * np.abs(gn).max() * (v @ v)
