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


def _excess(orc, ev, prm):
    """chi2 at the generated alignment minus chi2 at the Gauss-Newton minimum
    (4 steps, pseudo-inverse over the eigenvalues above 1e-9 of the largest),
    and the number of kept directions."""
    off, hits, _ = ev.truth_tracks(n_min=10)
    sec = ev.sector_of_cluster()
    gn = orc.gauss_newton(ev.y, ev.z, ev.row, sec, off, hits, ev.align, params=prm)
    w, V = np.linalg.eigh(gn)
    keep = w > 1e-9 * w[-1]
    P = (V[:, keep] / w[keep]) @ V[:, keep].T
    th = ev.align.copy()
    c0 = None
    for _ in range(4):
        c, g = orc.fit_adjoint(ev.y, ev.z, ev.row, sec, off, hits, th, params=prm)
        c0 = c if c0 is None else c0
        th = th - P @ g
    c = orc.fit_adjoint(ev.y, ev.z, ev.row, sec, off, hits, th, params=prm, want_grad=False)
    return c0 - c, int(keep.sum())


def test_noise_free_misaligned_sample_is_fitted_exactly(orc, monkeypatch):
    """With the smear switched off, the corrected clusters lie exactly on the
    fit's helices: the generator's displaced-plane crossing and the fit's
    rigid-body correction are the same model.  The seed is made from the
    uncorrected clusters, so its prior adds (p - p_seed)^T C0^-1 (p - p_seed)
    to every track's chi2; with the default prior that term alone is left at
    the generated alignment, and with a prior 1e4 times wider the summed chi2
    drops to FP32 storage rounding.  At zero correction it stays
    large either way."""
    monkeypatch.setattr(synth, "SIGMA_Y", 0.0)
    monkeypatch.setattr(synth, "SIGMA_Z", 0.0)
    ev, sec, off, hits, mis = _sample(n_tracks=500, seed=34)
    n_cl = int(off[-1])
    wide = orc.default_params(prior=[4e4, 4e4, 2.5e3, 2.5e3, 2.5e5])
    c_true, g = orc.fit_adjoint(ev.y, ev.z, ev.row, sec, off, hits, mis, params=wide)
    c_zero = orc.fit_adjoint(ev.y, ev.z, ev.row, sec, off, hits, np.zeros(216), params=wide,
                             want_grad=False)
    assert c_true < 1e-6 * n_cl, c_true
    assert c_zero > 1e6 * c_true
    # default prior: the prior term of the raw seed is what is left
    c_def = orc.fit_adjoint(ev.y, ev.z, ev.row, sec, off, hits, mis, want_grad=False)
    assert c_def > 1e3 * c_true and c_def < 1e-2 * c_zero


def test_excess_chi2_scales_with_the_noise_variance(orc, monkeypatch):
    """The chi2 that the alignment minimum gains over the generated alignment
    is the number of fitted directions plus a part that grows with the track
    count.  That part scales with the measurement variance (an O(sigma^2)
    bias of the joint minimum over 5 parameters per track and the shared
    alignment), not inversely to it as a generator/fit mismatch of fixed
    size would: halving the smear divides it by about 4."""
    per = []
    for f in (1.0, 0.5):
        monkeypatch.setattr(synth, "SIGMA_Y", 0.1 * f)
        monkeypatch.setattr(synth, "SIGMA_Z", 0.15 * f)
        prm = orc.default_params(sigma_y2=(0.1 * f) ** 2, sigma_z2=(0.15 * f) ** 2)
        ev = synth.alignment_sample(n_tracks=8000, seed=35, misalign=np.zeros(216))
        ex, kept = _excess(orc, ev, prm)
        per.append((ex - kept) / 8000)
    print(f"excess beyond the fitted directions per track: {per[0]:.4f} (nominal smear), "
          f"{per[1]:.4f} (half the smear)")
    assert per[0] > 0.03
    assert 2.5 < per[0] / per[1] < 6.0
