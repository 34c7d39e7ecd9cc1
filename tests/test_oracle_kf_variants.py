"""Pins of the oracle's Kalman-filter variants (material in the pad-row
planes: multiple-scattering process noise and mean energy loss; the
Rauch-Tung-Striebel smoother; the outward refit), against an independent
generator and exact identities.

The generator (synth.material_tracks) steps exact helices from plane to
plane and draws, at every plane a track crosses, two Gaussian scattering
angles of the Highland width and the mean energy loss; the oracle's fit
never sees those draws.  So:

* with the material in the fit, the pulls of the five parameters at the
  innermost cluster (the state arriving there) are unit-width; without it
  they are far too wide (multiple scattering dominates tan lambda);
* the smoothed states at every cluster have unit-width pulls too;
* the smoothed state at the innermost cluster is the filtered one, bit for
  bit (the smoother starts there);
* without material the smoothed state at every cluster is the final
  filtered state moved back along the helix (to 1e-9 of its own sigma);
* the energy-loss correction removes the momentum bias the loss causes:
  with it the charge-signed q/pT pull is the same as on tracks without any
  material (the extended filter's own small curvature bias), without it the
  bias grows with the loss;
* the outward refit (the fit in the direction of motion) gives unit-width
  pulls at the outermost cluster.
"""
import numpy as np
import pytest

from paper_2412_13755_gb300 import synth

DIAG = [0, 5, 9, 12, 14]


def _mat_params(orc, x0=synth.MAT_X_X0_ROW, el=synth.MAT_ELOSS_ROW):
    return orc.default_params(mat_x_x0=x0, mat_eloss=el, mass=synth.PION_MASS)


def _truth(ev, idx):
    return np.stack([ev.y_true[idx], ev.z_true[idx], ev.snp_true[idx], ev.tgl_true[idx],
                     ev.qpt_true[idx]], 1)


@pytest.fixture(scope="module")
def mat_event():
    ev = synth.material_tracks(3000)
    off, hits, _ = ev.truth_tracks(n_min=20)
    return ev, ev.sector_of_cluster(), off, hits


def test_material_pulls(orc, mat_event):
    ev, sec, off, hits = mat_event
    truth = _truth(ev, hits[off[1:] - 1])
    res = {}
    for lab, prm in (("material", _mat_params(orc)), ("none", orc.default_params())):
        par, cov, chi2, ndf = orc.fit_tracks(ev.y, ev.z, ev.row, sec, off, hits, params=prm)
        ok = ndf > 0
        assert ok.mean() > 0.99
        pull = ((par - truth) / np.sqrt(cov[:, DIAG]))[ok]
        res[lab] = (pull.mean(0), pull.std(0))
        print(lab, "mean", np.round(pull.mean(0), 3), "std", np.round(pull.std(0), 3))
    mu, sd = res["material"]
    assert np.all(np.abs(mu) < 0.07), mu
    assert np.all((sd > 0.95) & (sd < 1.05)), sd
    assert res["none"][1][3] > 1.5  # tan lambda: scattering dominates


def test_smoother_pulls_and_start(orc, mat_event):
    ev, sec, off, hits = mat_event
    prm = _mat_params(orc)
    sm, chi2, ndf = orc.smooth_tracks(ev.y, ev.z, ev.row, sec, off, hits, params=prm)
    par, cov, fchi2, fndf = orc.fit_tracks(ev.y, ev.z, ev.row, sec, off, hits, params=prm)
    ok = ndf > 0
    assert np.array_equal(ndf, fndf) and np.array_equal(chi2, fchi2)
    inner = off[1:] - 1
    assert np.array_equal(sm[inner[ok], :5], par[ok])
    assert np.array_equal(sm[inner[ok], 5:], cov[ok])
    rows_ok = np.repeat(ok, np.diff(off))
    pull = ((sm[:, :5] - _truth(ev, hits)) / np.sqrt(sm[:, 5 + np.array(DIAG)]))[rows_ok]
    print("smoothed pulls mean", np.round(pull.mean(0), 3), "std", np.round(pull.std(0), 3))
    assert np.all(np.abs(pull.mean(0)) < 0.07)
    assert np.all((pull.std(0) > 0.95) & (pull.std(0) < 1.05))


def test_smoother_without_material_is_the_moved_final_state(orc):
    ev = synth.material_tracks(300, x_x0_row=0.0, eloss_row=0.0, seed=79)
    sec = ev.sector_of_cluster()
    off, hits, _ = ev.truth_tracks(n_min=20)
    prm = orc.default_params()
    sm, _, ndf = orc.smooth_tracks(ev.y, ev.z, ev.row, sec, off, hits, params=prm)
    par, _, _, _ = orc.fit_tracks(ev.y, ev.z, ev.row, sec, off, hits, params=prm)
    worst = 0.0
    for t in np.flatnonzero(ndf > 0)[:150]:
        inner = hits[off[t + 1] - 1]
        x1 = synth.ROW_X[ev.row[inner]]
        for j in range(off[t], off[t + 1]):
            h = hits[j]
            q = orc.propagate(x1, int(sec[inner]), par[t], float(synth.ROW_X[ev.row[h]]), int(sec[h]))[0]
            sig = np.sqrt(sm[j, 5 + np.array(DIAG)])
            worst = max(worst, float(np.max(np.abs(sm[j, :5] - q) / sig)))
    assert worst < 1e-9, worst


def test_energy_loss_correction(orc):
    def signed_w_pull(ev, prm):
        sec = ev.sector_of_cluster()
        off, hits, _ = ev.truth_tracks(n_min=20)
        truth = _truth(ev, hits[off[1:] - 1])
        par, cov, _, ndf = orc.fit_tracks(ev.y, ev.z, ev.row, sec, off, hits, params=prm)
        ok = ndf > 0
        pull = (par[ok, 4] - truth[ok, 4]) / np.sqrt(cov[ok, 14])
        return float(np.mean(pull * np.sign(truth[ok, 4])))

    base = signed_w_pull(synth.material_tracks(6000, x_x0_row=0.0, eloss_row=0.0, seed=78),
                         orc.default_params())
    ev = synth.material_tracks(6000, eloss_row=1e-4, seed=78)
    corrected = signed_w_pull(ev, _mat_params(orc, el=1e-4))
    uncorrected = signed_w_pull(ev, _mat_params(orc, el=0.0))
    print(f"signed q/pT pull: no material {base:.3f}, loss corrected {corrected:.3f}, "
          f"loss ignored {uncorrected:.3f}")
    assert abs(corrected - base) < 0.06
    assert uncorrected - base > 0.25


def test_outward_refit_pulls(orc, mat_event):
    ev, sec, off, hits = mat_event
    prm = _mat_params(orc)
    par, cov, chi2, ndf = orc.fit_tracks(ev.y, ev.z, ev.row, sec, off, hits, params=prm, reverse=True)
    ok = ndf > 0
    truth = _truth(ev, hits[off[:-1]])
    pull = ((par - truth) / np.sqrt(cov[:, DIAG]))[ok]
    print("outward refit pulls mean", np.round(pull.mean(0), 3), "std", np.round(pull.std(0), 3))
    assert np.all(np.abs(pull.mean(0)) < 0.07)
    assert np.all((pull.std(0) > 0.95) & (pull.std(0) < 1.05))
