"""Pins of the oracle's helix transport (S5) against closed forms.

* The propagated state is compared with the crossings of the same helix with
  the row planes computed independently in the global frame by the event
  generator (circle / line intersection), for same- and adjacent-sector
  propagations in both directions.
* The analytic Jacobian (including the frame rotation at a sector change)
  is compared with FP64 central finite differences of the propagation.
"""
import numpy as np
import pytest

from paper_2412_13755_gb300 import synth


def _truth_state(ev, i, tid):
    return np.array([ev.y_true[i], ev.z_true[i], ev.snp_true[i], ev.trk_tgl[tid],
                     ev.trk_q[tid] / ev.trk_pt[tid]])


def test_transport_matches_global_helix(orc):
    ev = synth.central_event(n_tracks=200, noise=0.0, truth=True, seed=7)
    sec = ev.sector_of_cluster()
    worst = 0.0
    n = 0
    for tid in range(200):
        idx = np.nonzero(ev.mc_track == tid)[0]
        if len(idx) < 3:
            continue
        idx = idx[np.argsort(ev.arc_true[idx])]
        pairs = [(idx[0], idx[-1]), (idx[-1], idx[0]), (idx[len(idx) // 2], idx[0]),
                 (idx[1], idx[2])]
        for a, b in pairs:
            dphi = (sec[b] % 18 - sec[a] % 18) % 18
            if dphi not in (0, 1, 17):
                continue
            r = orc.propagate(synth.ROW_X[ev.row[a]], int(sec[a]), _truth_state(ev, a, tid),
                              synth.ROW_X[ev.row[b]], int(sec[b]))
            assert r is not None
            tb = _truth_state(ev, b, tid)
            worst = max(worst, np.abs(r[0] - tb).max())
            n += 1
    assert n > 300
    assert worst < 1e-9, worst


def test_transport_zero_length_is_identity(orc):
    p = np.array([3.0, -20.0, 0.3, 0.5, 1.7])
    r = orc.propagate(150.0, 4, p, 150.0, 4)
    assert np.array_equal(r[0], p)
    assert np.array_equal(r[1], np.eye(5))


@pytest.mark.parametrize("case", [
    (120.0, 3, [2.0, 40.0, 0.2, 0.6, 1.5], 125.3, 3),     # outward, same frame
    (200.0, 7, [-5.0, -80.0, -0.4, -0.9, -2.5], 190.0, 7),  # inward
    (180.0, 5, [28.0, 10.0, 0.35, 0.1, 0.8], 182.0, 6),   # across a boundary
    (181.0, 6, [-30.5, 10.0, -0.1, 0.1, 0.8], 179.0, 5),  # back across
    (100.0, 0, [12.0, 5.0, 0.6, 0.2, 4.5], 100.5, 0),     # low pT, short step
    (100.0, 20, [0.0, -5.0, 0.0, -0.2, 0.0], 110.0, 20),  # straight line
])
def test_jacobian_matches_finite_differences(orc, case):
    x1, s1, p, x2, s2 = case
    p = np.array(p, dtype=np.float64)
    base = orc.propagate(x1, s1, p, x2, s2)
    assert base is not None
    _, J, dx1, dx2 = base
    scale = np.array([1.0, 1.0, 0.1, 0.1, 0.1])
    for j in range(5):
        h = 1e-6 * scale[j]
        pp, pm = p.copy(), p.copy()
        pp[j] += h
        pm[j] -= h
        fd = (orc.propagate(x1, s1, pp, x2, s2)[0] - orc.propagate(x1, s1, pm, x2, s2)[0]) / (2 * h)
        np.testing.assert_allclose(J[:, j], fd, rtol=1e-6, atol=1e-8 * max(1.0, np.abs(fd).max()))
    h = 1e-6
    fd2 = (orc.propagate(x1, s1, p, x2 + h, s2)[0] - orc.propagate(x1, s1, p, x2 - h, s2)[0]) / (2 * h)
    np.testing.assert_allclose(dx2, fd2, rtol=1e-6, atol=1e-9)
    fd1 = (orc.propagate(x1 + h, s1, p, x2, s2)[0] - orc.propagate(x1 - h, s1, p, x2, s2)[0]) / (2 * h)
    np.testing.assert_allclose(dx1, fd1, rtol=1e-6, atol=1e-9)


def test_sign_convention_positive_charge_bends_clockwise(orc):
    # d(sin phi)/dx = -k with k = K Bz q/pT: a positive track loses sin phi outward
    r = orc.propagate(100.0, 0, np.array([0.0, 0.0, 0.0, 0.0, 1.0]), 110.0, 0)
    assert r[0][2] < 0 and r[0][0] < 0
    k = 2.99792458e-3 * 0.5 * 1.0
    assert abs(r[0][2] - (-k * 10.0)) < 1e-15
