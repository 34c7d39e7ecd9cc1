"""Pins of the oracle's NEXT-4 step: the drift-time offset t0 as a sixth
state parameter and the association of the A- and C-side segments of
membrane-crossing tracks (time frames of continuous readout, Sec. 1 and
Sec. 4; the measurement model z' = z - v t0 on side A, z + v t0 on side C).

* Linear special case: with Bz = 0 and the prior variances of sin(phi) and
  q/pT zero, the joint fit of a straight track whose outer part lies on one
  side and inner part on the other is linear in (y0; z0, tan lambda, t0), so
  the Kalman filter must reproduce the closed-form weighted least squares
  with the prior as pseudo-measurements (normal equations solved here),
  state, covariance and chi2.
* Noise-free helix: a generated crossing track measured exactly gives back
  its t0 and helix.
* Association on the generator's own segments: every crossing track's two
  segments are paired, no pair joins two tracks, the t0 pulls have unit
  width and the joint fit's chi2 increase averages 4 (the four extra
  degrees of freedom of two separate five-parameter fits over one
  six-parameter fit).
* Without a vertex spread no track crosses and no pair is made; a single
  collision (t0 = 0) gives t0 consistent with zero.
"""
import numpy as np

from paper_2412_13755_gb300 import synth


def test_linear_case_equals_weighted_least_squares(orc):
    rng = np.random.default_rng(41)
    prior = [4.0, 4.0, 0.0, 0.25, 0.0]
    prm = orc.default_params(bz=0.0, prior=prior)
    sp = orc.default_sides_params()
    v, tp = sp.v_drift, sp.t0_prior
    sy2, sz2 = float(np.float32(0.01)), float(np.float32(0.0225))
    for trial in range(6):
        r_j = int(rng.integers(20, 130))             # last row of the inner part
        rows = np.arange(152, dtype=np.uint16)
        rows = rows[rng.uniform(size=152) > 0.05]
        n = len(rows)
        outer_side = int(rng.integers(0, 2))         # 0: outer part on A
        phi = 4
        sec = np.where(rows > r_j, phi + 18 * outer_side, phi + 18 * (1 - outer_side)).astype(np.int32)
        sgn = np.where(sec < 18, 1.0, -1.0)
        s_dir, tgl = rng.uniform(-0.3, 0.3), rng.uniform(-0.05, 0.05)
        t0_true = rng.uniform(0.0, 2000.0)
        x = synth.ROW_X[rows]
        c = np.sqrt(1 - s_dir ** 2)
        y = (rng.uniform(-5, 5) + (x - 85.0) * s_dir / c + rng.normal(0, 0.1, n)).astype(np.float32)
        z = (rng.uniform(-3, 3) + (x - 85.0) * tgl / c - sgn * v * t0_true
             + rng.normal(0, 0.15, n)).astype(np.float32)
        hits = np.arange(n - 1, -1, -1, dtype=np.int32)   # outermost first
        n_outer = int(np.sum(rows > r_j))
        t0_seed = t0_true + rng.normal(0, 0.3)
        res = orc.fit_t0(y, z, rows, sec, hits, n_outer, t0_seed, params=prm, sides=sp)
        assert res is not None
        p6, c6, chi2 = res
        # the prior centre: the outer part's three-cluster seed, its z made
        # the true z with the t0 seed
        x0, frame, ps = orc.seed(y, z, rows, sec, hits[:n_outer], True, params=prm)
        s = ps[2]
        cc = np.sqrt(1 - s * s)
        T = s / cc
        xj = x.astype(np.float64)
        yj, zj = y.astype(np.float64), z.astype(np.float64)
        # y: one unknown y0 at x0 with the seed's slope
        a = 1 / prior[0] + n / sy2
        b = ps[0] / prior[0] + np.sum(yj - (xj - x0) * T) / sy2
        y0 = b / a
        x_in = xj.min()
        # z: unknowns (z0, t, t0), h_j = (1, (x_j - x0)/c, -sgn_j v)
        H = np.stack([np.ones(n), (xj - x0) / cc, -sgn * v], 1)
        z_seed = ps[1] + (1.0 if sec[hits[0]] < 18 else -1.0) * v * t0_seed
        P = np.diag([1 / prior[1], 1 / prior[3], 1 / tp ** 2])
        A = P + H.T @ H / sz2
        th0 = np.array([z_seed, ps[3], t0_seed])
        th = np.linalg.solve(A, P @ th0 + H.T @ zj / sz2)
        G = np.array([[1.0, (x_in - x0) / cc, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
        Cz = G @ np.linalg.inv(A) @ G.T
        want = [y0 + (x_in - x0) * T, th[0] + th[1] * (x_in - x0) / cc, s, th[1], 0.0, th[2]]
        np.testing.assert_allclose(p6, want, rtol=1e-10, atol=1e-9)
        assert abs(p6[5] - t0_true) < 5 * np.sqrt(Cz[2, 2])
        # covariance (upper triangle row by row: 11 -> 6, 13 -> 8, 15 -> 10,
        # 33 -> 15, 35 -> 17, 55 -> 20; y: 00 -> 0)
        np.testing.assert_allclose(c6[[0, 6, 8, 10, 15, 17, 20]],
                                   [1 / a, Cz[0, 0], Cz[0, 1], Cz[0, 2], Cz[1, 1], Cz[1, 2], Cz[2, 2]],
                                   rtol=1e-8, atol=1e-15)
        # the minimum of the objective equals the filter's predicted-residual chi2
        ry = yj - (y0 + (xj - x0) * T)
        rz = zj - H @ th
        wls = ((y0 - ps[0]) ** 2 / prior[0] + (th - th0) @ P @ (th - th0) + np.sum(ry ** 2) / sy2
               + np.sum(rz ** 2) / sz2)
        np.testing.assert_allclose(chi2, wls, rtol=1e-9)


def _crossing_segments(ev):
    off, hits, ids, sides = ev.truth_segments()
    u, cnt = np.unique(ids, return_counts=True)
    return off, hits, ids, sides, set(u[cnt == 2].tolist())


def test_noise_free_crossing_helix(orc):
    ev = synth.membrane_frame(n_collisions=3, n_tracks=1000, noise=0.0, truth=True, seed=77)
    off, hits, ids, sides, crossing = _crossing_segments(ev)
    sec = ev.sector_of_cluster()
    sp = orc.default_sides_params()
    y = ev.y_true.astype(np.float32)
    sgn = np.where(sec < 18, 1.0, -1.0)
    done = 0
    for k in sorted(crossing)[:12]:
        segs = np.nonzero(ids == k)[0]
        parts = [hits[off[s]:off[s + 1]] for s in segs]
        parts.sort(key=lambda h: -int(ev.row[h[0]]))       # outer segment first
        h = np.concatenate(parts)
        t0 = ev.trk_t0[k]
        z = (ev.z_true - sgn * sp.v_drift * t0).astype(np.float32)
        res = orc.fit_t0(y, z, ev.row, sec, h, len(parts[0]), t0 + 0.05, sides=sp)
        assert res is not None
        p6, c6, chi2 = res
        c_in = h[-1]
        assert abs(p6[5] - t0) < 2e-4, (p6[5], t0)
        np.testing.assert_allclose(p6[:5], [ev.y_true[c_in], ev.z_true[c_in], ev.snp_true[c_in],
                                            ev.trk_tgl[k], ev.trk_q[k] / ev.trk_pt[k]],
                                   rtol=1e-4, atol=2e-4)
        assert chi2 < 1e-3 * len(h)
        done += 1
    assert done >= 8


def test_association_on_generated_segments(orc):
    ev = synth.membrane_frame(n_collisions=10, n_tracks=1000, truth=True)
    off, hits, ids, sides, crossing = _crossing_segments(ev)
    assert len(crossing) > 120
    r = orc.match_sides(ev.y, ev.z, ev.row, ev.evt_sector_off, ev.n_events, off, hits)
    p = r["partner"]
    pairs = [(i, int(p[i])) for i in range(len(p)) if p[i] > i]
    assert r["n_pairs"] == len(pairs)
    assert all(p[j] == i for i, j in pairs)              # symmetric
    assert all(ids[i] == ids[j] for i, j in pairs)       # no pair joins two tracks
    assert {int(ids[i]) for i, _ in pairs} == crossing   # every crossing track paired
    sel = np.array([i for i, _ in pairs])
    assert np.all(r["ndf"][sel] == 2 * (np.diff(off)[sel] + np.diff(off)[p[sel]]) - 6)
    pull = (r["t0"][sel] - ev.trk_t0[ids[sel]]) / np.sqrt(r["cov6"][sel, 20])
    print(f"{len(pairs)} pairs; t0 pull mean {pull.mean():.3f} std {pull.std():.3f}; "
          f"dchi2 mean {r['dchi2'][sel].mean():.2f}")
    k = np.sqrt(len(sel))
    assert abs(pull.mean()) < 3 / k
    assert abs(pull.std() - 1) < 0.15
    assert abs(r["dchi2"][sel].mean() - 4.0) < 3 * np.sqrt(8.0) / k


def test_no_crossing_without_vertex_spread(orc):
    ev = synth.generate([(2000, 0.1)], seed=5)
    toc, off, hits = orc.find_tracks(ev.y, ev.z, ev.row, ev.evt_sector_off, 1)
    r = orc.match_sides(ev.y, ev.z, ev.row, ev.evt_sector_off, 1, off, hits)
    assert r["n_pairs"] == 0 and np.all(r["partner"] == -1) and np.all(r["ndf"] == -1)


def test_single_collision_gives_zero_t0(orc):
    ev = synth.generate([(3000, 0.1)], seed=9, vz_sigma=synth.VZ_SIGMA, truth=True)
    off, hits, ids, sides, crossing = _crossing_segments(ev)
    r = orc.match_sides(ev.y, ev.z, ev.row, ev.evt_sector_off, 1, off, hits)
    sel = np.nonzero(r["partner"] >= 0)[0]
    assert len(sel) >= 2 * 0.9 * len(crossing) and len(crossing) > 20
    pull = r["t0"][sel] / np.sqrt(r["cov6"][sel, 20])
    assert np.all(np.abs(pull) < 5) and abs(pull.mean()) < 0.5
