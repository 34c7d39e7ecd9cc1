"""Pins of the oracle's clusterizer (NEXT-2: peaks and centroids of
pad-time digits).

* The rule restated independently here with numpy (shifted views of the
  zero-padded arrays for the raster peak test, sliding 5 x 5 sums in int64,
  the positions in numpy float32, one rounding per operation) gives the same
  clusters bit for bit on random digit fields.
* A plateau of equal counts yields exactly one peak, its first digit in
  raster order; two deposits four pads apart yield two.
* On digitized events the clusters come back where they were generated:
  isolated ones within 0.05 cm in y and z (the 5 x 5 window holds all but
  ~1e-3 of a deposit); of the clusters of charge >= 20 (every signal
  cluster; noise clusters below it may stay under the peak threshold),
  >= 99% of those isolated by 3 cm and >= 93% of all are found within
  0.3 cm (the rest merge with a neighbour: their nearest other cluster is
  ~1.4 cm away, two pads).
"""
import numpy as np

from paper_2412_13755_gb300 import synth

NP = synth.N_PAD


def numpy_clusters(d, n_events, q_peak):
    planes, n_time, _ = d.shape
    pad = np.zeros((planes, n_time + 4, NP + 4), np.int64)
    pad[:, 2:-2, 2:-2] = d
    c = pad[:, 2:-2, 2:-2]

    def nb(dt, dp):
        return pad[:, 2 + dt:2 + dt + n_time, 2 + dp:2 + dp + NP]

    peak = (c >= q_peak) & (c > nb(-1, -1)) & (c > nb(-1, 0)) & (c > nb(-1, 1)) & (c > nb(0, -1)) & \
        (c >= nb(0, 1)) & (c >= nb(1, -1)) & (c >= nb(1, 0)) & (c >= nb(1, 1))
    Q = np.zeros_like(c)
    Sp = np.zeros_like(c)
    St = np.zeros_like(c)
    for dt in range(-2, 3):
        for dp in range(-2, 3):
            v = nb(dt, dp)
            Q += v
            Sp += v * dp
            St += v * dt
    pl, t, p = np.nonzero(peak)              # plane, then raster order
    q, sp, st = Q[pl, t, p], Sp[pl, t, p], St[pl, t, p]
    f32 = np.float32
    cp = p.astype(f32) + sp.astype(f32) / q.astype(f32)
    yy = (cp - f32(79.5)) * f32(0.6)
    ct = t.astype(f32) + st.astype(f32) / q.astype(f32)
    az = (ct + f32(0.5)) * f32(0.5)
    side_c = (pl // synth.N_ROWS) % synth.N_SECTORS >= synth.N_PHI
    zz = np.where(side_c, -az, az)
    off = np.searchsorted(pl // synth.N_ROWS, np.arange(n_events * synth.N_SECTORS + 1))
    return yy, zz, (pl % synth.N_ROWS).astype(np.uint16), np.minimum(q, 65535).astype(np.uint16), off


def random_field(rng, n_time, n_blobs):
    planes = synth.N_SECTORS * synth.N_ROWS
    d = np.zeros((planes, n_time, NP), np.uint16)
    for _ in range(n_blobs):
        pl = rng.integers(planes)
        t0, p0 = rng.integers(-2, n_time + 2), rng.integers(-2, NP + 2)
        a = rng.integers(1, 60)
        for dt in range(-2, 3):
            for dp in range(-2, 3):
                t, p = t0 + dt, p0 + dp
                if 0 <= t < n_time and 0 <= p < NP:
                    d[pl, t, p] = min(1023, int(d[pl, t, p]) + int(a * np.exp(-0.5 * (dt * dt + dp * dp))
                                                                   + rng.integers(0, 3)))
    # flat plateaus and isolated single digits at the edges
    d[5, 0, 0:3] = 20
    d[7, n_time - 1, NP - 1] = 30
    d[9, 3:6, 10:13] = 17
    return d


def test_oracle_matches_numpy_restatement(orc):
    rng = np.random.default_rng(5)
    for n_time in (8, 24):
        d = random_field(rng, n_time, 4000)
        a = orc.find_clusters(d, 1, q_peak=8)
        b = numpy_clusters(d, 1, 8)
        assert len(a[0]) > 500
        for x, y in zip(a, b):
            assert np.array_equal(np.asarray(x), np.asarray(y))


def test_plateau_and_pairs(orc):
    d = np.zeros((synth.N_SECTORS * synth.N_ROWS, 16, NP), np.uint16)
    d[3, 5:8, 20:23] = 40                    # plateau: one peak at (5, 20)
    d[4, 8, 30] = d[4, 8, 34] = 50           # two deposits four pads apart
    d[4, 7:10, 29:32] += 10
    d[4, 7:10, 33:36] += 10
    y, z, row, ch, off = orc.find_clusters(d, 1, q_peak=8)
    assert len(y) == 3
    assert row[0] == 3 and ch[0] == 9 * 40
    assert np.isclose(y[0], (21 - 79.5) * 0.6, atol=1e-5) and np.isclose(z[0], 6.5 * 0.5, atol=1e-5)
    assert list(row[1:]) == [4, 4] and y[1] < y[2]


def test_digitized_clusters_found(orc):
    ev = synth.one_sector(seed=synth.SEED_BASE + 60)
    d = synth.digitize(ev, n_time=synth.N_TIME)
    y, z, row, ch, off = orc.find_clusters(d, 1)
    g_in = np.repeat(np.arange(36), np.diff(ev.evt_sector_off))
    g_out = np.repeat(np.arange(36), np.diff(off))
    found = n_strong = found_iso = n_iso = 0
    isolated_err = []
    for g in np.unique(g_in):
        for r in range(synth.N_ROWS):
            a = np.flatnonzero((g_in == g) & (ev.row == r))
            b = np.flatnonzero((g_out == g) & (row == r))
            if len(a) == 0 or len(b) == 0:
                continue
            dy = ev.y[a][:, None] - y[b][None, :]
            dz = ev.z[a][:, None] - z[b][None, :]
            dist = np.hypot(dy, dz)
            best = dist.min(1)
            strong = ev.charge[a] >= 20
            found += int(np.sum((best < 0.3) & strong))
            n_strong += int(strong.sum())
            # isolated: no other generated cluster within 3 cm in the row
            da = np.hypot(ev.y[a][:, None] - ev.y[a][None, :], ev.z[a][:, None] - ev.z[a][None, :])
            np.fill_diagonal(da, np.inf)
            iso = (da.min(1) > 3.0) & strong
            found_iso += int(np.sum((best < 0.3) & iso))
            n_iso += int(iso.sum())
            j = dist.argmin(1)
            isolated_err += list(np.abs(dy[np.arange(len(a)), j])[iso]) + list(np.abs(dz[np.arange(len(a)), j])[iso])
    eff, eff_iso = found / n_strong, found_iso / n_iso
    print(f"efficiency {eff:.4f} (isolated {eff_iso:.4f}), isolated clusters: max error "
          f"{max(isolated_err):.4f} cm, median {np.median(isolated_err):.4f} cm")
    assert eff >= 0.93 and eff_iso >= 0.99
    assert np.median(isolated_err) < 0.05
