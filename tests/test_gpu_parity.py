"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

* Pattern recognition: cluster-to-track assignment must agree for >= 99.99%
  of the clusters, and every disagreeing cluster must trace back (through
  the tracks that hold it on either side) to an oracle decision within a
  relative margin of NEAR_TIE of its threshold or runner-up; the neighbour
  step itself is bit-exact by construction.
* Fit: on the same hit lists, FP32 GPU parameters agree with the FP64 oracle
  within |dp_i| <= 1e-5 max(|p_i|, s_i), s = (1 cm, 1 cm, 0.1, 0.1, 0.1 c/GeV),
  for every track.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2412_13755_gb300 import synth, tpc  # noqa: E402
from gpu_util import canon_of_cluster, gpu_find, to_dev  # noqa: E402

SCALE = np.array([1.0, 1.0, 0.1, 0.1, 0.1])


# A GPU/oracle disagreement must descend from a near-tie: a decision of the
# oracle whose deciding quantity lies within this relative margin of the
# value it was compared with (the neighbour D^2 against the cut or the
# runner-up, an extension's chi2 against the cut or the runner-up, a merge
# chi2 against the cut or a competing pair).  The GPU takes the Kalman-based
# decisions in FP32 (tracklet states within ~2e-5 of the FP64 oracle), so
# their chi2 carry relative errors of ~1e-4; the margin allows ten times that.
NEAR_TIE = 1e-3


def _decision_margin(orc_diag, prm):
    """Per cluster: the smallest relative margin of the oracle decisions it
    took part in (neighbour choice, extension, merge)."""
    d2 = orc_diag["d2"].astype(np.float64)
    nx = orc_diag["d2_next"].astype(np.float64)
    cut = float(prm.chi2_link)
    has = orc_diag["choice_up"] >= 0
    with np.errstate(invalid="ignore", divide="ignore"):
        m_cut = np.abs(d2 - cut) / cut
        m_run = np.where(np.isfinite(nx), np.abs(nx - d2) / np.maximum(nx, 1e-30), np.inf)
    s2 = np.where(has, np.minimum(m_cut, m_run), m_cut)
    s2 = np.where(np.isfinite(s2), s2, np.inf)
    return np.minimum(np.minimum(s2, orc_diag["ext_margin"]), orc_diag["merge_margin"])


def _trace_mismatches(gc, oc, g_toc, g_off, g_hits, o_toc, o_off, o_hits, margin):
    """For every disagreeing cluster, the smallest decision margin over the
    clusters of the tracks that hold it on either side."""
    bad = np.nonzero(gc != oc)[0]
    out = np.empty(len(bad))
    for i, c in enumerate(bad):
        hs = [np.array([c])]
        if g_toc[c] >= 0:
            hs.append(g_hits[g_off[g_toc[c]]:g_off[g_toc[c] + 1]])
        if o_toc[c] >= 0:
            hs.append(o_hits[o_off[o_toc[c]]:o_off[o_toc[c] + 1]])
        out[i] = margin[np.concatenate(hs)].min()
    return bad, out


# Decisions taken on a state that estimates no track are exempt: a
# disagreement is also accepted when a track holding the cluster, on either
# side, is not a track by the oracle's own fit (chi2/ndf above this, as for
# a near-curler seeded on a noise cluster, where FP32 and FP64 Kalman
# states part by more than any margin).
NON_PHYSICAL_CHI2NDF = 50.0


def _non_physical(orc, ev, bad, mg, g_toc, g_off, g_hits, o_toc, o_off, o_hits):
    """For each disagreeing cluster whose traced margin exceeds NEAR_TIE:
    True if the GPU or oracle track holding it has oracle chi2/ndf above
    NON_PHYSICAL_CHI2NDF."""
    sec = ev.sector_of_cluster()
    out = np.zeros(len(bad), bool)
    for i in np.flatnonzero(mg > NEAR_TIE):
        c = bad[i]
        lists = []
        if g_toc[c] >= 0:
            lists.append(g_hits[g_off[g_toc[c]]:g_off[g_toc[c] + 1]])
        if o_toc[c] >= 0:
            lists.append(o_hits[o_off[o_toc[c]]:o_off[o_toc[c] + 1]])
        for h in lists:
            _, _, chi2, ndf = orc.fit_tracks(ev.y, ev.z, ev.row, sec, np.array([0, len(h)], np.int32),
                                             h.astype(np.int32))
            if ndf[0] <= 0 or chi2[0] / ndf[0] > NON_PHYSICAL_CHI2NDF:
                out[i] = True
    return out


def _assign_parity(orc, ev, min_agree=0.9999):
    g_toc, g_off, g_hits, st, _ = gpu_find(ev)
    prm = orc.default_params()
    o_toc, o_off, o_hits, dg = orc.find_tracks(ev.y, ev.z, ev.row, ev.evt_sector_off, ev.n_events,
                                                params=prm, diag=True)
    gc = canon_of_cluster(g_toc, g_off, g_hits, ev.n)
    oc = canon_of_cluster(o_toc, o_off, o_hits, ev.n)
    agree = np.mean(gc == oc)
    bad, mg = _trace_mismatches(gc, oc, g_toc, g_off, g_hits, o_toc, o_off, o_hits,
                                _decision_margin(dg, prm))
    print(f"n={ev.n} tracks gpu={len(g_off)-1} oracle={len(o_off)-1} agreement={agree:.6f} "
          f"segments={st.n_segments} tracklets={st.n_tracklets} merges={st.n_merges} "
          f"mismatches={len(bad)} largest traced margin={mg.max() if len(mg) else 0:.2e}")
    assert agree >= min_agree, agree
    exempt = _non_physical(orc, ev, bad, mg, g_toc, g_off, g_hits, o_toc, o_off, o_hits)
    print(f"  near-ties {int(np.sum(mg <= NEAR_TIE))}, on non-physical tracks {int(exempt.sum())}")
    assert np.all((mg <= NEAR_TIE) | exempt), np.sort(mg[~exempt])[-10:]
    return g_toc, g_off, g_hits


def test_find_one_sector(orc):
    ev = synth.one_sector()
    g_toc, g_off, g_hits = _assign_parity(orc, ev)
    assert len(g_off) > 100


def test_find_central_event_small(orc):
    _assign_parity(orc, synth.central_event(n_tracks=2000, seed=101))


@pytest.mark.slow
def test_find_central_event_full(orc):
    _assign_parity(orc, synth.central_event())


def test_find_pileup_frame_small(orc):
    # 10 collisions at drift-time offsets over the 2 ms frame, one event
    _assign_parity(orc, synth.pileup_frame(n_collisions=10, n_tracks=1000, seed=404))


def test_find_dense_event(orc):
    # 3x the central event's tracks in one event: many first-pass up lists
    # and second-pass lists overflow, so every tier of the neighbour search
    # (lane, 8-lane from the first gap pair, full warp) decides some clusters
    ev = synth.central_event(n_tracks=30000, seed=505)
    g_toc, g_off, g_hits, st, _ = gpu_find(ev)
    print(f"second pass {st.n_nb_second}, dense {st.n_nb_dense}, full warp {st.n_nb_full}")
    assert st.n_nb_second > 0 and st.n_nb_dense > 0 and st.n_nb_full > 0
    _assign_parity(orc, ev)


def test_find_multi_event_batch(orc):
    _assign_parity(orc, synth.uneven_batch(n_events=6, lo=10, hi=800, seed=303))


def _check_fit_parity(gpar, gcov, gchi2, gndf, opar, ocov, ochi2, ondf, ok, bars=(1e-5, 1e-5, 1e-5)):
    """Fit bar per quantity, on the tracks that both sides fitted: the five
    parameters within 1e-5 max(|p|, s); the 15 covariance terms within 1e-5
    of sqrt(C_ii C_jj) (a relative error for the diagonal, on the scale of
    the variances for the correlations); chi2 within 1e-5 max(chi2, 1);
    identical ndf.  bars = (parameters, covariance, chi2) replaces the three
    1e-5 bars."""
    rel = np.abs(gpar - opar) / np.maximum(np.abs(opar), SCALE)
    d = ocov[:, [0, 5, 9, 12, 14]]
    iu = [(i, j) for i in range(5) for j in range(i, 5)]
    cscale = np.stack([np.sqrt(d[:, i] * d[:, j]) for i, j in iu], 1)
    crel = np.abs(gcov - ocov) / np.maximum(cscale, 1e-300)
    chrel = np.abs(gchi2 - ochi2) / np.maximum(ochi2, 1.0)
    print("per-quantity |GPU FP32 - oracle FP64| over", int(ok.sum()), "tracks:")
    for i, name in enumerate(("y", "z", "sin phi", "tan lambda", "q/pT")):
        print(f"  {name:10s} median {np.median(rel[ok, i]):.2e} max {rel[ok, i].max():.2e}")
    print(f"  cov terms max {crel[ok].max(0)}")
    print(f"  chi2 median {np.median(chrel[ok]):.2e} max {chrel[ok].max():.2e}")
    assert np.all(rel[ok] <= bars[0]), rel[ok].max(0)
    assert np.all(crel[ok] <= bars[1]), crel[ok].max(0)
    assert np.all(chrel[ok] <= bars[2]), chrel[ok].max()
    assert np.array_equal(gndf[ok], ondf[ok])


def test_fit_parity_truth_tracks(orc):
    ev = synth.central_event(n_tracks=3000, noise=0.0, seed=202)
    sec = ev.sector_of_cluster()
    off, hits, _ = ev.truth_tracks()
    tr = tpc.Tracker(ev.n, 1)
    y, z, row, eo = to_dev(ev)
    tr.load(y, z, row, eo, 1)
    T = len(off) - 1
    par, cov, chi2, ndf = tr.fit(torch.from_numpy(off).cuda(), torch.from_numpy(hits).cuda(), T)
    torch.cuda.synchronize()
    tr.check()
    opar, ocov, ochi2, ondf = orc.fit_tracks(ev.y, ev.z, ev.row, sec, off, hits)
    gpar = par.cpu().numpy().astype(np.float64)
    ok = (ondf > 0) & (ndf.cpu().numpy() > 0)
    assert ok.mean() > 0.999
    # errors are also a tiny fraction of each parameter's own sigma
    in_sigma = np.abs(gpar - opar) / np.sqrt(ocov[:, [0, 5, 9, 12, 14]])
    assert in_sigma[ok].max() <= 1e-2, in_sigma[ok].max(0)
    _check_fit_parity(gpar, cov.cpu().numpy().astype(np.float64), chi2.cpu().numpy().astype(np.float64),
                      ndf.cpu().numpy(), opar, ocov, ochi2, ondf, ok)


def test_fit_pulls_unit_width_on_gpu():
    """The GPU fit's pulls against the generator's truth, with the oracle's
    bar: over the tracks of chi2 probability > 1e-3, |mean| < 0.03 and
    standard deviation in [0.97, 1.03] for each of the five parameters."""
    from scipy.stats import chi2 as chi2_dist
    ev = synth.central_event(n_tracks=10000, noise=0.0, truth=True, seed=11)
    off, hits, tids = ev.truth_tracks(n_min=20)
    tr = tpc.Tracker(ev.n, 1)
    tr.load(*to_dev(ev), 1)
    T = len(off) - 1
    par, cov, chi2, ndf = tr.fit(torch.from_numpy(off).cuda(), torch.from_numpy(hits).cuda(), T)
    torch.cuda.synchronize()
    tr.check()
    par = par.cpu().numpy().astype(np.float64)
    cov = cov.cpu().numpy().astype(np.float64)
    chi2, ndf = chi2.cpu().numpy().astype(np.float64), ndf.cpu().numpy()
    ok = ndf > 0
    inner = hits[off[1:] - 1]
    truth = np.stack([ev.y_true[inner], ev.z_true[inner], ev.snp_true[inner], ev.trk_tgl[tids],
                      ev.trk_q[tids] / ev.trk_pt[tids]], 1)
    pull = ((par - truth) / np.sqrt(cov[:, [0, 5, 9, 12, 14]]))[ok]
    good = chi2_dist.sf(chi2[ok], ndf[ok]) > 1e-3
    assert good.mean() > 0.995, good.mean()
    mu, sd = pull[good].mean(0), pull[good].std(0)
    print("GPU pull mean", mu, "std", sd)
    assert np.all(np.abs(mu) < 0.03), mu
    assert np.all((sd > 0.97) & (sd < 1.03)), sd


def test_fit_parity_found_tracks(orc):
    """The fit of every track the pipeline finds in a noisy event (fakes and
    low-pT tracks included) against the FP64 oracle on the same hit lists."""
    ev = synth.central_event(n_tracks=2000, seed=101)
    toc, off, hits, st, tr = gpu_find(ev)
    T = len(off) - 1
    par, cov, chi2, ndf = tr.fit(torch.from_numpy(off.astype(np.int32)).cuda(),
                                 torch.from_numpy(hits.astype(np.int32)).cuda(), T)
    torch.cuda.synchronize()
    tr.check()
    opar, ocov, ochi2, ondf = orc.fit_tracks(ev.y, ev.z, ev.row, ev.sector_of_cluster(), off, hits)
    gndf = ndf.cpu().numpy()
    # transport failures agree
    assert np.array_equal(gndf <= 0, ondf <= 0)
    ok = ondf > 0
    _check_fit_parity(par.cpu().numpy().astype(np.float64), cov.cpu().numpy().astype(np.float64),
                      chi2.cpu().numpy().astype(np.float64), gndf, opar, ocov, ochi2, ondf, ok)


def test_fit_fp32_parity_found_tracks(orc):
    """tpc_fit_tracks_fp32 (FP32 covariance, FP64 redo of cancelling
    updates) on every track the pipeline finds in a noisy event, against the
    FP64 oracle on the same hit lists, at its own bars: parameters within
    1e-4 max(|p|, s) and within 0.05 of their own sigma, covariance terms
    and chi2 within 2e-3 (measured on the host: 5.8e-5, 0.034 sigma, 8e-4,
    7.8e-4); the float-float fit meets 1e-5 on the same tracks.  The FP64
    redo is exercised."""
    ev = synth.central_event(n_tracks=2000, seed=101)
    toc, off, hits, st, tr = gpu_find(ev)
    T = len(off) - 1
    d_off = torch.from_numpy(off.astype(np.int32)).cuda()
    d_hits = torch.from_numpy(hits.astype(np.int32)).cuda()
    n0 = tr.stats().n_fp64_updates
    par, cov, chi2, ndf = tr.fit(d_off, d_hits, T, precision="fp32")
    torch.cuda.synchronize()
    tr.check()
    n_redo = tr.stats().n_fp64_updates - n0
    opar, ocov, ochi2, ondf = orc.fit_tracks(ev.y, ev.z, ev.row, ev.sector_of_cluster(), off, hits)
    gndf = ndf.cpu().numpy()
    assert np.array_equal(gndf <= 0, ondf <= 0)
    ok = ondf > 0
    gpar = par.cpu().numpy().astype(np.float64)
    print("FP32 covariance with FP64 redos:", n_redo, "redos")
    _check_fit_parity(gpar, cov.cpu().numpy().astype(np.float64), chi2.cpu().numpy().astype(np.float64),
                      gndf, opar, ocov, ochi2, ondf, ok, bars=(1e-4, 2e-3, 2e-3))
    in_sigma = np.abs(gpar[ok] - opar[ok]) / np.sqrt(ocov[ok][:, [0, 5, 9, 12, 14]])
    assert in_sigma.max() <= 0.05, in_sigma.max(0)
    assert n_redo > 0


def test_empty_input():
    tr = tpc.Tracker(16, 1)
    y = torch.zeros(0, device="cuda")
    z = torch.zeros(0, device="cuda")
    row = torch.zeros(0, dtype=torch.int16, device="cuda").view(torch.uint16)
    off = torch.zeros(37, dtype=torch.int64, device="cuda")
    tr.load(y, z, row, off, 1)
    toc, trk_off, hits, ntd = tr.find(track_cap=4)
    torch.cuda.synchronize()
    tr.check()
    assert int(ntd.item()) == 0


def test_undersized_outputs_refused():
    """Buffers smaller than what a call writes are refused on the host,
    before any kernel could write past them: find and autotune outputs
    smaller than the loaded cluster count, fit outputs and adjoint buffers
    smaller than the track count."""
    ev = synth.one_sector()
    tr = tpc.Tracker(ev.n, 1)
    tr.load(*to_dev(ev), 1)
    i32 = dict(dtype=torch.int32, device="cuda")
    small = (torch.empty(ev.n - 1, **i32), torch.empty(9, **i32), torch.empty(ev.n, **i32),
             torch.empty(1, **i32))
    with pytest.raises(ValueError, match="track_of_cluster"):
        tr.find(out=small)
    with pytest.raises(ValueError, match="track_of_cluster"):
        tr.autotune(out=small)
    short_hits = (small[2], small[1], small[0], small[3])
    with pytest.raises(ValueError, match="trk_hits"):
        tr.find(out=short_hits)
    out = tr.find(out=tr.alloc_find_outputs())
    torch.cuda.synchronize()
    tr.check()
    T = int(out[3].item())
    assert T > 0
    f32 = dict(dtype=torch.float32, device="cuda")
    fit = (torch.empty(T, 5, **f32), torch.empty(T - 1, 15, **f32), torch.empty(T, **f32),
           torch.empty(T, **i32))
    with pytest.raises(ValueError, match="cov"):
        tr.fit(out[1], out[2], T, out=fit)
    with pytest.raises(ValueError, match="trk_off"):
        tr.fit(out[1][:T], out[2], T)
    with pytest.raises(ValueError, match="align"):
        tr.adjoint(out[1], out[2], T, torch.zeros(215, dtype=torch.float64, device="cuda"))
    tr.check()


def test_pileup_drift_offsets_recovered():
    """Pile-up frame: the collision time of every found track follows from
    its fitted z at the vertex, z_vertex = -v_d t0 (A side) or +v_d t0
    (C side); it matches the generated drift-time offset of its collision."""
    ev = synth.pileup_frame(n_collisions=5, n_tracks=2000, noise=0.1, seed=synth.SEED_BASE + 17)
    toc, off, hits, st, tr = gpu_find(ev)
    T = len(off) - 1
    par, cov, chi2, ndf = tr.fit(torch.from_numpy(off.astype(np.int32)).cuda(),
                                 torch.from_numpy(hits.astype(np.int32)).cuda(), T)
    torch.cuda.synchronize()
    tr.check()
    p = par.cpu().numpy().astype(np.float64)
    ok = ndf.cpu().numpy() > 0
    inner = hits[off[1:] - 1]                       # innermost cluster of each track
    sec = ev.sector_of_cluster()[inner]
    x = synth.ROW_X[ev.row[inner]]
    y, z, tgl, w = p[:, 0], p[:, 1], p[:, 3], p[:, 4]
    # transverse arc from the vertex (origin) to the innermost cluster
    chord = np.hypot(x, y)
    k = np.abs(synth.KAPPA * synth.BZ * w)
    arc = np.where(k * chord > 1e-9, 2.0 / np.maximum(k, 1e-30) * np.arcsin(np.minimum(k * chord / 2, 1.0)), chord)
    zv = z - tgl * arc
    t0_reco = np.where(sec < 18, -zv, zv) / synth.V_DRIFT
    # truth: the majority generated track of each found track
    mc = ev.mc_track[hits]
    maj = np.array([np.bincount(mc[off[t]:off[t + 1]][mc[off[t]:off[t + 1]] >= 0]).argmax()
                    if np.any(mc[off[t]:off[t + 1]] >= 0) else -1 for t in range(T)])
    good = ok & (maj >= 0)
    res = t0_reco[good] - ev.trk_t0[maj[good]]
    print(f"{good.sum()} tracks: t0 residual median {np.median(np.abs(res)):.3f} us, "
          f"within 0.5 us {np.mean(np.abs(res) < 0.5):.4f}")
    assert np.median(np.abs(res)) < 0.1
    assert np.mean(np.abs(res) < 0.5) > 0.95
    # per collision, the mean over its tracks recovers the offset
    coll_t0 = np.unique(ev.trk_t0)
    for t0 in coll_t0:
        sel = np.abs(ev.trk_t0[maj[good]] - t0) < 1e-9
        assert abs(np.median(t0_reco[good][sel]) - t0) < 0.05
