"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times:

* the 512-event uneven batch (about 1e8 clusters) as one autotuned context,
  its load, find and fit replayed from the library's CUDA graph:
  the whole track list passes the structural checks; sampled events (the
  smallest, the largest and six drawn with a fixed seed) are found again by
  the oracle one by one (events are independent) and their cluster-to-track
  assignment must agree for >= 99.99% of the clusters; the fit of every
  track of those events must match the oracle's fit of the same hit list
  within |dp_i| <= 1e-5 max(|p_i|, s_i);
* the 100-collision pile-up frame (about 1.8e8 clusters, one event): the
  whole track list passes the structural checks, and the fit of 5000 tracks
  drawn with a fixed seed matches the oracle's fit of their hit lists;
* NEXT-4 on the same frame shape with a vertex z spread: the generator's
  A/C segments associated on the GPU and by the oracle over the whole
  frame, every track's partner and every pair's joint fit compared, and
  each collision's t0 recovered from its pairs.

The oracle cannot find a whole frame in seconds; for it the assignment is
covered by the smaller pile-up parity test and, at full size, by the
structural properties that hold at any size.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from paper_2412_13755_gb300 import synth, tpc  # noqa: E402
import track_checks as tc  # noqa: E402

SCALE = np.array([1.0, 1.0, 0.1, 0.1, 0.1])


def _device_inputs(ev, dev="cuda"):
    y = torch.from_numpy(ev.y).to(dev)
    z = torch.from_numpy(ev.z).to(dev)
    row = torch.from_numpy(ev.row.view(np.int16)).to(dev).view(torch.uint16)
    off = torch.from_numpy(ev.evt_sector_off).to(dev)
    return y, z, row, off


def _fit_outputs(cap, dev="cuda"):
    return (torch.empty(cap, 5, dtype=torch.float32, device=dev),
            torch.empty(cap, 15, dtype=torch.float32, device=dev),
            torch.empty(cap, dtype=torch.float32, device=dev),
            torch.empty(cap, dtype=torch.int32, device=dev))


def _to_host(out, fit):
    T = int(out[3].item())
    off = out[1][:T + 1].cpu().numpy()
    hits = out[2][:int(off[-1])].cpu().numpy()
    toc = out[0].cpu().numpy()
    par, _, _, ndf = (f[:T].cpu().numpy() for f in fit)
    return toc, off, hits, par, ndf


def _fit_parity(orc, ev, off, hits, par, ndf, keep):
    s_off, s_hits = tc.sub_tracks(off, hits, keep)
    opar, _, _, ondf = orc.fit_tracks(ev.y, ev.z, ev.row, ev.sector_of_cluster(), s_off, s_hits)
    gpar, gndf = par[keep].astype(np.float64), ndf[keep]
    assert np.array_equal(gndf <= 0, ondf <= 0), "transport failures differ"
    ok = ondf > 0
    assert np.array_equal(gndf[ok], ondf[ok])
    rel = np.abs(gpar - opar) / np.maximum(np.abs(opar), SCALE)
    print(f"  fit of {len(keep)} tracks: max relative error per parameter {rel[ok].max(0)}")
    assert np.all(rel[ok] <= 1e-5), rel[ok].max(0)


def test_uneven_batch_full_size(orc):
    ev = synth.uneven_batch_parallel()
    n, E = ev.n, ev.n_events
    cap = n // 10 + 16
    tr = tpc.Tracker(n, E)
    try:
        y, z, row, off = _device_inputs(ev)
        tr.load(y, z, row, off, E)
        out = tr.alloc_find_outputs(cap)
        fit = _fit_outputs(cap)
        tr.autotune(out=out)
        # as the benchmark times it: the batch call in the library's graph
        tr.capture(y, z, row, off, E, out, fit)
        tr.replay()
        torch.cuda.synchronize()
        tr.check()
        toc, t_off, hits, par, ndf = _to_host(out, fit)
    finally:
        tr.close()
    print(f"\nbatch: {E} events, {n} clusters, {len(t_off) - 1} tracks")
    tc.check_structure(ev, toc, t_off, hits)
    canon = tc.canon_of_cluster(t_off, hits, n)
    events = tc.sample_events(ev, 8, seed=11)
    agree, total = tc.per_event_agreement(orc, ev, events, canon)
    print(f"  events {events}: {total} clusters, agreement {agree / total:.6f}")
    assert agree >= 0.9999 * total
    evt = tc.event_of_cluster(ev.evt_sector_off, E)
    keep = np.flatnonzero(np.isin(evt[hits[t_off[:-1]]], events))
    assert len(keep) > 0
    _fit_parity(orc, ev, t_off, hits, par, ndf, keep)


def test_pileup_frame_full_size(orc):
    ev = synth.pileup_frame_parallel()
    n = ev.n
    cap = n // 10 + 16
    tr = tpc.Tracker(n, 1)
    try:
        y, z, row, off = _device_inputs(ev)
        tr.load(y, z, row, off, 1)
        out = tr.alloc_find_outputs(cap)
        fit = _fit_outputs(cap)
        tr.find(out=out)
        tr.fit(out[1], out[2], cap, out[3], out=fit)
        torch.cuda.synchronize()
        tr.check()
        toc, t_off, hits, par, ndf = _to_host(out, fit)
    finally:
        tr.close()
    T = len(t_off) - 1
    print(f"\npile-up frame: {n} clusters, {T} tracks")
    tc.check_structure(ev, toc, t_off, hits)
    keep = np.sort(np.random.default_rng(12).choice(T, min(T, 5000), replace=False))
    _fit_parity(orc, ev, t_off, hits, par, ndf, keep)


def test_alignment_descent_full_size(orc):
    """The alignment workload at its stated size: 2e5 tracks with pT > 1
    GeV/c on 36 x 6 drawn misalignments, 50 descent steps
    theta <- theta - P g(theta), g the library's adjoint gradient on the GPU,
    P the pseudo-inverse of the oracle's FP64 Gauss-Newton matrix at
    theta = 0 over its eigenvalues above 1e-9 of the largest.  Checks: chi2
    falls; the end point is a stationary point of the oracle's FP64 chi2 in
    every kept direction (gradient below 0.1 of its statistical sigma); and
    recovery against the generated misalignment, reported per direction in
    units of the target (10 um / 0.01 mrad) for the directions the sample
    determines to better than the target."""
    mis = synth.draw_misalignment(synth.SEED_BASE + 4)
    ev = synth.alignment_sample_parallel(n_tracks=200000, misalign=mis)
    off, hits, _ = ev.truth_tracks(n_min=10)
    sec = ev.sector_of_cluster()
    gn = orc.gauss_newton(ev.y, ev.z, ev.row, sec, off, hits, np.zeros(216))
    w, V = np.linalg.eigh(gn)
    keep = w > 1e-9 * w[-1]
    P = (V[:, keep] / w[keep]) @ V[:, keep].T
    tr = tpc.Tracker(ev.n, 1)
    try:
        y, z, row, eo = _device_inputs(ev)
        tr.load(y, z, row, eo, 1)
        d_off, d_hits = torch.from_numpy(off).cuda(), torch.from_numpy(hits).cuda()
        T = len(off) - 1
        theta = np.zeros(216)
        chi2s = []
        for _ in range(50):
            chi2, g = tr.adjoint(d_off, d_hits, T, torch.from_numpy(theta).cuda())
            chi2s.append(chi2.item())
            theta = theta - P @ g.cpu().numpy()
        tr.check()
    finally:
        tr.close()
    _, go = orc.fit_adjoint(ev.y, ev.z, ev.row, sec, off, hits, theta)
    stat = np.abs(V[:, keep].T @ go) / np.sqrt(2 * w[keep])
    units = np.tile([1e-3, 1e-3, 1e-3, 1e-5, 1e-5, 1e-5], 36)
    Hs = gn * np.outer(units, units)
    ws, Vs = np.linalg.eigh(Hs)
    sig = np.sqrt(2.0 / np.maximum(ws, 1e-300))
    good = (ws > 1e-9 * ws[-1]) & (sig < 1.0)
    err = Vs[:, good].T @ ((theta - mis) / units)
    print(f"\nalignment: {T} tracks, chi2 {chi2s[0]:.6e} -> {chi2s[-1]:.6e}; oracle gradient at the end "
          f"max {stat.max():.3f} sigma over {keep.sum()} directions; {good.sum()} directions determined "
          f"to better than the target, {int(np.sum(np.abs(err) <= 1.0))} of them recovered within it "
          f"(largest error {np.abs(err).max():.1f} target units)")
    assert chi2s[-1] < chi2s[0]
    assert stat.max() < 0.1


def test_sides_membrane_frame_full_size(orc):
    from test_gpu_sides import _compare
    ev = synth.membrane_frame_parallel(n_collisions=100)
    off, hits, ids, sides = ev.truth_segments()
    T = len(off) - 1
    tr = tpc.Tracker(ev.n, 1)
    tr.load(*_device_inputs(ev), 1)
    r = tr.match_sides(torch.from_numpy(off).cuda(), torch.from_numpy(hits).cuda(), T)
    torch.cuda.synchronize()
    tr.check()
    g = {k: v.cpu().numpy() for k, v in r.items()}
    del tr
    o = orc.match_sides(ev.y, ev.z, ev.row, ev.evt_sector_off, 1, off, hits)
    both = _compare(g, o, T)
    u, cnt = np.unique(ids, return_counts=True)
    crossing = set(u[cnt == 2].tolist())
    p = g["partner"][:T]
    pairs = [(i, int(p[i])) for i in range(T) if p[i] > i]
    good = sum(1 for i, j in pairs if ids[i] == ids[j])
    print(f"{T} segments, {len(crossing)} crossing tracks, {len(pairs)} pairs, {good} of one track")
    assert good >= 0.995 * len(pairs) and good >= 0.97 * len(crossing)
    # each collision's t0 from the median of its pairs
    sel = np.array([i for i, j in pairs if ids[i] == ids[j]])
    t0_true = ev.trk_t0[ids[sel]]
    res = []
    for t0c in np.unique(t0_true):
        m = t0_true == t0c
        res.append(np.median(g["t0"][sel][m]) - t0c)
    res = np.abs(np.array(res))
    print(f"per-collision t0: median |residual| {np.median(res) * 1e3:.2f} ns, largest {res.max() * 1e3:.2f} ns")
    assert len(res) == 100 and res.max() < 0.01
