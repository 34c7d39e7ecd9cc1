"""NEXT-4 on the GPU through the C ABI: the association of the A- and
C-side segments of membrane-crossing tracks with t0 as a sixth parameter,
against the FP64 oracle.

* On the generator's own segments of a membrane-crossing frame (10
  collisions): the partner of every track is the oracle's (a difference is
  allowed only where the oracle's decision margin is <= 1e-6 relative, the
  near-tie rule), and t0, the six parameters and chi2 of every pair agree to
  1e-9 of their scale, the covariance to 1e-7 (both FP64, the bars of the
  host check in tests/test_sides_host.py).
* End to end: the GPU's find on the same frame, then its association; the
  oracle's find, then the oracle's association; the pairs (as cluster sets)
  are the same and the recovered t0 agree with the collisions' truth.
* Two events in one batch are never paired across; a frame without vertex
  spread gives no pair; an empty track list writes nothing; too small a
  candidate capacity is reported in the status word.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2412_13755_gb300 import synth, tpc  # noqa: E402
from gpu_util import gpu_find, to_dev  # noqa: E402

SCALE = np.array([1.0, 1.0, 0.1, 0.1, 0.1, 0.01])
IU6 = [(i, j) for i in range(6) for j in range(i, 6)]
DIAG6 = [IU6.index((i, i)) for i in range(6)]


def _np(r):
    return {k: v.cpu().numpy() for k, v in r.items()}


def _gpu_sides(ev, off, hits, tr=None):
    if tr is None:
        tr = tpc.Tracker(ev.n, ev.n_events)
        tr.load(*to_dev(ev), ev.n_events)
    d_off, d_hits = torch.from_numpy(off).cuda(), torch.from_numpy(hits).cuda()
    r = tr.match_sides(d_off, d_hits, len(off) - 1)
    torch.cuda.synchronize()
    tr.check()
    return _np(r), tr


def _compare(g, o, T):
    gp, op = g["partner"][:T], o["partner"]
    diff = np.nonzero(gp != op)[0]
    # a different partner only at a near-tie of the oracle's decisions
    assert np.all(o["margin"][diff] <= 1e-6), (diff[:10], o["margin"][diff][:10])
    assert int(g["n_pairs"][0]) == int(np.sum(gp >= 0)) // 2
    both = np.nonzero((gp >= 0) & (gp == op))[0]
    o6, oc = o["params6"][both], o["cov6"][both]
    s = np.sqrt(oc[:, DIAG6])
    err_p = np.abs(g["params6"][both] - o6) / np.maximum(np.abs(o6), np.maximum(s, SCALE))
    sd = np.sqrt(np.abs(oc[:, [DIAG6[i] for i, _ in IU6]] * oc[:, [DIAG6[j] for _, j in IU6]]))
    err_c = np.abs(g["cov6"][both] - oc) / sd
    err_x = np.abs(g["chi2"][both] - o["chi2"][both]) / o["chi2"][both]
    err_d = np.abs(g["dchi2"][both] - o["dchi2"][both]) / np.maximum(np.abs(o["dchi2"][both]), 1.0)
    assert np.array_equal(g["ndf"][:T], o["ndf"])
    assert np.array_equal(g["t0"][both], g["params6"][both, 5])
    print(f"pairs gpu={int(g['n_pairs'][0])} oracle={int(np.sum(op >= 0)) // 2} partner differences={len(diff)}; "
          f"params {err_p.max():.2e} cov {err_c.max():.2e} chi2 {err_x.max():.2e} dchi2 {err_d.max():.2e}")
    assert err_p.max() < 1e-9 and err_x.max() < 1e-9 and err_d.max() < 1e-8 and err_c.max() < 1e-7
    return both


def test_sides_parity_on_generated_segments(orc):
    ev = synth.membrane_frame(n_collisions=10, n_tracks=1000, truth=True)
    off, hits, ids, sides = ev.truth_segments()
    g, _ = _gpu_sides(ev, off, hits)
    o = orc.match_sides(ev.y, ev.z, ev.row, ev.evt_sector_off, ev.n_events, off, hits)
    both = _compare(g, o, len(off) - 1)
    assert len(both) > 2 * 150
    # t0 pulls of the GPU's pairs against the collisions' truth
    pull = (g["t0"][both] - ev.trk_t0[ids[both]]) / np.sqrt(g["cov6"][both, 20])
    assert abs(pull.mean()) < 0.25 and abs(pull.std() - 1) < 0.15


def _track_sets(off, hits):
    return [frozenset(hits[off[t]:off[t + 1]].tolist()) for t in range(len(off) - 1)]


def _pairs(partner, sets):
    return {frozenset((sets[t], sets[p])): t for t, p in enumerate(partner) if p > t}


def test_sides_end_to_end(orc):
    ev = synth.membrane_frame(n_collisions=10, n_tracks=1000, truth=True, seed=synth.SEED_BASE + 9)
    g_toc, g_off, g_hits, st, tr = gpu_find(ev)
    g, _ = _gpu_sides(ev, g_off, g_hits, tr)
    o_toc, o_off, o_hits = orc.find_tracks(ev.y, ev.z, ev.row, ev.evt_sector_off, ev.n_events)
    o = orc.match_sides(ev.y, ev.z, ev.row, ev.evt_sector_off, ev.n_events, o_off, o_hits)
    gs, os_ = _track_sets(g_off, g_hits), _track_sets(o_off, o_hits)
    common = set(gs) & set(os_)
    gk = _pairs(g["partner"][:len(g_off) - 1], gs)
    ok = _pairs(o["partner"], os_)
    # pairs of tracks that both finds produced identically must be identical;
    # a pair touching a track only one side found (a find near-tie) is left out
    gk_c = {k for k in gk if k <= common}
    ok_c = {k for k in ok if k <= common}
    print(f"tracks gpu={len(gs)} oracle={len(os_)} identical={len(common)}; pairs gpu={len(gk)} "
          f"oracle={len(ok)} on identical tracks {len(gk_c)} / {len(ok_c)}")
    assert len(ok) > 120 and len(ok_c) >= 0.98 * len(ok)
    assert gk_c == ok_c
    # the recovered t0 against the truth of the majority MC track
    t = np.array([gk[k] for k in gk])
    mc = np.array([np.bincount(np.maximum(ev.mc_track[g_hits[g_off[i]:g_off[i + 1]]], 0)).argmax() for i in t])
    pull = (g["t0"][t] - ev.trk_t0[mc]) / np.sqrt(g["cov6"][t, 20])
    assert np.median(np.abs(pull)) < 1.0 and np.mean(np.abs(pull) < 5) > 0.97


def test_sides_not_across_events(orc):
    ev = synth.generate([(1500, 0.1), (1500, 0.1)], seed=17, vz_sigma=synth.VZ_SIGMA, truth=True)
    off, hits, ids, sides = ev.truth_segments()
    g, _ = _gpu_sides(ev, off, hits)
    o = orc.match_sides(ev.y, ev.z, ev.row, ev.evt_sector_off, ev.n_events, off, hits)
    _compare(g, o, len(off) - 1)
    p = g["partner"][:len(off) - 1]
    paired = np.nonzero(p >= 0)[0]
    assert len(paired) > 20
    assert np.all(ev.trk_event[ids[paired]] == ev.trk_event[ids[p[paired]]])


def test_sides_no_crossing_and_empty():
    ev = synth.generate([(2000, 0.1)], seed=5)
    _, g_off, g_hits, _, tr = gpu_find(ev)
    g, _ = _gpu_sides(ev, g_off, g_hits, tr)
    assert int(g["n_pairs"][0]) == 0 and np.all(g["partner"][:len(g_off) - 1] == -1)
    z = torch.zeros(1, dtype=torch.int32, device="cuda")
    r = tr.match_sides(z, z, 0)
    torch.cuda.synchronize()
    tr.check()
    assert int(r["n_pairs"].item()) == 0


def test_sides_candidate_capacity_reported():
    ev = synth.membrane_frame(n_collisions=3, n_tracks=1000, seed=synth.SEED_BASE + 10)
    off, hits, ids, sides = ev.truth_segments()
    tr = tpc.Tracker(ev.n, ev.n_events)
    tr.load(*to_dev(ev), ev.n_events)
    r = tr.match_sides(torch.from_numpy(off).cuda(), torch.from_numpy(hits).cuda(), len(off) - 1, cand_cap=2)
    torch.cuda.synchronize()
    with pytest.raises(tpc.TPCError, match="CAPACITY|capacity"):
        tr.check()
    tr.reset_status()
    assert int(r["n_pairs"].item()) <= 2
