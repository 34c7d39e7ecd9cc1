"""Pins of the oracle's pattern recognition (S1-S4).

* Brute force on tiny events (one sector, rows 0-23, <= 5 tracks, <= 5 noise
  clusters): an exhaustive depth-first enumeration of all maximal admissible
  chains must contain every generated track with >= 10 clusters, and the
  cellular automaton must output exactly that chain's clusters for it.
* Canonical output: shuffling the input order inside each (event, sector)
  group leaves the set of tracks unchanged (ids are input indices).
* Mirror symmetry: reflecting the event about the X axis (sector phi-index
  i -> 17 - i, local y -> -y) leaves the cluster-to-track assignment
  unchanged.
* Efficiency against the generator's truth on a central event (sanity bound).
"""
import numpy as np
import pytest

from paper_2412_13755_gb300 import synth


def tiny_event(seed, n_tracks=5, n_noise=5):
    ev = synth.generate([(n_tracks, 0.0)], seed, wedge=0)
    sec = ev.sector_of_cluster()
    keep = (sec == 0) & (ev.row < 24)
    rng = np.random.default_rng(seed + 99)
    nr = rng.integers(0, 24, n_noise)
    ny = rng.uniform(-1, 1, n_noise) * synth.ROW_X[nr] * synth.TAN_HALF_SECTOR
    nz = rng.uniform(0, 60, n_noise)
    y = np.concatenate([ev.y[keep], ny.astype(np.float32)])
    z = np.concatenate([ev.z[keep], nz.astype(np.float32)])
    row = np.concatenate([ev.row[keep], nr.astype(np.uint16)])
    mc = np.concatenate([ev.mc_track[keep], np.full(n_noise, -1, np.int32)])
    perm = rng.permutation(len(y))
    y, z, row, mc = y[perm], z[perm], row[perm], mc[perm]
    off = np.zeros(37, np.int64)
    off[1:] = len(y)
    return y, z, row, mc, off


@pytest.mark.parametrize("seed", range(12))
def test_bruteforce_tiny_events(orc, seed):
    y, z, row, mc, off = tiny_event(1000 + seed)
    chains = orc.bruteforce_chains(y, z, row, 0)
    chain_set = {tuple(c.tolist()) for c in chains}
    toc, trk_off, hits = orc.find_tracks(y, z, row, off, 1)
    for t in np.unique(mc[mc >= 0]):
        idx = np.nonzero(mc == t)[0]
        if len(idx) < 10:
            continue
        idx = idx[np.argsort(row[idx], kind="stable")]
        truth = tuple(idx.tolist())
        assert truth in chain_set, (seed, t)
        k = toc[idx[0]]
        assert k >= 0
        got = hits[trk_off[k]:trk_off[k + 1]][::-1]
        assert tuple(got.tolist()) == truth, (seed, t)


def _canon_tracks(toc, trk_off, hits, perm=None):
    tracks = set()
    for k in range(len(trk_off) - 1):
        h = hits[trk_off[k]:trk_off[k + 1]]
        if perm is not None:
            h = perm[h]
        tracks.add(tuple(sorted(h.tolist())))
    return tracks


def test_shuffle_within_groups_changes_only_tie_breaks(orc):
    # Canonical ids are input indices and break ties (equal tracklet lengths,
    # equal D^2), so a permutation may flip those decisions but nothing else:
    # almost every cluster keeps the same companions.
    ev = synth.central_event(n_tracks=1500, seed=21)
    base = orc.find_tracks(ev.y, ev.z, ev.row, ev.evt_sector_off, ev.n_events)
    rng = np.random.default_rng(5)
    perm = np.arange(ev.n)
    off = ev.evt_sector_off
    for g in range(len(off) - 1):
        perm[off[g]:off[g + 1]] = off[g] + rng.permutation(off[g + 1] - off[g])
    sh = orc.find_tracks(ev.y[perm], ev.z[perm], ev.row[perm], off, ev.n_events)
    # cluster-level: the track of every cluster keeps (almost) all its members
    toc_b = base[0]
    toc_s = np.full(ev.n, -1, np.int32)
    toc_s[perm] = sh[0]
    assert np.mean((toc_b >= 0) == (toc_s >= 0)) > 0.998
    both = (toc_b >= 0) & (toc_s >= 0)
    pairs = toc_b[both].astype(np.int64) * (1 << 20) + toc_s[both]
    _, cnt = np.unique(pairs, return_counts=True)
    # clusters whose (old track, new track) pair is the dominant one
    major = np.zeros(toc_b.max() + 1, np.int64)
    u, c = np.unique(pairs, return_counts=True)
    np.maximum.at(major, (u >> 20).astype(np.int64), c)
    assert major.sum() >= 0.995 * both.sum()
    # identical input order gives bit-identical output (determinism)
    again = orc.find_tracks(ev.y, ev.z, ev.row, ev.evt_sector_off, ev.n_events)
    for u, v in zip(base, again):
        assert np.array_equal(u, v)


def test_mirror_symmetry(orc):
    ev = synth.central_event(n_tracks=1500, seed=22)
    base = orc.find_tracks(ev.y, ev.z, ev.row, ev.evt_sector_off, ev.n_events)
    sec = ev.sector_of_cluster()
    phi = sec % 18
    side = sec // 18
    msec = (17 - phi) + 18 * side
    # regroup the mirrored clusters by their new sector, keeping input order
    order = np.argsort(msec, kind="stable")
    y = -ev.y[order]
    counts = np.bincount(msec, minlength=36)
    off = np.zeros(37, np.int64)
    off[1:] = np.cumsum(counts)
    mir = orc.find_tracks(y, ev.z[order], ev.row[order], off, 1)
    assert _canon_tracks(*mir, perm=order) == _canon_tracks(*base)


def test_efficiency_central_event(orc):
    ev = synth.central_event(n_tracks=3000, seed=23)
    toc, off, hits = orc.find_tracks(ev.y, ev.z, ev.row, ev.evt_sector_off, ev.n_events)
    toff, thits, tids = ev.truth_tracks()
    found = 0
    for i in range(len(tids)):
        tr = toc[thits[toff[i]:toff[i + 1]]]
        tr = tr[tr >= 0]
        if len(tr) and np.bincount(tr).max() >= 0.5 * (toff[i + 1] - toff[i]):
            found += 1
    assert found / len(tids) > 0.98
    fakes = 0
    for k in range(len(off) - 1):
        m = ev.mc_track[hits[off[k]:off[k + 1]]]
        v, c = np.unique(m, return_counts=True)
        if v[c.argmax()] < 0 or c.max() < 0.5 * len(m):
            fakes += 1
    assert fakes / (len(off) - 1) < 0.01
