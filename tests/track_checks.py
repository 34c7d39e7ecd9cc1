"""Checks of a track list that need neither torch nor a GPU, shared by the
CPU tests (applied to the oracle's own output) and the full-size GPU tests.

A track list is the find step's output: track_of_cluster[n] (track index or
-1), trk_off[T+1] and trk_hits (input-order cluster indices, outermost
first), as the C ABI defines it."""
import numpy as np

N_SECTORS = 36
N_PHI = 18
N_MIN = 10  # minimum clusters of a final track (the merge's acceptance)


def canon_of_cluster(trk_off, hits, n):
    """Per cluster: the smallest input index of its track (-1 = none).  This
    names a track independently of the order in which tracks are listed."""
    out = np.full(n, -1, np.int64)
    T = len(trk_off) - 1
    if T == 0:
        return out
    lens = np.diff(trk_off)
    assert np.all(lens > 0)
    mins = np.minimum.reduceat(hits[:trk_off[-1]], trk_off[:-1])
    out[hits[:trk_off[-1]]] = np.repeat(mins, lens)
    return out


def event_of_cluster(evt_sector_off, n_events):
    return np.repeat(np.arange(n_events * N_SECTORS) // N_SECTORS, np.diff(evt_sector_off))


def check_structure(ev, toc, trk_off, hits, n_min=N_MIN):
    """Asserts what holds for any output of the method at any size:
    - every track has at least n_min clusters;
    - every cluster is on at most one track, and track_of_cluster names it;
    - a track's clusters lie in one event and on one side (A or C);
    - between consecutive clusters of a track in one sector the row does not
      increase (outermost first), and a change of sector goes to a
      phi-adjacent sector.
    A track may come back into a sector it left, and two of its clusters
    may share a row (merged fakes in dense events); neither is asserted."""
    n = ev.n
    T = len(trk_off) - 1
    assert trk_off[0] == 0 and np.all(np.diff(trk_off) >= n_min), "track length"
    h = hits[:trk_off[-1]].astype(np.int64)
    assert np.all((h >= 0) & (h < n)), "hit index range"
    assert len(h) == 0 or np.bincount(h, minlength=n).max() <= 1, "cluster on two tracks"
    tid = np.repeat(np.arange(T), np.diff(trk_off))
    assert np.array_equal(toc[h], tid), "track_of_cluster disagrees with the hit lists"
    assert int((toc[:n] >= 0).sum()) == len(h), "assigned clusters outside the hit lists"
    assert np.all((toc[:n] >= -1) & (toc[:n] < T)), "track_of_cluster range"
    if T == 0:
        return
    grp = np.repeat(np.arange(ev.n_events * N_SECTORS), np.diff(ev.evt_sector_off))[h]
    evt, sec = grp // N_SECTORS, grp % N_SECTORS
    row = ev.row[h].astype(np.int64)
    same = tid[1:] == tid[:-1]
    assert np.all(evt[1:][same] == evt[:-1][same]), "track spans two events"
    assert np.all((sec[1:] < N_PHI)[same] == (sec[:-1] < N_PHI)[same]), "track spans both sides"
    in_sec = same & (sec[1:] == sec[:-1])
    assert np.all(row[1:][in_sec] <= row[:-1][in_sec]), "rows not outermost first"
    chg = same & (sec[1:] != sec[:-1])
    i0, i1 = sec[:-1][chg] % N_PHI, sec[1:][chg] % N_PHI
    assert np.all(((i1 - i0) % N_PHI == 1) | ((i0 - i1) % N_PHI == 1)), "jump to a non-adjacent sector"


def event_slice(ev, e):
    """Clusters of event e of a batch as a one-event input: (y, z, row,
    evt_sector_off, first cluster index, cluster count)."""
    off = ev.evt_sector_off
    b, m = int(off[N_SECTORS * e]), int(off[N_SECTORS * (e + 1)] - off[N_SECTORS * e])
    loc = (off[N_SECTORS * e:N_SECTORS * (e + 1) + 1] - b).astype(np.int64)
    return ev.y[b:b + m], ev.z[b:b + m], ev.row[b:b + m], loc, b, m


def sample_events(ev, k, seed):
    """The smallest and the largest event plus k - 2 others drawn with a
    seeded generator, in increasing order."""
    off = ev.evt_sector_off
    sizes = off[N_SECTORS::N_SECTORS] - off[0:-1:N_SECTORS]
    pick = {int(np.argmin(sizes)), int(np.argmax(sizes))}
    rng = np.random.default_rng(seed)
    rest = [e for e in rng.permutation(ev.n_events).tolist() if e not in pick]
    pick.update(rest[:max(0, k - len(pick))])
    return sorted(pick)


def per_event_agreement(orc, ev, events, batch_canon):
    """Finds each listed event alone with the oracle and compares the
    cluster-to-track assignment with the batch result (canonical ids in
    batch input indices).  Returns (agreeing clusters, clusters)."""
    agree = total = 0
    for e in events:
        y, z, row, loc, b, m = event_slice(ev, e)
        _, o_off, o_hits = orc.find_tracks(y, z, row, loc, 1)
        oc = canon_of_cluster(o_off, o_hits, m)
        gc = batch_canon[b:b + m]
        gc = np.where(gc >= 0, gc - b, -1)
        agree += int((gc == oc).sum())
        total += m
    return agree, total


def sub_tracks(trk_off, hits, keep):
    """The CSR of the listed tracks (hit indices unchanged)."""
    keep = np.asarray(keep, np.int64)
    lens = (trk_off[keep + 1] - trk_off[keep]).astype(np.int64)
    off = np.zeros(len(keep) + 1, np.int32)
    off[1:] = np.cumsum(lens)
    idx = np.repeat(trk_off[keep].astype(np.int64) - off[:-1], lens) + np.arange(off[-1])
    return off, hits[idx].astype(np.int32)
