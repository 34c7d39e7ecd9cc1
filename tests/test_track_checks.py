"""CPU checks of the track-list checker used by the full-size GPU tests, and
of the two facts those tests rest on:

* the oracle's output satisfies every structural property the checker
  asserts (central, dense, pile-up and batched events), and the checker
  rejects planted corruptions of it;
* events of a batch are independent: the oracle run on a whole batch and on
  each event alone gives the same assignment, so sampled events of a large
  batch can be compared one by one;
* a fit of a subset of tracks equals the same rows of the fit of all.
"""
import numpy as np
import pytest

from paper_2412_13755_gb300 import synth
import track_checks as tc


@pytest.fixture(scope="module")
def found(orc):
    cases = {
        "central": synth.central_event(n_tracks=2000, seed=101),
        "dense": synth.central_event(n_tracks=15000, seed=505),
        "pileup": synth.pileup_frame(n_collisions=10, n_tracks=1000, seed=404),
        "batch": synth.uneven_batch(n_events=8, lo=10, hi=1500, seed=303),
    }
    return {k: (ev, *orc.find_tracks(ev.y, ev.z, ev.row, ev.evt_sector_off, ev.n_events))
            for k, ev in cases.items()}


@pytest.mark.parametrize("case", ["central", "dense", "pileup", "batch"])
def test_oracle_output_has_the_structure(found, case):
    ev, toc, off, hits = found[case]
    assert len(off) > 100
    tc.check_structure(ev, toc, off, hits)


def test_canon_matches_its_definition(found):
    ev, toc, off, hits = found["central"]
    want = np.full(ev.n, -1, np.int64)
    for k in range(len(off) - 1):
        h = hits[off[k]:off[k + 1]]
        want[h] = h.min()
    assert np.array_equal(tc.canon_of_cluster(off, hits, ev.n), want)


def _corruptions(ev, toc, off, hits):
    """Each yields (name, track_of_cluster, hits, offsets): a track list
    that breaks one asserted property."""
    T = len(off) - 1
    h = hits.copy()
    h[off[1] - 1] = h[off[1]]  # a cluster on two tracks
    yield "duplicate", toc, h, off
    t = toc.copy()
    t[hits[off[3]]] = 5  # track_of_cluster names another track
    yield "toc", t, hits, off
    t = toc.copy()
    t[np.flatnonzero(toc < 0)[0]] = 0  # an assigned cluster outside the lists
    yield "stray", t, hits, off
    o = off.copy()
    o[1] = o[0] + tc.N_MIN - 1  # a short track
    yield "short", toc, hits, o
    # the outermost and innermost cluster of a long one-sector track swapped
    grp = np.repeat(np.arange(ev.n_events * tc.N_SECTORS), np.diff(ev.evt_sector_off))
    for k in range(T):
        s = grp[hits[off[k]:off[k + 1]]]
        if np.all(s == s[0]):
            h = hits.copy()
            h[off[k]], h[off[k + 1] - 1] = h[off[k + 1] - 1], h[off[k]]
            yield "order", toc, h, off
            break
    # a free cluster moved into the second place of a track: from a sector
    # that is not phi-adjacent on the same side, then from another event
    def moved_in(k, c):
        h = hits.copy()
        t = toc.copy()
        t[h[off[k] + 1]] = -1
        h[off[k] + 1] = c
        t[c] = k
        return t, h

    evt, sec = grp // tc.N_SECTORS, grp % tc.N_SECTORS
    a = hits[off[0] + 1]
    far = np.flatnonzero((toc < 0) & (evt == evt[a]) & ((sec < 18) == (sec[a] < 18))
                         & ((sec - sec[a]) % 18 >= 2) & ((sec[a] - sec) % 18 >= 2))
    yield ("jump", *moved_in(0, far[0]), off)
    if ev.n_events > 1:
        other = np.flatnonzero((toc < 0) & (evt != evt[a]))
        yield ("event", *moved_in(0, other[0]), off)


EXPECT = {"duplicate": "cluster on two tracks", "toc": "track_of_cluster disagrees",
          "stray": "assigned clusters outside", "short": "track length",
          "order": "rows not outermost first", "jump": "non-adjacent sector",
          "event": "spans two events"}


@pytest.mark.parametrize("case", ["central", "batch"])
def test_checker_rejects_corruptions(found, case):
    ev, toc, off, hits = found[case]
    seen = set()
    for name, t, h, o in _corruptions(ev, toc, off, hits):
        with pytest.raises(AssertionError, match=EXPECT[name]):
            tc.check_structure(ev, t, o, h)
        seen.add(name)
    assert seen == set(EXPECT) - ({"event"} if ev.n_events == 1 else set()), seen


def test_events_of_a_batch_are_independent(orc, found):
    ev, toc, off, hits = found["batch"]
    canon = tc.canon_of_cluster(off, hits, ev.n)
    events = tc.sample_events(ev, ev.n_events, seed=1)
    assert events == list(range(ev.n_events))
    agree, total = tc.per_event_agreement(orc, ev, events, canon)
    assert total == ev.n and agree == total


def test_sample_events_includes_the_extremes(found):
    ev = found["batch"][0]
    off = ev.evt_sector_off
    sizes = off[36::36] - off[0:-1:36]
    pick = tc.sample_events(ev, 4, seed=7)
    assert len(pick) == 4 and int(np.argmin(sizes)) in pick and int(np.argmax(sizes)) in pick
    assert pick == tc.sample_events(ev, 4, seed=7)


def test_fit_of_a_subset_equals_rows_of_the_full_fit(orc, found):
    ev, toc, off, hits = found["central"]
    sec = ev.sector_of_cluster()
    full = orc.fit_tracks(ev.y, ev.z, ev.row, sec, off, hits)
    keep = np.random.default_rng(3).choice(len(off) - 1, 200, replace=False)
    s_off, s_hits = tc.sub_tracks(off, hits, keep)
    sub = orc.fit_tracks(ev.y, ev.z, ev.row, sec, s_off, s_hits)
    for a, b in zip(full, sub):
        assert np.array_equal(a[keep], b)
