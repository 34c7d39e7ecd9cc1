"""S7 through the C ABI: the one-call batch, its CUDA graph held by the
library, and the autotuned work-queue configurations.

* tpc_track_batch returns, bit for bit, what the separate load, find and fit
  calls return.
* A graph captured by tpc_graph_capture and replayed by tpc_graph_launch
  gives the same result again; after the inputs are rewritten in place (the
  clusters of every group shuffled: same sizes, other content) a replay
  tracks the new content, identically to a fresh batch call on it.
* Every configuration the autotuner can choose (lanes per queued cluster of
  the second neighbour pass, tracklet-lane blocks and tile) gives identical
  tracks; the autotuner returns one of them.
"""
import itertools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2412_13755_gb300 import synth, tpc  # noqa: E402
from gpu_util import to_dev  # noqa: E402


def _host(find_out, fit_out):
    toc, off, hits, ntd = (t.cpu().numpy() for t in find_out)
    T = int(ntd[0])
    res = [toc, off[:T + 1], hits[:off[T]], np.array([T])]
    if fit_out is not None:
        res += [t.cpu().numpy()[:T] for t in fit_out]
    return res


def _same(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert x.shape == y.shape and np.array_equal(x.view(np.uint8), y.view(np.uint8))


def test_track_batch_equals_separate_calls():
    ev = synth.uneven_batch(n_events=6, lo=10, hi=800, seed=303)
    E = ev.n_events
    tr = tpc.Tracker(ev.n, E)
    y, z, row, off = to_dev(ev)
    cap = ev.n // 10 + 16
    tr.load(y, z, row, off, E)
    f1 = tr.find(out=tr.alloc_find_outputs(cap))
    p1 = tr.alloc_fit_outputs(cap)
    tr.fit(f1[1], f1[2], cap, f1[3], out=p1)
    f2, p2 = tr.alloc_find_outputs(cap), tr.alloc_fit_outputs(cap)
    tr.track_batch(y, z, row, off, E, f2, p2)
    torch.cuda.synchronize()
    tr.check()
    a, b = _host(f1, p1), _host(f2, p2)
    assert a[3][0] > 100
    _same(a, b)


def test_graph_replay_tracks_inputs_in_place():
    ev = synth.central_event(n_tracks=2000, seed=101)
    n = ev.n
    cap = n // 10 + 16
    y, z, row, off = to_dev(ev)
    ref = tpc.Tracker(n, 1)
    fr, pr = ref.alloc_find_outputs(cap), ref.alloc_fit_outputs(cap)
    ref.track_batch(y, z, row, off, 1, fr, pr)
    torch.cuda.synchronize()
    ref.check()
    want = _host(fr, pr)

    tr = tpc.Tracker(n, 1)
    gy, gz, grow, goff = y.clone(), z.clone(), row.clone(), off.clone()
    fo, po = tr.alloc_find_outputs(cap), tr.alloc_fit_outputs(cap)
    tr.capture(gy, gz, grow, goff, 1, fo, po)
    for _ in range(2):
        for t in fo:
            t.fill_(-9)
        tr.replay()
        torch.cuda.synchronize()
        tr.check()
        _same(_host(fo, po), want)

    # same sizes, other content: every group's clusters shuffled in place
    rng = np.random.default_rng(9)
    o = ev.evt_sector_off
    perm = np.concatenate([o[g] + rng.permutation(o[g + 1] - o[g]) for g in range(36)])
    gy.copy_(y[torch.from_numpy(perm).cuda()])
    gz.copy_(z[torch.from_numpy(perm).cuda()])
    grow.view(torch.int16).copy_(row.view(torch.int16)[torch.from_numpy(perm).cuda()])
    tr.replay()
    torch.cuda.synchronize()
    tr.check()
    fr2, pr2 = ref.alloc_find_outputs(cap), ref.alloc_fit_outputs(cap)
    ref.track_batch(gy.clone(), gz.clone(), grow.clone(), goff.clone(), 1, fr2, pr2)
    torch.cuda.synchronize()
    shuffled = _host(fr2, pr2)
    _same(_host(fo, po), shuffled)
    assert not np.array_equal(shuffled[0], want[0])


def test_every_tuning_gives_identical_tracks():
    ev = synth.uneven_batch(n_events=8, lo=10, hi=3000, seed=313)
    E = ev.n_events
    tr = tpc.Tracker(ev.n, E)
    d = to_dev(ev)
    tr.load(*d, E)
    cap = ev.n // 10 + 16
    base = _host(tr.find(out=tr.alloc_find_outputs(cap)), None)
    for sub, bps, tile in itertools.product((4, 8, 16), (4, 8, 16), (1, 4)):
        tr.set_tune(tpc.Tune(bps, tile, sub))
        got = _host(tr.find(out=tr.alloc_find_outputs(cap)), None)
        torch.cuda.synchronize()
        tr.check()
        _same(got, base)
    best = tr.autotune(out=tr.alloc_find_outputs(cap))
    assert best.nb_sub_lanes in (4, 8, 16) and best.lane_blocks_per_sm in (4, 8, 16)
    assert best.lane_tile in (1, 4)
    _same(_host(tr.find(out=tr.alloc_find_outputs(cap)), None), base)


def test_stage_times_from_graph_replays():
    """With stage timing on at capture the stage events are event nodes of
    the graph: each replay's stages are positive, the find stages add up to
    the find total, and the replay's own duration bounds them."""
    ev = synth.central_event(n_tracks=2000, seed=31)
    tr = tpc.Tracker(ev.n, 1)
    y, z, row, off = to_dev(ev)
    find_out = tr.alloc_find_outputs(ev.n // 10 + 16)
    fit_out = tr.alloc_fit_outputs(ev.n // 10 + 16)
    tr.load(y, z, row, off, 1)
    tr.stage_timing(True)
    tr.capture(y, z, row, off, 1, find_out, fit_out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        e0.record()
        tr.replay()
        e1.record()
        torch.cuda.synchronize()
        st = tr.stage_times()
        total = e0.elapsed_time(e1)
        parts = [st[k] for k in ("bin", "neighbours", "links", "chains", "tracklets", "select", "merge_cand",
                                 "match", "output")]
        assert all(p > 0 for p in parts) and st["fit"] > 0
        assert abs(sum(parts) - st["find_total"]) <= 1e-3 * st["find_total"] + 1e-3
        assert st["find_total"] + st["fit"] <= total * 1.001
    tr.check()
