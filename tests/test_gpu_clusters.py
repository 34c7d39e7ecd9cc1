"""NEXT-2 on the GPU through the C ABI: tpc_find_clusters against the
oracle's clusterizer, bit for bit (every decision is on integer counts and
every position a fixed sequence of FP32 operations): positions, rows,
charges, group offsets and count, on a digitized central event (0.9 GB of
digits, 1.6e6 clusters), on random fields with a partial last tile
(n_time = 24) and peaks on every edge, and on an empty field; a capacity
below the count is reported and truncates; and the clusters feed the
tracker, which finds what the oracle finds on the same clusters."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2412_13755_gb300 import synth, tpc  # noqa: E402
from gpu_util import canon_of_cluster, gpu_find  # noqa: E402
from test_oracle_clusters import random_field  # noqa: E402


def _dev_digits(d):
    return torch.from_numpy(np.ascontiguousarray(d).view(np.int16)).cuda().view(torch.uint16)


def _gpu(d, n_events, cap=None):
    cap = cap or max(int(np.count_nonzero(d)), 1)
    cl = tpc.Clusterizer(n_events, d.shape[1], cap)
    out = cl.run(_dev_digits(d))
    torch.cuda.synchronize()
    y, z, row, ch, off, n, st = out
    k = int(n.item())
    return (y[:k].cpu().numpy(), z[:k].cpu().numpy(), row.view(torch.int16)[:k].cpu().numpy().view(np.uint16),
            ch.view(torch.int16)[:k].cpu().numpy().view(np.uint16), off.cpu().numpy(), st.cpu().numpy())


def _same(g, o):
    for a, b in zip(g[:5], o):
        assert np.array_equal(np.asarray(a).view(np.uint8), np.asarray(b).view(np.uint8))


def test_central_event_bit_exact(orc):
    ev = synth.central_event()
    d = synth.digitize(ev)
    g = _gpu(d, 1)
    o = orc.find_clusters(d, 1)
    print(f"{len(o[0])} clusters from {np.count_nonzero(d)} digits ({ev.n} generated)")
    assert g[5][0] == tpc.TPC_OK
    _same(g, o)


def test_random_fields_and_edges(orc):
    rng = np.random.default_rng(6)
    for n_time in (24, 64):
        d = random_field(rng, n_time, 6000)
        g = _gpu(d, 1)
        assert g[5][0] == tpc.TPC_OK
        _same(g, orc.find_clusters(d, 1))
    d = np.zeros((36 * 152, 32, 160), np.uint16)
    g = _gpu(d, 1)
    assert g[5][0] == tpc.TPC_OK and len(g[0]) == 0 and np.all(g[4] == 0)


def test_capacity_truncates(orc):
    rng = np.random.default_rng(7)
    d = random_field(rng, 32, 3000)
    o = orc.find_clusters(d, 1)
    cap = len(o[0]) // 2
    g = _gpu(d, 1, cap=cap)
    assert g[5][0] == tpc.TPC_ERR_CAPACITY
    assert len(g[0]) == cap
    for a, b in zip(g[:4], o[:4]):
        assert np.array_equal(a, b[:cap])


def test_clusters_feed_the_tracker(orc):
    ev = synth.central_event(n_tracks=2000, seed=909)
    d = synth.digitize(ev)
    y, z, row, ch, off, st = _gpu(d, 1)
    import types
    cev = types.SimpleNamespace(y=y, z=z, row=row, evt_sector_off=off, n_events=1, n=len(y))
    g_toc, g_off, g_hits, _, _ = gpu_find(cev)
    o_toc, o_off, o_hits = orc.find_tracks(y, z, row, off, 1)
    agree = np.mean(canon_of_cluster(g_toc, g_off, g_hits, cev.n) == canon_of_cluster(o_toc, o_off, o_hits, cev.n))
    print(f"{len(y)} clusters, {len(g_off) - 1} tracks, agreement {agree:.6f}")
    assert len(g_off) - 1 > 1500 and agree >= 0.9999
