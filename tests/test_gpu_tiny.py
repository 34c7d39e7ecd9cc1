"""The brute-force events on the GPU: one sector, rows 0-23, at most five
tracks and five noise clusters, the other 35 sectors empty.  For every
generated track with >= 10 clusters, the GPU must return exactly that
track's chain (the admissible chain the exhaustive enumeration contains,
outermost first), and its whole cluster-to-track assignment must equal the
oracle's.  These are the smallest non-empty batches the library takes.
"""
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import canon_of_cluster, gpu_find  # noqa: E402
from test_oracle_ca import tiny_event  # noqa: E402


@pytest.mark.parametrize("seed", range(12))
def test_tiny_events_exact(orc, seed):
    y, z, row, mc, off = tiny_event(1000 + seed)
    ev = types.SimpleNamespace(y=y, z=z, row=row, evt_sector_off=off, n_events=1, n=len(y))
    g_toc, g_off, g_hits, st, _ = gpu_find(ev)
    o_toc, o_off, o_hits = orc.find_tracks(y, z, row, off, 1)
    assert np.array_equal(canon_of_cluster(g_toc, g_off, g_hits, ev.n),
                          canon_of_cluster(o_toc, o_off, o_hits, ev.n))
    for t in np.unique(mc[mc >= 0]):
        idx = np.nonzero(mc == t)[0]
        if len(idx) < 10:
            continue
        idx = idx[np.argsort(row[idx], kind="stable")]
        k = g_toc[idx[0]]
        assert k >= 0, (seed, t)
        got = g_hits[g_off[k]:g_off[k + 1]][::-1]
        assert tuple(got.tolist()) == tuple(idx.tolist()), (seed, t)
