"""tpc_find_tracks_noalloc against tpc_find_tracks.

The no-allocation entry point is for callers that may not reserve device
memory (their memory belongs to another allocator, or a cudaMalloc's implicit
synchronisation is not acceptable); its scratch is a fixed array inside the
library image.  Called three times in a row on different events through the C ABI,
it must return exactly what the regular entry point returns (integer outputs:
assignment, offsets, hit lists and the track count are compared bit for bit),
with a clean device status.  A third, smaller call follows the larger one,
so that contents a larger call leaves in the shared array cannot leak into a
later result unnoticed.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2412_13755_gb300 import synth, tpc  # noqa: E402
from gpu_util import gpu_find, to_dev  # noqa: E402


def _noalloc(lib, ev, track_cap):
    y, z, row, off = to_dev(ev)
    n = ev.n
    toc = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    trk_off = torch.full((track_cap + 1,), -7, dtype=torch.int32, device="cuda")
    hits = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    ntd = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    st = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    p = C.c_void_p
    rc = lib.tpc_find_tracks_noalloc(
        None, p(y.data_ptr()), p(z.data_ptr()), p(row.data_ptr()), C.c_int64(n),
        p(off.data_ptr()), C.c_int32(ev.n_events), p(toc.data_ptr()), p(trk_off.data_ptr()),
        p(hits.data_ptr()), p(ntd.data_ptr()), p(st.data_ptr()), C.c_int32(track_cap),
        p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert rc == tpc.TPC_OK
    assert int(st.item()) == tpc.TPC_OK
    T = int(ntd.item())
    o = trk_off[:T + 1].cpu().numpy()
    return toc.cpu().numpy()[:n], o, hits[:o[-1]].cpu().numpy()


def test_noalloc_matches_find_tracks_twice():
    lib = tpc.load_library()
    lib.tpc_find_tracks_noalloc.restype = C.c_int
    # a larger batch followed by a smaller one: what the larger call left in
    # the shared array must not leak into the smaller call's result
    events = [synth.one_sector(seed=synth.SEED_BASE + 50),
              synth.uneven_batch(n_events=3, lo=20, hi=120, seed=synth.SEED_BASE + 51),
              synth.one_sector(n_tracks=20, seed=synth.SEED_BASE + 52)]
    for ev in events:
        assert ev.n <= 65536 and ev.n_events <= 4
        g_toc, g_off, g_hits, _, _ = gpu_find(ev)
        cap = max(16, ev.n // 10 + 16)
        n_toc, n_off, n_hits = _noalloc(lib, ev, cap)
        assert len(g_off) > 3
        assert np.array_equal(n_toc, g_toc)
        assert np.array_equal(n_off, g_off)
        assert np.array_equal(n_hits, g_hits)


def test_noalloc_rejects_oversize():
    lib = tpc.load_library()
    lib.tpc_find_tracks_noalloc.restype = C.c_int
    dummy = torch.zeros(8, dtype=torch.int64, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    rc = lib.tpc_find_tracks_noalloc(None, p, p, p, C.c_int64(65537), p, C.c_int32(1), p, p, p, p, p,
                                     C.c_int32(16), None)
    assert rc == tpc.TPC_ERR_CAPACITY
    rc = lib.tpc_find_tracks_noalloc(None, p, p, p, C.c_int64(100), p, C.c_int32(5), p, p, p, p, p,
                                     C.c_int32(16), None)
    assert rc == tpc.TPC_ERR_CAPACITY
