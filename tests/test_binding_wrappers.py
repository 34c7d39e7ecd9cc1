"""Every public wrapper of the binding, driven end to end on CPU (no GPU).

The library is replaced by a stub that checks each call's argument count
against the argtypes the binding declares for the real library and returns
TPC_OK; the device check of the tensors is relaxed to "right dtype,
contiguous".  So each wrapper's own code runs: its tensor checks, its size
checks (undersized buffers must be refused with the buffer's name) and its
library call with the declared arity.  A slip in a wrapper's call into the
checks or into the library fails here, not on a GPU machine.
"""
import ctypes as C

import pytest

torch = pytest.importorskip("torch")

from paper_2412_13755_gb300 import tpc  # noqa: E402


class StubLib:
    def __init__(self, real):
        self.real = real
        self.calls = []

    def __getattr__(self, name):
        real_f = getattr(self.real, name)
        if name in ("tpc_field_voxels", "tpc_cluster_workspace_bytes",
                    "tpc_sides_workspace_bytes"):  # host-only: the real one
            return real_f

        def f(*args):
            if real_f.argtypes is not None:
                assert len(args) == len(real_f.argtypes), (name, len(args), len(real_f.argtypes))
            self.calls.append(name)
            if name == "tpc_last_error":
                return 0
            return tpc.TPC_OK

        return f


def _need_cpu(t, dtype, name):
    if not isinstance(t, torch.Tensor) or t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")


@pytest.fixture()
def stub(monkeypatch):
    real = tpc.load_library()
    s = StubLib(real)
    monkeypatch.setattr(tpc, "load_library", lambda *a, **k: s)
    monkeypatch.setattr(tpc, "_need", _need_cpu)
    monkeypatch.setattr(tpc, "_stream", lambda stream: None)
    return s


def i32(n):
    return torch.zeros(n, dtype=torch.int32)


def f32(*s):
    return torch.zeros(*s, dtype=torch.float32)


def f64(*s):
    return torch.zeros(*s, dtype=torch.float64)


def u16(n):
    return torch.zeros(n, dtype=torch.uint16)


def i64(n):
    return torch.zeros(n, dtype=torch.int64)


CTX = C.c_void_p(0x1234)


def _load(stub, n):
    tpc.tpc_load_clusters(CTX, f32(n), f32(n), u16(n), None, i64(37), 1)
    assert stub.calls[-1] == "tpc_load_clusters"


def test_find_and_autotune(stub):
    n = 500
    _load(stub, n)
    tpc.tpc_find_tracks(CTX, i32(n), i32(61), i32(n), i32(1))
    assert stub.calls[-1] == "tpc_find_tracks"
    best = tpc.tpc_autotune(CTX, i32(n), i32(61), i32(n), i32(1))
    assert stub.calls[-1] == "tpc_autotune" and isinstance(best, tpc.Tune)
    for fn in (tpc.tpc_find_tracks, tpc.tpc_autotune):
        with pytest.raises(ValueError, match="track_of_cluster"):
            fn(CTX, i32(n - 1), i32(61), i32(n), i32(1))
        with pytest.raises(ValueError, match="trk_hits"):
            fn(CTX, i32(n), i32(61), i32(n - 1), i32(1))
        with pytest.raises(TypeError, match="trk_off"):
            fn(CTX, i32(n), f32(61), i32(n), i32(1))
    tpc.tpc_set_tune(CTX, tpc.Tune(4, 2))
    tpc.tpc_set_tune(CTX, None)


def test_load_refusals(stub):
    with pytest.raises(ValueError, match="evt_sector_off"):
        tpc.tpc_load_clusters(CTX, f32(10), f32(10), u16(10), None, i64(36), 1)
    with pytest.raises(ValueError, match="charge"):
        tpc.tpc_load_clusters(CTX, f32(10), f32(10), u16(10), u16(9), i64(37), 1)
    with pytest.raises(TypeError, match="row"):
        tpc.tpc_load_clusters(CTX, f32(10), f32(10), i32(10), None, i64(37), 1)


def test_fit(stub):
    T = 7
    tpc.tpc_fit_tracks(CTX, i32(T + 1), i32(100), T, i32(1), f32(T, 5), f32(T, 15), f32(T), i32(T))
    tpc.tpc_fit_tracks(CTX, i32(T + 1), i32(100), T, None, f32(T, 5), f32(T, 15), f32(T), i32(T))
    assert stub.calls[-1] == "tpc_fit_tracks"
    with pytest.raises(ValueError, match="cov"):
        tpc.tpc_fit_tracks(CTX, i32(T + 1), i32(100), T, None, f32(T, 5), f32(T, 14), f32(T), i32(T))
    with pytest.raises(ValueError, match="trk_off"):
        tpc.tpc_fit_tracks(CTX, i32(T), i32(100), T, None, f32(T, 5), f32(T, 15), f32(T), i32(T))


def test_fit_fp32(stub):
    T = 5
    tpc.tpc_fit_tracks_fp32(CTX, i32(T + 1), i32(100), T, i32(1), f32(T, 5), f32(T, 15), f32(T), i32(T))
    assert stub.calls[-1] == "tpc_fit_tracks_fp32"
    with pytest.raises(ValueError, match="tpc_fit_tracks_fp32.*chi2"):
        tpc.tpc_fit_tracks_fp32(CTX, i32(T + 1), i32(100), T, None, f32(T, 5), f32(T, 15), f32(T - 1), i32(T))


def test_adjoint(stub):
    T = 9
    tpc.tpc_fit_adjoint(CTX, i32(T + 1), i32(100), T, f64(216), f64(1), f64(216))
    tpc.tpc_fit_adjoint(CTX, i32(T + 1), i32(100), T, f64(216), f64(1), None)
    assert stub.calls[-1] == "tpc_fit_adjoint"
    with pytest.raises(ValueError, match="grad"):
        tpc.tpc_fit_adjoint(CTX, i32(T + 1), i32(100), T, f64(216), f64(1), f64(200))
    with pytest.raises(TypeError, match="align"):
        tpc.tpc_fit_adjoint(CTX, i32(T + 1), i32(100), T, f32(216), f64(1), None)


def test_adjoint_field(stub):
    T = 3
    g = tpc.field_grid(8, 4, 5, -0.2, 2.5, 0.01)
    nv = tpc.tpc_field_voxels(g)
    assert nv == 36 * 8 * 4 * 5
    tpc.tpc_fit_adjoint_field(CTX, i32(T + 1), i32(50), T, f64(216), g, f64(nv, 3), f64(1),
                              f64(216), f64(nv, 3))
    tpc.tpc_fit_adjoint_field(CTX, i32(T + 1), i32(50), T, f64(216), g, f64(nv, 3), f64(1))
    assert stub.calls[-1] == "tpc_fit_adjoint_field"
    with pytest.raises(ValueError, match="grad_field"):
        tpc.tpc_fit_adjoint_field(CTX, i32(T + 1), i32(50), T, f64(216), g, f64(nv, 3), f64(1),
                                  f64(216), f64(nv - 1, 3))
    with pytest.raises(ValueError, match="invalid field grid"):
        tpc.tpc_fit_adjoint_field(CTX, i32(T + 1), i32(50), T, f64(216),
                                  tpc.field_grid(7, 4, 5, 0, 1, 1), f64(nv, 3), f64(1))


def test_noalloc(stub):
    n = 300
    args = (f32(n), f32(n), u16(n), i64(37), 1, i32(n), i32(46), i32(n), i32(1), i32(1))
    tpc.tpc_find_tracks_noalloc(*args)
    tpc.tpc_find_tracks_noalloc(*args, params=tpc.Params())
    assert stub.calls[-1] == "tpc_find_tracks_noalloc"
    bad = list(args)
    bad[7] = i32(n - 1)
    with pytest.raises(ValueError, match="trk_hits"):
        tpc.tpc_find_tracks_noalloc(*bad)
    bad = list(args)
    bad[9] = i32(0)
    with pytest.raises(ValueError, match="status_dev"):
        tpc.tpc_find_tracks_noalloc(*bad)


def test_status_and_timing_calls(stub):
    assert isinstance(tpc.tpc_get_stats(CTX), tpc.Stats)
    tpc.tpc_reset_status(CTX)
    tpc.tpc_stage_timing(CTX, True)
    t = tpc.tpc_stage_times(CTX)
    assert set(t) == set(tpc.STAGE_NAMES)


def test_tracker_methods(stub):
    """The Tracker's convenience methods, on a Tracker whose context and
    workspace were set up by hand (its constructor needs a CUDA device)."""
    tr = object.__new__(tpc.Tracker)
    tr.device = torch.device("cpu")
    tr.ctx = CTX
    tr.max_clusters = 400
    tr.max_events = 1
    tr.n = 0
    n = 400
    tr.load(f32(n), f32(n), u16(n), i64(37), 1)
    out = tr.find()
    assert out[0].numel() == n and out[2].numel() == n
    assert isinstance(tr.autotune(), tpc.Tune)
    tr.set_tune(None)
    tr.fit(out[1], out[2], 5, out[3])
    tr.adjoint(out[1], out[2], 5, f64(216))
    g = tpc.field_grid(4, 2, 2, -0.2, 5.0, 0.01)
    tr.adjoint_field(out[1], out[2], 5, g, f64(tpc.tpc_field_voxels(g), 3))
    tr.stats()
    tr.reset_status()
    tr.stage_timing(True)
    tr.stage_times()
    assert "tpc_autotune" in stub.calls and "tpc_fit_adjoint_field" in stub.calls
    tr.ctx = None  # nothing to destroy


def test_default_track_capacity_fits_small_contexts(stub):
    """The default track capacity never exceeds what the context takes
    (max_clusters tracks): a 12-cluster batch gets 12, not 12 // 10 + 16."""
    tr = object.__new__(tpc.Tracker)
    tr.device = torch.device("cpu")
    tr.ctx = CTX
    tr.max_clusters = 12
    tr.max_events = 1
    tr.n = 0
    tr.load(f32(12), f32(12), u16(12), i64(37), 1)
    toc, trk_off, hits, ntd = tr.alloc_find_outputs()
    assert trk_off.numel() - 1 <= 12
    tr.max_clusters = 10_000
    tr.n = 5000
    assert tr.alloc_find_outputs()[1].numel() - 1 == 5000 // 10 + 16
    tr.ctx = None


def test_batch_and_graph(stub):
    n, cap = 300, 46
    find = (i32(n), i32(cap + 1), i32(n), i32(1))
    fit = (f32(cap, 5), f32(cap, 15), f32(cap), i32(cap))
    tpc.tpc_track_batch(CTX, f32(n), f32(n), u16(n), None, i64(37), 1, find, fit)
    assert stub.calls[-1] == "tpc_track_batch"
    tpc.tpc_track_batch(CTX, f32(n), f32(n), u16(n), u16(n), i64(37), 1, find)
    tpc.tpc_graph_capture(CTX, f32(n), f32(n), u16(n), None, i64(37), 1, find, fit)
    assert stub.calls[-1] == "tpc_graph_capture"
    tpc.tpc_graph_launch(CTX)
    assert stub.calls[-1] == "tpc_graph_launch"
    with pytest.raises(ValueError, match="trk_hits"):
        tpc.tpc_track_batch(CTX, f32(n), f32(n), u16(n), None, i64(37), 1,
                            (i32(n), i32(cap + 1), i32(n - 1), i32(1)), fit)
    with pytest.raises(ValueError, match="cov"):
        tpc.tpc_graph_capture(CTX, f32(n), f32(n), u16(n), None, i64(37), 1, find,
                              (f32(cap, 5), f32(cap - 1, 15), f32(cap), i32(cap)))
    tr = object.__new__(tpc.Tracker)
    tr.device = torch.device("cpu")
    tr.ctx = CTX
    tr.max_clusters = n
    tr.max_events = 1
    tr.n = 0
    tr.track_batch(f32(n), f32(n), u16(n), i64(37), 1, find, tr.alloc_fit_outputs(cap))
    tr.capture(f32(n), f32(n), u16(n), i64(37), 1, find)
    tr.replay()
    assert stub.calls[-3:] == ["tpc_track_batch", "tpc_graph_capture", "tpc_graph_launch"]
    tr.ctx = None


def test_fit_ex(stub):
    T = 6
    o = tpc.fit_options(1e-4, 2e-6, 0.13957, outward=False)
    tpc.tpc_fit_tracks_ex(CTX, i32(T + 1), i32(100), T, i32(1), o, f32(T, 5), f32(T, 15), f32(T), i32(T),
                          f64(100, 20))
    tpc.tpc_fit_tracks_ex(CTX, i32(T + 1), i32(100), T, None, None, f32(T, 5), f32(T, 15), f32(T), i32(T))
    assert stub.calls[-1] == "tpc_fit_tracks_ex"
    with pytest.raises(ValueError, match="smoothed"):
        tpc.tpc_fit_tracks_ex(CTX, i32(T + 1), i32(100), T, None, o, f32(T, 5), f32(T, 15), f32(T), i32(T),
                              f64(99, 20))
    with pytest.raises(TypeError, match="smoothed"):
        tpc.tpc_fit_tracks_ex(CTX, i32(T + 1), i32(100), T, None, o, f32(T, 5), f32(T, 15), f32(T), i32(T),
                              f32(100, 20))
    tr = object.__new__(tpc.Tracker)
    tr.device = torch.device("cpu")
    tr.ctx = CTX
    par, cov, chi2, ndf, sm = tr.fit_ex(i32(T + 1), i32(100), T, o, smooth=True)
    assert sm.shape == (100, 20) and par.shape == (T, 5)
    tr.ctx = None


def test_find_clusters(stub):
    n_ev, n_time = 1, 32
    nb = tpc.tpc_cluster_workspace_bytes(n_ev, n_time)
    assert nb > 0 and tpc.tpc_cluster_workspace_bytes(0, 32) == 0 and tpc.tpc_cluster_workspace_bytes(1, 5000) == 0
    d = torch.zeros(36 * 152, n_time, 160, dtype=torch.uint16)
    outs = (f32(100), f32(100), u16(100), u16(100), i64(37), i32(1), i32(2))
    tpc.tpc_find_clusters(d, n_ev, torch.zeros(nb, dtype=torch.uint8), outs)
    assert stub.calls[-1] == "tpc_find_clusters"
    with pytest.raises(ValueError, match="workspace"):
        tpc.tpc_find_clusters(d, n_ev, torch.zeros(nb - 1, dtype=torch.uint8), outs)
    with pytest.raises(ValueError, match="digits"):
        tpc.tpc_find_clusters(torch.zeros(36 * 152, n_time, 150, dtype=torch.uint16), n_ev,
                              torch.zeros(nb, dtype=torch.uint8), outs)
    with pytest.raises(ValueError, match="status_dev"):
        tpc.tpc_find_clusters(d, n_ev, torch.zeros(nb, dtype=torch.uint8), outs[:6] + (i32(1),))


def test_match_sides(stub):
    T, E, cap = 50, 2, 64
    nb = tpc.tpc_sides_workspace_bytes(T, E, cap)
    assert nb > 0 and tpc.tpc_sides_workspace_bytes(-1, 1, 1) == 0 and tpc.tpc_sides_workspace_bytes(5, 0, 1) == 0
    assert tpc.tpc_sides_workspace_bytes(T, E, 2 * cap) > nb
    out = (i32(T), f64(T), f64(T, 6), f64(T, 21), f64(T), i32(T), f64(T))
    ws = torch.zeros(nb, dtype=torch.uint8)
    o = tpc.sides_options(gap_max=5)
    tpc.tpc_match_sides(CTX, i32(T + 1), i32(100), T, i32(1), o, ws, cap, out, i32(1), E)
    tpc.tpc_match_sides(CTX, i32(T + 1), i32(100), T, None, None, ws, cap, out, i32(1), E)
    assert stub.calls[-1] == "tpc_match_sides"
    for k, name in enumerate(("partner", "t0", "params6", "cov6", "chi2", "ndf", "dchi2")):
        short = list(out)
        short[k] = short[k].reshape(-1)[:-1].clone()
        with pytest.raises(ValueError, match=name):
            tpc.tpc_match_sides(CTX, i32(T + 1), i32(100), T, None, None, ws, cap, tuple(short), i32(1), E)
    with pytest.raises(ValueError, match="workspace"):
        tpc.tpc_match_sides(CTX, i32(T + 1), i32(100), T, None, None, ws[:-1].clone(), cap, out, i32(1), E)
    with pytest.raises(ValueError, match="trk_off"):
        tpc.tpc_match_sides(CTX, i32(T), i32(100), T, None, None, ws, cap, out, i32(1), E)
    with pytest.raises(TypeError, match="cov6"):
        tpc.tpc_match_sides(CTX, i32(T + 1), i32(100), T, None, None, ws, cap,
                            out[:3] + (f32(T, 21),) + out[4:], i32(1), E)
    tr = object.__new__(tpc.Tracker)
    tr.device = torch.device("cpu")
    tr.ctx = CTX
    tr.n_events_loaded = E
    r = tr.match_sides(i32(T + 1), i32(100), T)
    assert r["params6"].shape == (T, 6) and r["cov6"].shape == (T, 21) and r["partner"].shape == (T,)
    assert r["n_pairs"].shape == (1,)
    tr.ctx = None
