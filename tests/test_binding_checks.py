"""The binding's host-side buffer checks (no GPU): the C ABI takes plain
pointers, so the binding refuses, before any launch, a buffer smaller than
what the call writes.  Run here on CPU tensors; the GPU test of the same
refusals goes through the Tracker."""
import pytest

torch = pytest.importorskip("torch")

from paper_2412_13755_gb300 import tpc  # noqa: E402


def i32(n):
    return torch.empty(n, dtype=torch.int32)


def test_find_outputs_sized_by_the_loaded_count():
    n = 1000
    tpc.check_find_outputs(n, i32(n), i32(2), i32(n), i32(1))
    for args, name in (((i32(n - 1), i32(2), i32(n), i32(1)), "track_of_cluster"),
                       ((i32(n), i32(2), i32(n - 1), i32(1)), "trk_hits"),
                       ((i32(n), i32(1), i32(n), i32(1)), "trk_off"),
                       ((i32(n), i32(2), i32(n), i32(0)), "n_tracks_dev")):
        with pytest.raises(ValueError, match=name):
            tpc.check_find_outputs(n, *args, what="tpc_autotune")
    # one-element buffers, as allocated for an empty batch, against a full load
    with pytest.raises(ValueError, match="track_of_cluster"):
        tpc.check_find_outputs(137_000_000, i32(1), i32(2), i32(1), i32(1))


def test_fit_buffers_sized_by_the_track_count():
    T = 50
    f32 = lambda *s: torch.empty(*s, dtype=torch.float32)  # noqa: E731
    tpc.check_fit_buffers(T, i32(T + 1), f32(T, 5), f32(T, 15), f32(T), i32(T))
    tpc.check_fit_buffers(0, i32(1), f32(0, 5), f32(0, 15), f32(0), i32(0))
    for args, name in (((i32(T), f32(T, 5), f32(T, 15), f32(T), i32(T)), "trk_off"),
                       ((i32(T + 1), f32(T - 1, 5), f32(T, 15), f32(T), i32(T)), "params"),
                       ((i32(T + 1), f32(T, 5), f32(T, 14), f32(T), i32(T)), "cov"),
                       ((i32(T + 1), f32(T, 5), f32(T, 15), f32(T - 1), i32(T)), "chi2"),
                       ((i32(T + 1), f32(T, 5), f32(T, 15), f32(T), i32(T - 1)), "ndf")):
        with pytest.raises(ValueError, match=name):
            tpc.check_fit_buffers(T, *args)
    with pytest.raises(ValueError, match="n_tracks"):
        tpc.check_fit_buffers(-1, i32(1), f32(1, 5), f32(1, 15), f32(1), i32(1))


def test_adjoint_buffers():
    f64 = lambda n: torch.empty(n, dtype=torch.float64)  # noqa: E731
    tpc.check_adjoint_buffers(10, i32(11), f64(216), f64(1), None)
    tpc.check_adjoint_buffers(10, i32(11), f64(216), f64(1), f64(216))
    for args, name in (((i32(10), f64(216), f64(1), None), "trk_off"),
                       ((i32(11), f64(215), f64(1), None), "align"),
                       ((i32(11), f64(216), f64(0), None), "chi2_total"),
                       ((i32(11), f64(216), f64(1), f64(215)), "grad")):
        with pytest.raises(ValueError, match=name):
            tpc.check_adjoint_buffers(10, *args)


def test_field_buffers():
    f64 = lambda *s: torch.empty(*s, dtype=torch.float64)  # noqa: E731
    nv = 5760
    tpc.check_field_buffers(nv, f64(nv, 3), None)
    tpc.check_field_buffers(nv, f64(nv, 3), f64(nv, 3))
    with pytest.raises(ValueError, match="field holds"):
        tpc.check_field_buffers(nv, f64(nv - 1, 3), None)
    with pytest.raises(ValueError, match="grad_field"):
        tpc.check_field_buffers(nv, f64(nv, 3), f64(nv, 2))
    with pytest.raises(ValueError, match="invalid field grid"):
        tpc.check_field_buffers(-1, f64(nv, 3), None)


def test_load_inputs():
    f32 = lambda n: torch.empty(n, dtype=torch.float32)  # noqa: E731
    u16 = lambda n: torch.empty(n, dtype=torch.int16)  # noqa: E731  (size only)
    i64 = lambda n: torch.empty(n, dtype=torch.int64)  # noqa: E731
    n = 100
    tpc.check_load_inputs(f32(n), f32(n), u16(n), None, i64(37), 1)
    tpc.check_load_inputs(f32(n), f32(n), u16(n), u16(n), i64(73), 2)
    for args, name in (((f32(n), f32(n - 1), u16(n), None, i64(37), 1), "z"),
                       ((f32(n), f32(n), u16(n - 1), None, i64(37), 1), "row"),
                       ((f32(n), f32(n), u16(n), u16(n - 1), i64(37), 1), "charge"),
                       ((f32(n), f32(n), u16(n), None, i64(37), 2), "evt_sector_off"),
                       ((f32(n), f32(n), u16(n), None, i64(37), 0), "n_events")):
        with pytest.raises(ValueError, match=name):
            tpc.check_load_inputs(*args)
