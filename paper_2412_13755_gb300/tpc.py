"""Thin Python binding of libtpctrack (include/tpc_track.h).

Argument marshalling only: tensors are passed to the C ABI as device
pointers, every step of the tracking path runs in the library's CUDA
kernels.  PyTorch provides device memory and streams.  There is no fallback:
if the library is not built, or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import build as _build

TPC_OK, TPC_ERR_ARG, TPC_ERR_CUDA, TPC_ERR_CAPACITY, TPC_ERR_TIMEOUT, TPC_ERR_STATE, \
    TPC_ERR_INPUT = range(7)
STATUS_NAMES = {0: "TPC_OK", 1: "TPC_ERR_ARG", 2: "TPC_ERR_CUDA", 3: "TPC_ERR_CAPACITY",
                4: "TPC_ERR_TIMEOUT", 5: "TPC_ERR_STATE", 6: "TPC_ERR_INPUT"}

EXPORTS = ("tpc_default_params", "tpc_create", "tpc_destroy", "tpc_workspace_bytes",
           "tpc_set_workspace", "tpc_load_clusters", "tpc_find_tracks", "tpc_fit_tracks",
           "tpc_fit_adjoint", "tpc_get_stats", "tpc_last_error", "tpc_reset_status",
           "tpc_stage_timing", "tpc_stage_times", "tpc_find_tracks_noalloc", "tpc_set_tune",
           "tpc_autotune", "tpc_field_voxels", "tpc_fit_adjoint_field", "tpc_track_batch",
           "tpc_graph_capture", "tpc_graph_launch", "tpc_fit_tracks_ex", "tpc_cluster_workspace_bytes",
           "tpc_find_clusters", "tpc_sides_workspace_bytes", "tpc_match_sides", "tpc_fit_tracks_fp32")
STAGE_NAMES = ("bin", "neighbours", "links", "chains", "tracklets", "select", "merge_cand",
               "match", "output", "fit", "adjoint", "find_total", "sides")


class Params(C.Structure):
    _fields_ = [
        ("win_y", C.c_float), ("win_z", C.c_float), ("chi2_link", C.c_float),
        ("sigma_y2", C.c_float), ("sigma_z2", C.c_float),
        ("max_gap", C.c_int32), ("n_seg", C.c_int32), ("n_min", C.c_int32),
        ("merge_max_row_gap", C.c_int32), ("merge_max_overlap", C.c_int32),
        ("merge_z_slope", C.c_float), ("merge_z_margin", C.c_float),
        ("chi2_merge", C.c_float), ("chi2_ext", C.c_float), ("ext_max_miss", C.c_int32),
        ("bz", C.c_float), ("prior", C.c_float * 5), ("seed_snp_max", C.c_float),
        ("seed_qpt_max", C.c_float), ("snp_max", C.c_float),
        ("fp64_ratio", C.c_float), ("fp64_det", C.c_float), ("fp64_weak_qpt", C.c_float),
    ]


class Tune(C.Structure):
    _fields_ = [("lane_blocks_per_sm", C.c_int32), ("lane_tile", C.c_int32),
                ("nb_sub_lanes", C.c_int32)]


class FitOptions(C.Structure):
    """Kalman-filter variants of the fit (tpc_fit_options)."""
    _fields_ = [("mat_x_x0", C.c_float), ("mat_eloss", C.c_float), ("mass", C.c_float),
                ("direction", C.c_int32)]


def fit_options(mat_x_x0=0.0, mat_eloss=0.0, mass=0.13957, outward=False) -> FitOptions:
    return FitOptions(float(mat_x_x0), float(mat_eloss), float(mass), 1 if outward else 0)


class SidesOptions(C.Structure):
    """Options of the A/C-side association with t0 (tpc_sides_options)."""
    _fields_ = [("n_min", C.c_int32), ("gap_max", C.c_int32), ("chi2_junction", C.c_double),
                ("z_membrane", C.c_double), ("z_pre", C.c_double), ("chi2_joint", C.c_double),
                ("t0_prior", C.c_double), ("v_drift", C.c_double)]


def sides_options(n_min=10, gap_max=8, chi2_junction=30.0, z_membrane=3.0, z_pre=10.0, chi2_joint=40.0,
                  t0_prior=1.0, v_drift=2.58) -> SidesOptions:
    """The library's defaults unless overridden."""
    return SidesOptions(int(n_min), int(gap_max), float(chi2_junction), float(z_membrane), float(z_pre),
                        float(chi2_joint), float(t0_prior), float(v_drift))


class BatchOutputs(C.Structure):
    """Outputs of one batch (tpc_batch_outputs): device pointers."""
    _fields_ = [("track_of_cluster", C.c_void_p), ("trk_off", C.c_void_p), ("trk_hits", C.c_void_p),
                ("n_tracks_dev", C.c_void_p), ("track_cap", C.c_int32), ("params", C.c_void_p),
                ("cov", C.c_void_p), ("chi2", C.c_void_p), ("ndf", C.c_void_p)]


class FieldGrid(C.Structure):
    """Voxel grid of a displacement field (tpc_field_grid)."""
    _fields_ = [("n_band", C.c_int32), ("n_y", C.c_int32), ("n_z", C.c_int32),
                ("u_lo", C.c_float), ("u_inv", C.c_float), ("z_inv", C.c_float)]


def field_grid(n_band, n_y, n_z, u_lo, u_inv, z_inv) -> FieldGrid:
    return FieldGrid(int(n_band), int(n_y), int(n_z), float(u_lo), float(u_inv), float(z_inv))


class Stats(C.Structure):
    _fields_ = [
        ("n_clusters", C.c_int64), ("n_segments", C.c_int32), ("n_tracklets", C.c_int32),
        ("n_merge_cand", C.c_int32), ("n_merges", C.c_int32), ("n_tracks", C.c_int32),
        ("n_fp64_updates", C.c_int32), ("status", C.c_int32), ("status_detail", C.c_int32),
        ("n_launches", C.c_int64), ("n_kf_steps", C.c_int64),
        ("n_nb_second", C.c_int32), ("n_nb_dense", C.c_int32), ("n_nb_full", C.c_int32),
        ("reserved", C.c_int32),
    ]


_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Loads libtpctrack.so (building it first if asked)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libtpctrack.so is not built (run __graft_entry__.build())")
    lib = C.CDLL(_build.LIB)
    vp, i32, i64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
    lib.tpc_default_params.argtypes = [vp]
    lib.tpc_default_params.restype = None
    lib.tpc_create.argtypes = [vp, vp]
    lib.tpc_destroy.argtypes = [vp]
    lib.tpc_destroy.restype = None
    lib.tpc_workspace_bytes.argtypes = [vp, i64, i32]
    lib.tpc_workspace_bytes.restype = sz
    lib.tpc_set_workspace.argtypes = [vp, vp, sz, i64, i32]
    lib.tpc_load_clusters.argtypes = [vp, vp, vp, vp, vp, i64, vp, i32, vp]
    lib.tpc_find_tracks.argtypes = [vp, vp, vp, vp, vp, i32, vp]
    lib.tpc_fit_tracks.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp, vp, vp]
    lib.tpc_fit_tracks_fp32.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp, vp, vp]
    lib.tpc_fit_adjoint.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp]
    lib.tpc_get_stats.argtypes = [vp, vp, vp]
    lib.tpc_last_error.argtypes = [vp, C.c_char_p, sz]
    lib.tpc_reset_status.argtypes = [vp, vp]
    lib.tpc_stage_timing.argtypes = [vp, C.c_int]
    lib.tpc_set_tune.argtypes = [vp, vp]
    lib.tpc_autotune.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp]
    lib.tpc_stage_times.argtypes = [vp, vp]
    lib.tpc_field_voxels.argtypes = [vp]
    lib.tpc_field_voxels.restype = i64
    lib.tpc_fit_adjoint_field.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp, vp, vp, vp]
    lib.tpc_find_tracks_noalloc.argtypes = [vp, vp, vp, vp, i64, vp, i32, vp, vp, vp, vp, vp, i32,
                                            vp]
    lib.tpc_track_batch.argtypes = [vp, vp, vp, vp, vp, i64, vp, i32, vp, vp]
    lib.tpc_graph_capture.argtypes = [vp, vp, vp, vp, vp, i64, vp, i32, vp]
    lib.tpc_graph_launch.argtypes = [vp, vp]
    lib.tpc_fit_tracks_ex.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.tpc_cluster_workspace_bytes.argtypes = [i32, i32]
    lib.tpc_cluster_workspace_bytes.restype = sz
    lib.tpc_sides_workspace_bytes.argtypes = [i32, i32, i32]
    lib.tpc_sides_workspace_bytes.restype = sz
    lib.tpc_match_sides.argtypes = [vp, vp, vp, i32, vp, vp, vp, sz, i32] + [vp] * 8 + [vp]
    lib.tpc_find_clusters.argtypes = [vp, i32, i32, i32, vp, sz, vp, vp, vp, vp, vp, i64, vp, vp, vp]
    for name in EXPORTS:
        f = getattr(lib, name)
        if name not in ("tpc_default_params", "tpc_destroy", "tpc_workspace_bytes",
                        "tpc_field_voxels", "tpc_cluster_workspace_bytes", "tpc_sides_workspace_bytes"):
            f.restype = C.c_int
    _lib = lib
    return lib


def default_params(**kw) -> Params:
    p = Params()
    load_library().tpc_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "prior":
            for i in range(5):
                p.prior[i] = v[i]
        else:
            setattr(p, k, v)
    return p


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class TPCError(RuntimeError):
    pass


def _check(ctx, rc, what):
    if rc != TPC_OK:
        buf = C.create_string_buffer(512)
        load_library().tpc_last_error(ctx, buf, 512)
        raise TPCError(f"{what}: {STATUS_NAMES.get(rc, rc)} {buf.value.decode(errors='replace')}")


def _need(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous CUDA {dtype} tensor")


# The C ABI takes plain pointers: it cannot see how large a caller's buffer
# is.  The binding records the cluster count of each context's last load and
# refuses, before any launch, a buffer smaller than what the call writes.
_loaded_n: dict[int, int] = {}


def _need_len(t, n, name, what):
    if t.numel() < n:
        raise ValueError(f"{what}: {name} holds {t.numel()} entries, the call needs {n}")


def check_find_outputs(n, track_of_cluster, trk_off, trk_hits, n_tracks_dev, what="tpc_find_tracks"):
    """tpc_find_tracks and tpc_autotune write n entries of track_of_cluster
    and trk_hits (n = clusters loaded), trk_off.numel() entries of trk_off
    (the track capacity plus one) and one of n_tracks_dev."""
    _need_len(track_of_cluster, n, "track_of_cluster", what)
    _need_len(trk_hits, n, "trk_hits", what)
    _need_len(trk_off, 2, "trk_off", what)
    _need_len(n_tracks_dev, 1, "n_tracks_dev", what)


def check_fit_buffers(n_tracks, trk_off, params, cov, chi2, ndf, what="tpc_fit_tracks"):
    """tpc_fit_tracks reads trk_off[n_tracks + 1] and writes n_tracks rows of
    params (5), cov (15), chi2 and ndf."""
    T = int(n_tracks)
    if T < 0:
        raise ValueError(f"{what}: n_tracks {T} < 0")
    _need_len(trk_off, T + 1, "trk_off", what)
    _need_len(params, 5 * T, "params", what)
    _need_len(cov, 15 * T, "cov", what)
    _need_len(chi2, T, "chi2", what)
    _need_len(ndf, T, "ndf", what)


def check_adjoint_buffers(n_tracks, trk_off, align, chi2_total, grad, what="tpc_fit_adjoint"):
    """tpc_fit_adjoint reads trk_off[n_tracks + 1] and align[216] and writes
    chi2_total[1] and, when given, grad[216]."""
    T = int(n_tracks)
    if T < 0:
        raise ValueError(f"{what}: n_tracks {T} < 0")
    _need_len(trk_off, T + 1, "trk_off", what)
    _need_len(align, 216, "align", what)
    _need_len(chi2_total, 1, "chi2_total", what)
    if grad is not None:
        _need_len(grad, 216, "grad", what)


# --- the C ABI, one Python function per entry point --------------------------

def tpc_create(params: Params | None = None):
    ctx = C.c_void_p()
    rc = load_library().tpc_create(C.byref(ctx), C.byref(params) if params is not None else None)
    if rc != TPC_OK:
        raise TPCError(f"tpc_create: {STATUS_NAMES.get(rc, rc)}")
    return ctx


def tpc_destroy(ctx):
    _loaded_n.pop(ctx.value, None)
    load_library().tpc_destroy(ctx)


def tpc_workspace_bytes(ctx, max_clusters: int, max_events: int) -> int:
    return int(load_library().tpc_workspace_bytes(ctx, int(max_clusters), int(max_events)))


def tpc_set_workspace(ctx, ws: torch.Tensor, max_clusters: int, max_events: int):
    _need(ws, torch.uint8, "workspace")
    rc = load_library().tpc_set_workspace(ctx, _ptr(ws), ws.numel(), int(max_clusters),
                                          int(max_events))
    _check(ctx, rc, "tpc_set_workspace")


def check_load_inputs(y, z, row, charge, evt_sector_off, n_events, what="tpc_load_clusters"):
    """tpc_load_clusters reads n = y.numel() entries of y, z, row (and
    charge) and 36 n_events + 1 entries of evt_sector_off."""
    n = y.numel()
    _need_len(z, n, "z", what)
    _need_len(row, n, "row", what)
    if charge is not None:
        _need_len(charge, n, "charge", what)
    if int(n_events) < 1:
        raise ValueError(f"{what}: n_events {int(n_events)} < 1")
    _need_len(evt_sector_off, 36 * int(n_events) + 1, "evt_sector_off", what)


def tpc_load_clusters(ctx, y, z, row, charge, evt_sector_off, n_events, stream=None):
    _need(y, torch.float32, "y")
    _need(z, torch.float32, "z")
    _need(row, torch.uint16, "row")
    if charge is not None:
        _need(charge, torch.uint16, "charge")
    _need(evt_sector_off, torch.int64, "evt_sector_off")
    check_load_inputs(y, z, row, charge, evt_sector_off, n_events)
    rc = load_library().tpc_load_clusters(ctx, _ptr(y), _ptr(z), _ptr(row), _ptr(charge),
                                          y.numel(), _ptr(evt_sector_off), int(n_events),
                                          _stream(stream))
    _check(ctx, rc, "tpc_load_clusters")
    _loaded_n[ctx.value] = y.numel()


def tpc_find_tracks(ctx, track_of_cluster, trk_off, trk_hits, n_tracks_dev, stream=None):
    for t, n in ((track_of_cluster, "track_of_cluster"), (trk_off, "trk_off"),
                 (trk_hits, "trk_hits"), (n_tracks_dev, "n_tracks_dev")):
        _need(t, torch.int32, n)
    check_find_outputs(_loaded_n.get(ctx.value, 0), track_of_cluster, trk_off, trk_hits, n_tracks_dev)
    rc = load_library().tpc_find_tracks(ctx, _ptr(track_of_cluster), _ptr(trk_off), _ptr(trk_hits),
                                        _ptr(n_tracks_dev), trk_off.numel() - 1, _stream(stream))
    _check(ctx, rc, "tpc_find_tracks")


def _fit_call(what, ctx, trk_off, trk_hits, n_tracks, n_tracks_dev, params, cov, chi2, ndf, stream):
    """tpc_fit_tracks and tpc_fit_tracks_fp32 take the same arguments."""
    _need(trk_off, torch.int32, "trk_off")
    _need(trk_hits, torch.int32, "trk_hits")
    for t, n in ((params, "params"), (cov, "cov"), (chi2, "chi2")):
        _need(t, torch.float32, n)
    _need(ndf, torch.int32, "ndf")
    if n_tracks_dev is not None:
        _need(n_tracks_dev, torch.int32, "n_tracks_dev")
    check_fit_buffers(n_tracks, trk_off, params, cov, chi2, ndf, what=what)
    fn = getattr(load_library(), what)
    rc = fn(ctx, _ptr(trk_off), _ptr(trk_hits), int(n_tracks), _ptr(n_tracks_dev), _ptr(params),
            _ptr(cov), _ptr(chi2), _ptr(ndf), _stream(stream))
    _check(ctx, rc, what)


def tpc_fit_tracks(ctx, trk_off, trk_hits, n_tracks, n_tracks_dev, params, cov, chi2, ndf,
                   stream=None):
    _fit_call("tpc_fit_tracks", ctx, trk_off, trk_hits, n_tracks, n_tracks_dev, params, cov, chi2, ndf,
              stream)


def tpc_fit_tracks_fp32(ctx, trk_off, trk_hits, n_tracks, n_tracks_dev, params, cov, chi2, ndf,
                        stream=None):
    """The fit with the covariance in FP32 and cancelling updates redone in
    FP64 (same arguments as tpc_fit_tracks)."""
    _fit_call("tpc_fit_tracks_fp32", ctx, trk_off, trk_hits, n_tracks, n_tracks_dev, params, cov, chi2,
              ndf, stream)


def tpc_fit_tracks_ex(ctx, trk_off, trk_hits, n_tracks, n_tracks_dev, options, params, cov, chi2, ndf,
                      smoothed=None, stream=None):
    _need(trk_off, torch.int32, "trk_off")
    _need(trk_hits, torch.int32, "trk_hits")
    for t, n in ((params, "params"), (cov, "cov"), (chi2, "chi2")):
        _need(t, torch.float32, n)
    _need(ndf, torch.int32, "ndf")
    if n_tracks_dev is not None:
        _need(n_tracks_dev, torch.int32, "n_tracks_dev")
    what = "tpc_fit_tracks_ex"
    check_fit_buffers(n_tracks, trk_off, params, cov, chi2, ndf, what)
    if smoothed is not None:
        _need(smoothed, torch.float64, "smoothed")
        # entries are written at 20 x (position in trk_hits)
        _need_len(smoothed, 20 * trk_hits.numel(), "smoothed", what)
    rc = load_library().tpc_fit_tracks_ex(ctx, _ptr(trk_off), _ptr(trk_hits), int(n_tracks),
                                          _ptr(n_tracks_dev), C.byref(options) if options is not None else None,
                                          _ptr(params), _ptr(cov), _ptr(chi2), _ptr(ndf), _ptr(smoothed),
                                          _stream(stream))
    _check(ctx, rc, what)


def tpc_sides_workspace_bytes(max_tracks: int, n_events: int, cand_cap: int) -> int:
    return int(load_library().tpc_sides_workspace_bytes(int(max_tracks), int(n_events), int(cand_cap)))


SIDES_OUT = (("partner", torch.int32, 1), ("t0", torch.float64, 1), ("params6", torch.float64, 6),
             ("cov6", torch.float64, 21), ("chi2", torch.float64, 1), ("ndf", torch.int32, 1),
             ("dchi2", torch.float64, 1))


def check_sides_buffers(n_tracks, trk_off, out, n_pairs_dev, workspace, need, what="tpc_match_sides"):
    """tpc_match_sides reads trk_off[n_tracks + 1] and writes n_tracks
    entries of each per-track output (partner, t0, params6 x 6, cov6 x 21,
    chi2, ndf, dchi2), one of n_pairs_dev, and uses need bytes of scratch."""
    T = int(n_tracks)
    if T < 0:
        raise ValueError(f"{what}: n_tracks {T} < 0")
    _need_len(trk_off, T + 1, "trk_off", what)
    for (name, _, k), t in zip(SIDES_OUT, out):
        _need_len(t, k * T, name, what)
    _need_len(n_pairs_dev, 1, "n_pairs_dev", what)
    if need == 0:
        raise ValueError(f"{what}: invalid sizes")
    if workspace.numel() * workspace.element_size() < need:
        raise ValueError(f"{what}: workspace holds {workspace.numel() * workspace.element_size()} bytes, "
                         f"the call needs {need}")


def tpc_match_sides(ctx, trk_off, trk_hits, n_tracks, n_tracks_dev, options, workspace, cand_cap, out,
                    n_pairs_dev, n_events, stream=None):
    """out = (partner, t0, params6, cov6, chi2, ndf, dchi2) as SIDES_OUT."""
    what = "tpc_match_sides"
    _need(trk_off, torch.int32, "trk_off")
    _need(trk_hits, torch.int32, "trk_hits")
    for (name, dt, _), t in zip(SIDES_OUT, out):
        _need(t, dt, name)
    _need(n_pairs_dev, torch.int32, "n_pairs_dev")
    if n_tracks_dev is not None:
        _need(n_tracks_dev, torch.int32, "n_tracks_dev")
    _need(workspace, torch.uint8, "workspace")
    need = tpc_sides_workspace_bytes(n_tracks, n_events, cand_cap)
    check_sides_buffers(n_tracks, trk_off, out, n_pairs_dev, workspace, need, what)
    rc = load_library().tpc_match_sides(ctx, _ptr(trk_off), _ptr(trk_hits), int(n_tracks), _ptr(n_tracks_dev),
                                        C.byref(options) if options is not None else None, _ptr(workspace),
                                        workspace.numel() * workspace.element_size(), int(cand_cap),
                                        *[_ptr(t) for t in out], _ptr(n_pairs_dev), _stream(stream))
    _check(ctx, rc, what)


def tpc_fit_adjoint(ctx, trk_off, trk_hits, n_tracks, align, chi2_total, grad=None, stream=None):
    _need(trk_off, torch.int32, "trk_off")
    _need(trk_hits, torch.int32, "trk_hits")
    _need(align, torch.float64, "align")
    _need(chi2_total, torch.float64, "chi2_total")
    if grad is not None:
        _need(grad, torch.float64, "grad")
    check_adjoint_buffers(n_tracks, trk_off, align, chi2_total, grad)
    rc = load_library().tpc_fit_adjoint(ctx, _ptr(trk_off), _ptr(trk_hits), int(n_tracks),
                                        _ptr(align), _ptr(chi2_total), _ptr(grad), _stream(stream))
    _check(ctx, rc, "tpc_fit_adjoint")


def tpc_field_voxels(grid: FieldGrid) -> int:
    return int(load_library().tpc_field_voxels(C.byref(grid)))


def check_field_buffers(n_voxels, field, grad_field, what="tpc_fit_adjoint_field"):
    """tpc_fit_adjoint_field reads field[3 n_voxels] and writes, when given,
    grad_field[3 n_voxels]."""
    if n_voxels < 0:
        raise ValueError(f"{what}: invalid field grid")
    _need_len(field, 3 * n_voxels, "field", what)
    if grad_field is not None:
        _need_len(grad_field, 3 * n_voxels, "grad_field", what)


def tpc_fit_adjoint_field(ctx, trk_off, trk_hits, n_tracks, align, grid: FieldGrid, field,
                          chi2_total, grad_align=None, grad_field=None, stream=None):
    _need(trk_off, torch.int32, "trk_off")
    _need(trk_hits, torch.int32, "trk_hits")
    _need(align, torch.float64, "align")
    _need(field, torch.float64, "field")
    _need(chi2_total, torch.float64, "chi2_total")
    for t, n in ((grad_align, "grad_align"), (grad_field, "grad_field")):
        if t is not None:
            _need(t, torch.float64, n)
    check_adjoint_buffers(n_tracks, trk_off, align, chi2_total, grad_align, "tpc_fit_adjoint_field")
    check_field_buffers(tpc_field_voxels(grid), field, grad_field)
    rc = load_library().tpc_fit_adjoint_field(ctx, _ptr(trk_off), _ptr(trk_hits), int(n_tracks),
                                              _ptr(align), C.byref(grid), _ptr(field),
                                              _ptr(chi2_total), _ptr(grad_align), _ptr(grad_field),
                                              _stream(stream))
    _check(ctx, rc, "tpc_fit_adjoint_field")


# Limits of tpc_find_tracks_noalloc (include/tpc_track.h).
NOALLOC_MAX_CLUSTERS = 65536
NOALLOC_MAX_EVENTS = 4


def tpc_find_tracks_noalloc(y, z, row, evt_sector_off, n_events, track_of_cluster, trk_off,
                            trk_hits, n_tracks_dev, status_dev, params: Params | None = None,
                            stream=None):
    """Load + find in one call whose scratch is the library's own fixed
    device array: the call allocates nothing.  The device status word is
    copied to status_dev[0]."""
    _need(y, torch.float32, "y")
    _need(z, torch.float32, "z")
    _need(row, torch.uint16, "row")
    _need(evt_sector_off, torch.int64, "evt_sector_off")
    for t, nm in ((track_of_cluster, "track_of_cluster"), (trk_off, "trk_off"),
                  (trk_hits, "trk_hits"), (n_tracks_dev, "n_tracks_dev"), (status_dev, "status_dev")):
        _need(t, torch.int32, nm)
    what = "tpc_find_tracks_noalloc"
    check_load_inputs(y, z, row, None, evt_sector_off, n_events, what)
    check_find_outputs(y.numel(), track_of_cluster, trk_off, trk_hits, n_tracks_dev, what)
    _need_len(status_dev, 1, "status_dev", what)
    rc = load_library().tpc_find_tracks_noalloc(
        C.byref(params) if params is not None else None, _ptr(y), _ptr(z), _ptr(row), y.numel(),
        _ptr(evt_sector_off), int(n_events), _ptr(track_of_cluster), _ptr(trk_off), _ptr(trk_hits),
        _ptr(n_tracks_dev), _ptr(status_dev), trk_off.numel() - 1, _stream(stream))
    if rc != TPC_OK:
        raise TPCError(f"{what}: {STATUS_NAMES.get(rc, rc)}")


def tpc_set_tune(ctx, tune: Tune | None):
    _check(ctx, load_library().tpc_set_tune(ctx, C.byref(tune) if tune is not None else None),
           "tpc_set_tune")


def tpc_autotune(ctx, track_of_cluster, trk_off, trk_hits, n_tracks_dev, stream=None) -> Tune:
    for t, n in ((track_of_cluster, "track_of_cluster"), (trk_off, "trk_off"),
                 (trk_hits, "trk_hits"), (n_tracks_dev, "n_tracks_dev")):
        _need(t, torch.int32, n)
    check_find_outputs(_loaded_n.get(ctx.value, 0), track_of_cluster, trk_off, trk_hits, n_tracks_dev,
                       what="tpc_autotune")
    best = Tune()
    rc = load_library().tpc_autotune(ctx, _ptr(track_of_cluster), _ptr(trk_off), _ptr(trk_hits),
                                     _ptr(n_tracks_dev), trk_off.numel() - 1, C.byref(best),
                                     _stream(stream))
    _check(ctx, rc, "tpc_autotune")
    return best


def _batch_args(ctx, y, z, row, charge, evt_sector_off, n_events, find_out, fit_out, what):
    """Checks and marshals the arguments of tpc_track_batch /
    tpc_graph_capture; returns the BatchOutputs structure."""
    _need(y, torch.float32, "y")
    _need(z, torch.float32, "z")
    _need(row, torch.uint16, "row")
    if charge is not None:
        _need(charge, torch.uint16, "charge")
    _need(evt_sector_off, torch.int64, "evt_sector_off")
    check_load_inputs(y, z, row, charge, evt_sector_off, n_events, what)
    toc, trk_off, trk_hits, ntd = find_out
    for t, nm in ((toc, "track_of_cluster"), (trk_off, "trk_off"), (trk_hits, "trk_hits"),
                  (ntd, "n_tracks_dev")):
        _need(t, torch.int32, nm)
    check_find_outputs(y.numel(), toc, trk_off, trk_hits, ntd, what)
    cap = trk_off.numel() - 1
    o = BatchOutputs(_ptr(toc), _ptr(trk_off), _ptr(trk_hits), _ptr(ntd), cap, None, None, None, None)
    if fit_out is not None:
        params, cov, chi2, ndf = fit_out
        for t, nm in ((params, "params"), (cov, "cov"), (chi2, "chi2")):
            _need(t, torch.float32, nm)
        _need(ndf, torch.int32, "ndf")
        check_fit_buffers(cap, trk_off, params, cov, chi2, ndf, what)
        o.params, o.cov, o.chi2, o.ndf = _ptr(params), _ptr(cov), _ptr(chi2), _ptr(ndf)
    return o


def tpc_track_batch(ctx, y, z, row, charge, evt_sector_off, n_events, find_out, fit_out=None,
                    stream=None):
    o = _batch_args(ctx, y, z, row, charge, evt_sector_off, n_events, find_out, fit_out,
                    "tpc_track_batch")
    rc = load_library().tpc_track_batch(ctx, _ptr(y), _ptr(z), _ptr(row), _ptr(charge), y.numel(),
                                        _ptr(evt_sector_off), int(n_events), C.byref(o), _stream(stream))
    _check(ctx, rc, "tpc_track_batch")
    _loaded_n[ctx.value] = y.numel()


def tpc_graph_capture(ctx, y, z, row, charge, evt_sector_off, n_events, find_out, fit_out=None):
    o = _batch_args(ctx, y, z, row, charge, evt_sector_off, n_events, find_out, fit_out,
                    "tpc_graph_capture")
    rc = load_library().tpc_graph_capture(ctx, _ptr(y), _ptr(z), _ptr(row), _ptr(charge), y.numel(),
                                          _ptr(evt_sector_off), int(n_events), C.byref(o))
    _check(ctx, rc, "tpc_graph_capture")
    _loaded_n[ctx.value] = y.numel()


def tpc_graph_launch(ctx, stream=None):
    _check(ctx, load_library().tpc_graph_launch(ctx, _stream(stream)), "tpc_graph_launch")


# --- NEXT-2: clusterization ------------------------------------------------------

N_PAD = 160


def tpc_cluster_workspace_bytes(n_events: int, n_time: int) -> int:
    return int(load_library().tpc_cluster_workspace_bytes(int(n_events), int(n_time)))


def tpc_find_clusters(digits, n_events, workspace, outputs, q_peak=8, stream=None):
    """outputs = (y f32[cap], z f32[cap], row u16[cap], charge u16[cap],
    evt_sector_off i64[36 n_events + 1], n_clusters_dev i32[1],
    status_dev i32[2])."""
    what = "tpc_find_clusters"
    _need(digits, torch.uint16, "digits")
    _need(workspace, torch.uint8, "workspace")
    y, z, row, charge, off, ncl, status = outputs
    _need(y, torch.float32, "y")
    _need(z, torch.float32, "z")
    _need(row, torch.uint16, "row")
    _need(charge, torch.uint16, "charge")
    _need(off, torch.int64, "evt_sector_off")
    _need(ncl, torch.int32, "n_clusters_dev")
    _need(status, torch.int32, "status_dev")
    if digits.dim() != 3 or digits.shape[0] != int(n_events) * 36 * 152 or digits.shape[2] != N_PAD:
        raise ValueError(f"{what}: digits must be [n_events*36*152, n_time, {N_PAD}]")
    cap = y.numel()
    for t, nm in ((z, "z"), (row, "row"), (charge, "charge")):
        _need_len(t, cap, nm, what)
    _need_len(off, 36 * int(n_events) + 1, "evt_sector_off", what)
    _need_len(ncl, 1, "n_clusters_dev", what)
    _need_len(status, 2, "status_dev", what)
    need = tpc_cluster_workspace_bytes(n_events, digits.shape[1])
    if need == 0 or workspace.numel() < need:
        raise ValueError(f"{what}: workspace holds {workspace.numel()} bytes, the call needs {need}")
    rc = load_library().tpc_find_clusters(_ptr(digits), int(n_events), int(digits.shape[1]), int(q_peak),
                                          _ptr(workspace), workspace.numel(), _ptr(y), _ptr(z), _ptr(row),
                                          _ptr(charge), _ptr(off), cap, _ptr(ncl), _ptr(status),
                                          _stream(stream))
    if rc != TPC_OK:
        raise TPCError(f"{what}: {STATUS_NAMES.get(rc, rc)}")


class Clusterizer:
    """Workspace and outputs for the clusterization of batches of up to
    n_events events of n_time time bins."""

    def __init__(self, n_events: int, n_time: int, cap: int, device="cuda"):
        self.device = torch.device(device)
        self.n_events, self.n_time, self.cap = int(n_events), int(n_time), int(cap)
        nb = tpc_cluster_workspace_bytes(self.n_events, self.n_time)
        if nb == 0:
            raise ValueError("unsupported clusterization shape")
        self.workspace = torch.empty(nb, dtype=torch.uint8, device=self.device)
        d = self.device
        self.out = (torch.empty(self.cap, dtype=torch.float32, device=d),
                    torch.empty(self.cap, dtype=torch.float32, device=d),
                    torch.empty(self.cap, dtype=torch.int16, device=d).view(torch.uint16),
                    torch.empty(self.cap, dtype=torch.int16, device=d).view(torch.uint16),
                    torch.empty(36 * self.n_events + 1, dtype=torch.int64, device=d),
                    torch.empty(1, dtype=torch.int32, device=d),
                    torch.empty(2, dtype=torch.int32, device=d))

    def run(self, digits, q_peak=8, stream=None):
        tpc_find_clusters(digits, self.n_events, self.workspace, self.out, q_peak, stream)
        return self.out


def tpc_get_stats(ctx, stream=None) -> Stats:
    st = Stats()
    load_library().tpc_get_stats(ctx, C.byref(st), _stream(stream))
    return st


def tpc_stage_timing(ctx, enable: bool):
    _check(ctx, load_library().tpc_stage_timing(ctx, 1 if enable else 0), "tpc_stage_timing")


def tpc_stage_times(ctx) -> dict:
    ms = (C.c_float * len(STAGE_NAMES))()
    _check(ctx, load_library().tpc_stage_times(ctx, ms), "tpc_stage_times")
    return dict(zip(STAGE_NAMES, [float(v) for v in ms]))


def tpc_reset_status(ctx, stream=None):
    _check(ctx, load_library().tpc_reset_status(ctx, _stream(stream)), "tpc_reset_status")


# --- convenience wrapper -------------------------------------------------------

class Tracker:
    """Owns a context and its workspace tensor for batches of up to
    max_clusters clusters in max_events events."""

    def __init__(self, max_clusters: int, max_events: int = 1, params: Params | None = None,
                 device: str | torch.device = "cuda"):
        if not torch.cuda.is_available():
            raise RuntimeError("libtpctrack needs a CUDA device")
        self.device = torch.device(device)
        self.params = params or default_params()
        self.ctx = tpc_create(self.params)
        self.max_clusters = int(max_clusters)
        self.max_events = int(max_events)
        self.n_events_loaded = 1
        nbytes = tpc_workspace_bytes(self.ctx, self.max_clusters, self.max_events)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        tpc_set_workspace(self.ctx, self.workspace, self.max_clusters, self.max_events)
        self.n = 0

    def close(self):
        if self.ctx is not None:
            tpc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, y, z, row, evt_sector_off, n_events, charge=None, stream=None, validate=False):
        """Registers a batch.  The library checks it on the device (rows,
        finite coordinates, offsets) into the status word; with validate the
        status is read here (a synchronisation) and a batch that fails is
        refused before any find kernel could run on it."""
        self._inputs = (y, z, row, charge, evt_sector_off)  # keep alive
        tpc_load_clusters(self.ctx, y, z, row, charge, evt_sector_off, n_events, stream)
        self.n_events_loaded = int(n_events)
        self.n = y.numel()
        if validate:
            self.check(stream)

    def alloc_find_outputs(self, track_cap=None):
        """Outputs of find for the loaded batch; before a load, for the
        largest batch the context takes (max_clusters)."""
        m = max(self.n if self.n > 0 else self.max_clusters, 1)
        # the context takes at most max_clusters tracks (a track has >= 1
        # cluster); small batches get that bound instead of n/10 + 16
        cap = int(track_cap if track_cap is not None else min(m // 10 + 16, max(self.max_clusters, 1)))
        dev = self.device
        return (torch.empty(m, dtype=torch.int32, device=dev),
                torch.empty(cap + 1, dtype=torch.int32, device=dev),
                torch.empty(m, dtype=torch.int32, device=dev),
                torch.empty(1, dtype=torch.int32, device=dev))

    def find(self, out=None, track_cap=None, stream=None):
        out = out or self.alloc_find_outputs(track_cap)
        tpc_find_tracks(self.ctx, *out, stream=stream)
        return out

    def fit(self, trk_off, trk_hits, n_tracks, n_tracks_dev=None, out=None, stream=None,
            precision="ff"):
        """precision "ff": float-float covariance (tpc_fit_tracks); "fp32":
        FP32 covariance with FP64 redos (tpc_fit_tracks_fp32)."""
        if precision not in ("ff", "fp32"):
            raise ValueError(f"precision must be 'ff' or 'fp32', not {precision!r}")
        dev = self.device
        T = max(int(n_tracks), 1)
        out = out or (torch.empty(T, 5, dtype=torch.float32, device=dev),
                      torch.empty(T, 15, dtype=torch.float32, device=dev),
                      torch.empty(T, dtype=torch.float32, device=dev),
                      torch.empty(T, dtype=torch.int32, device=dev))
        fn = tpc_fit_tracks if precision == "ff" else tpc_fit_tracks_fp32
        fn(self.ctx, trk_off, trk_hits, n_tracks, n_tracks_dev, *out, stream=stream)
        return out

    def fit_ex(self, trk_off, trk_hits, n_tracks, options=None, n_tracks_dev=None, smooth=False,
               stream=None):
        """The Kalman-filter variants (material, outward refit, smoother):
        (params, cov, chi2, ndf, smoothed or None); smoothed holds 20
        doubles (state, covariance) per entry of trk_hits."""
        dev = self.device
        T = max(int(n_tracks), 1)
        out = (torch.empty(T, 5, dtype=torch.float32, device=dev),
               torch.empty(T, 15, dtype=torch.float32, device=dev),
               torch.empty(T, dtype=torch.float32, device=dev),
               torch.empty(T, dtype=torch.int32, device=dev))
        sm = torch.zeros(max(trk_hits.numel(), 1), 20, dtype=torch.float64, device=dev) if smooth else None
        tpc_fit_tracks_ex(self.ctx, trk_off, trk_hits, n_tracks, n_tracks_dev, options, *out, sm, stream)
        return (*out, sm)

    def match_sides(self, trk_off, trk_hits, n_tracks, n_tracks_dev=None, options=None, cand_cap=None,
                    stream=None):
        """NEXT-4: pairs the A- and C-side segments of membrane-crossing
        tracks among the found tracks and fits each pair with t0.  Returns a
        dict of per-track device tensors (partner, t0, params6, cov6, chi2,
        ndf, dchi2) and n_pairs (device int32[1])."""
        dev = self.device
        T = int(n_tracks)
        cap = max(T, 1024) if cand_cap is None else int(cand_cap)
        out = tuple(torch.empty(max(T, 1), *(() if k == 1 else (k,)), dtype=dt, device=dev)
                    for _, dt, k in SIDES_OUT)
        n_pairs = torch.zeros(1, dtype=torch.int32, device=dev)
        E = self.n_events_loaded
        need = tpc_sides_workspace_bytes(T, E, cap)
        ws = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
        tpc_match_sides(self.ctx, trk_off, trk_hits, T, n_tracks_dev, options, ws, cap, out, n_pairs, E, stream)
        res = {name: t for (name, _, _), t in zip(SIDES_OUT, out)}
        res["n_pairs"] = n_pairs
        return res

    def adjoint(self, trk_off, trk_hits, n_tracks, align, want_grad=True, stream=None):
        chi2 = torch.zeros(1, dtype=torch.float64, device=self.device)
        grad = torch.zeros(216, dtype=torch.float64, device=self.device) if want_grad else None
        tpc_fit_adjoint(self.ctx, trk_off, trk_hits, n_tracks, align, chi2, grad, stream=stream)
        return chi2, grad

    def adjoint_field(self, trk_off, trk_hits, n_tracks, grid: FieldGrid, field, align=None,
                      want_grad=True, stream=None):
        """Summed chi2 with the displacement field[n_voxels, 3] added to the
        aligned clusters, and its gradients with respect to the alignment
        and the field (None when want_grad is false)."""
        dev = self.device
        if align is None:
            align = torch.zeros(216, dtype=torch.float64, device=dev)
        chi2 = torch.zeros(1, dtype=torch.float64, device=dev)
        nv = tpc_field_voxels(grid)
        g_al = torch.zeros(216, dtype=torch.float64, device=dev) if want_grad else None
        g_f = torch.zeros(max(nv, 0), 3, dtype=torch.float64, device=dev) if want_grad else None
        tpc_fit_adjoint_field(self.ctx, trk_off, trk_hits, n_tracks, align, grid, field, chi2,
                              g_al, g_f, stream=stream)
        return chi2, g_al, g_f

    def stats(self, stream=None) -> Stats:
        return tpc_get_stats(self.ctx, stream)

    def check(self, stream=None):
        st = self.stats(stream)
        if st.status != TPC_OK:
            raise TPCError(f"device status {STATUS_NAMES.get(st.status, st.status)} "
                           f"(detail {st.status_detail})")
        return st

    def reset_status(self, stream=None):
        tpc_reset_status(self.ctx, stream)

    def alloc_fit_outputs(self, track_cap):
        dev = self.device
        T = max(int(track_cap), 1)
        return (torch.empty(T, 5, dtype=torch.float32, device=dev),
                torch.empty(T, 15, dtype=torch.float32, device=dev),
                torch.empty(T, dtype=torch.float32, device=dev),
                torch.empty(T, dtype=torch.int32, device=dev))

    def track_batch(self, y, z, row, evt_sector_off, n_events, find_out, fit_out=None, charge=None,
                    stream=None):
        """S7: load + find (+ fit when fit_out is given) of a whole batch in
        one call."""
        self._inputs = (y, z, row, charge, evt_sector_off)
        tpc_track_batch(self.ctx, y, z, row, charge, evt_sector_off, n_events, find_out, fit_out, stream)
        self.n = y.numel()
        self.n_events_loaded = int(n_events)

    def capture(self, y, z, row, evt_sector_off, n_events, find_out, fit_out=None, charge=None):
        """Records the batch call into the context's CUDA graph; replay()
        runs it.  The buffers stay bound to the graph: keep them alive."""
        self._graph_buffers = (y, z, row, charge, evt_sector_off, find_out, fit_out)
        tpc_graph_capture(self.ctx, y, z, row, charge, evt_sector_off, n_events, find_out, fit_out)
        self.n = y.numel()
        self.n_events_loaded = int(n_events)

    def replay(self, stream=None):
        tpc_graph_launch(self.ctx, stream)

    def autotune(self, out=None, stream=None) -> Tune:
        out = out or self.alloc_find_outputs()
        return tpc_autotune(self.ctx, *out, stream=stream)

    def set_tune(self, tune: Tune | None):
        tpc_set_tune(self.ctx, tune)

    def stage_timing(self, enable: bool = True):
        tpc_stage_timing(self.ctx, enable)

    def stage_times(self) -> dict:
        return tpc_stage_times(self.ctx)
