"""FP64 CPU oracle of the TPC tracking path -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and
shares no code with it.  ``build()`` compiles ``tpc_oracle.cpp`` with plain
g++ (OpenMP, no floating-point contraction, so FP32 neighbour decisions round
once per operation exactly like the kernel's).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

N_SECTORS = 36


class Params(C.Structure):
    _fields_ = [
        ("win_y", C.c_float), ("win_z", C.c_float), ("chi2_link", C.c_float),
        ("sigma_y2", C.c_float), ("sigma_z2", C.c_float),
        ("max_gap", C.c_int32), ("n_seg", C.c_int32), ("n_min", C.c_int32),
        ("merge_max_row_gap", C.c_int32), ("merge_max_overlap", C.c_int32),
        ("merge_z_slope", C.c_float), ("merge_z_margin", C.c_float),
        ("chi2_merge", C.c_double), ("chi2_ext", C.c_double),
        ("ext_max_miss", C.c_int32), ("bz", C.c_double),
        ("prior", C.c_double * 5), ("seed_snp_max", C.c_double),
        ("seed_qpt_max", C.c_double),
        ("snp_max", C.c_double),
        ("s2_fp64", C.c_int32),
        ("mat_x_x0", C.c_double), ("mat_eloss", C.c_double), ("mass", C.c_double),
    ]


class Diag(C.Structure):
    _fields_ = [
        ("choice_dn", C.c_void_p), ("choice_up", C.c_void_p),
        ("d2", C.c_void_p), ("d2_next", C.c_void_p),
        ("link_dn", C.c_void_p), ("link_up", C.c_void_p),
        ("seg_of", C.c_void_p), ("merge_margin", C.c_void_p),
        ("ext_margin", C.c_void_p),
    ]


class SidesParams(C.Structure):
    """Parameters of the A/C-side association with t0 (orc_sides_params)."""
    _fields_ = [("n_min", C.c_int32), ("gap_max", C.c_int32), ("chi2_junction", C.c_double),
                ("z_membrane", C.c_double), ("z_pre", C.c_double), ("chi2_joint", C.c_double),
                ("t0_prior", C.c_double),
                ("v_drift", C.c_double)]


class FieldGrid(C.Structure):
    """Voxel grid of a displacement field (orc_field_grid)."""
    _fields_ = [("n_band", C.c_int32), ("n_y", C.c_int32), ("n_z", C.c_int32),
                ("u_lo", C.c_float), ("u_inv", C.c_float), ("z_inv", C.c_float)]


def field_grid(n_band, n_y, n_z, u_lo, u_inv, z_inv) -> FieldGrid:
    return FieldGrid(int(n_band), int(n_y), int(n_z), float(u_lo), float(u_inv), float(z_inv))


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "tpc_oracle.cpp")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "tpc_oracle.h"))):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC",
           "-shared", "-o", tmp, src]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(_SO)
        _lib.orc_find_tracks.restype = C.c_int64
        _lib.orc_bruteforce_chains.restype = C.c_int64
        _lib.orc_voxel_of.restype = C.c_int64
        _lib.orc_tracklet.restype = C.c_int64
        _lib.orc_find_clusters.restype = C.c_int64
        _lib.orc_match_sides.restype = C.c_int64
        _lib.orc_fit_t0.argtypes = [C.c_void_p] * 5 + [C.c_int32, C.c_int32, C.c_double] + [C.c_void_p] * 5
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def default_params(**kw) -> Params:
    p = Params()
    lib().orc_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "prior":
            for i in range(5):
                p.prior[i] = v[i]
        else:
            setattr(p, k, v)
    return p


def set_threads(n: int):
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def find_tracks(y, z, row, evt_sector_off, n_events, params=None, diag=False):
    """Returns (track_of_cluster, trk_off, trk_hits[, diag dict])."""
    y, z, row = _c(y, np.float32), _c(z, np.float32), _c(row, np.uint16)
    off = _c(evt_sector_off, np.int64)
    n = y.shape[0]
    prm = params or default_params()
    toc = np.empty(n, np.int32)
    trk_off = np.empty(n + 1, np.int32)
    hits = np.empty(max(n, 1), np.int32)
    d = None
    dg = None
    if diag:
        d = dict(choice_dn=np.empty(n, np.int32), choice_up=np.empty(n, np.int32),
                 d2=np.empty(n, np.float32), d2_next=np.empty(n, np.float32),
                 link_dn=np.empty(n, np.int32), link_up=np.empty(n, np.int32),
                 seg_of=np.empty(n, np.int32), merge_margin=np.empty(n, np.float64),
                 ext_margin=np.empty(n, np.float64))
        dg = Diag(**{k: v.ctypes.data for k, v in d.items()})
    T = lib().orc_find_tracks(_p(y), _p(z), _p(row), C.c_int64(n), _p(off),
                              C.c_int32(n_events), C.byref(prm), _p(toc), _p(trk_off),
                              _p(hits), C.byref(dg) if dg is not None else None)
    if T < 0:
        raise ValueError("oracle rejected the input")
    trk_off = trk_off[:T + 1].copy()
    hits = hits[:trk_off[-1]].copy()
    return (toc, trk_off, hits, d) if diag else (toc, trk_off, hits)


def fit_tracks(y, z, row, sector_of, trk_off, trk_hits, align=None, params=None,
               reverse=False):
    """FP64 fit; returns (params[T,5], cov[T,15], chi2[T], ndf[T])."""
    y, z, row = _c(y, np.float32), _c(z, np.float32), _c(row, np.uint16)
    sec = _c(sector_of, np.int32)
    off, hits = _c(trk_off, np.int32), _c(trk_hits, np.int32)
    T = off.shape[0] - 1
    prm = params or default_params()
    par = np.empty((T, 5)); cov = np.empty((T, 15)); chi2 = np.empty(T)
    ndf = np.empty(T, np.int32)
    al = _c(align, np.float64) if align is not None else None
    lib().orc_fit_tracks_dir(_p(y), _p(z), _p(row), _p(sec), _p(off), _p(hits),
                             C.c_int32(T), _p(al), C.byref(prm), C.c_int(1 if reverse else 0),
                             _p(par), _p(cov), _p(chi2), _p(ndf))
    return par, cov, chi2, ndf


def fit_adjoint(y, z, row, sector_of, trk_off, trk_hits, align, params=None,
                want_grad=True):
    """Total chi2 and d chi2 / d align[216] (exact, dual numbers)."""
    y, z, row = _c(y, np.float32), _c(z, np.float32), _c(row, np.uint16)
    sec = _c(sector_of, np.int32)
    off, hits = _c(trk_off, np.int32), _c(trk_hits, np.int32)
    T = off.shape[0] - 1
    prm = params or default_params()
    al = _c(align, np.float64)
    tot = C.c_double(0.0)
    g = np.zeros(216) if want_grad else None
    lib().orc_fit_adjoint(_p(y), _p(z), _p(row), _p(sec), _p(off), _p(hits),
                          C.c_int32(T), _p(al), C.byref(prm), C.byref(tot), _p(g))
    return (tot.value, g) if want_grad else tot.value


def voxel_of(y, z, row, sector_of, grid: FieldGrid):
    """Voxel of each cluster; returns (vox[n], number of voxels)."""
    y, z, row = _c(y, np.float32), _c(z, np.float32), _c(row, np.uint16)
    sec = _c(sector_of, np.int32)
    vox = np.empty(y.shape[0], np.int32)
    nv = lib().orc_voxel_of(_p(y), _p(z), _p(row), _p(sec), C.c_int64(y.shape[0]),
                            C.byref(grid), _p(vox))
    if nv < 0:
        raise ValueError("invalid field grid")
    return vox, int(nv)


def field_adjoint(y, z, row, sector_of, trk_off, trk_hits, grid: FieldGrid, field,
                  align=None, params=None, want_grad=True):
    """Total chi2 with the displacement field[n_vox, 3] added to the aligned
    clusters, and d chi2 / d field (exact, dual numbers)."""
    y, z, row = _c(y, np.float32), _c(z, np.float32), _c(row, np.uint16)
    sec = _c(sector_of, np.int32)
    off, hits = _c(trk_off, np.int32), _c(trk_hits, np.int32)
    T = off.shape[0] - 1
    prm = params or default_params()
    fld = _c(field, np.float64)
    nv = 36 * grid.n_band * grid.n_y * grid.n_z
    if fld.size != 3 * nv:
        raise ValueError(f"field holds {fld.size} values, the grid has {nv} voxels x 3")
    al = _c(align, np.float64) if align is not None else None
    tot = C.c_double(0.0)
    g = np.zeros((nv, 3)) if want_grad else None
    rc = lib().orc_field_adjoint(_p(y), _p(z), _p(row), _p(sec), _p(off), _p(hits),
                                 C.c_int32(T), _p(al), C.byref(grid), _p(fld), C.byref(prm),
                                 C.byref(tot), _p(g))
    if rc != 0:
        raise ValueError("invalid field grid")
    return (tot.value, g) if want_grad else tot.value


def field_gn_blocks(y, z, row, sector_of, trk_off, trk_hits, grid: FieldGrid, field,
                    align=None, params=None):
    """Per-voxel 3x3 diagonal blocks [n_vox, 3, 3] of the field's
    Gauss-Newton matrix (dual numbers through the fit)."""
    y, z, row = _c(y, np.float32), _c(z, np.float32), _c(row, np.uint16)
    sec = _c(sector_of, np.int32)
    off, hits = _c(trk_off, np.int32), _c(trk_hits, np.int32)
    T = off.shape[0] - 1
    prm = params or default_params()
    fld = _c(field, np.float64)
    nv = 36 * grid.n_band * grid.n_y * grid.n_z
    if fld.size != 3 * nv:
        raise ValueError(f"field holds {fld.size} values, the grid has {nv} voxels x 3")
    al = _c(align, np.float64) if align is not None else None
    out = np.zeros((nv, 3, 3))
    rc = lib().orc_field_gn_blocks(_p(y), _p(z), _p(row), _p(sec), _p(off), _p(hits), C.c_int32(T),
                                   _p(al), C.byref(grid), _p(fld), C.byref(prm), _p(out))
    if rc != 0:
        raise ValueError("invalid field grid")
    return out


def gauss_newton(y, z, row, sector_of, trk_off, trk_hits, align, params=None):
    y, z, row = _c(y, np.float32), _c(z, np.float32), _c(row, np.uint16)
    sec = _c(sector_of, np.int32)
    off, hits = _c(trk_off, np.int32), _c(trk_hits, np.int32)
    T = off.shape[0] - 1
    prm = params or default_params()
    al = _c(align, np.float64)
    gn = np.zeros((216, 216))
    lib().orc_gauss_newton(_p(y), _p(z), _p(row), _p(sec), _p(off), _p(hits),
                           C.c_int32(T), _p(al), C.byref(prm), _p(gn))
    return gn


def propagate(x1, s1, p, x2, s2, params=None):
    """One propagation; returns (p_out, jac[5,5], dx1[5], dx2[5]) or None."""
    prm = params or default_params()
    p = _c(p, np.float64)
    po = np.empty(5); J = np.empty(25); d1 = np.empty(5); d2 = np.empty(5)
    rc = lib().orc_propagate(C.c_double(x1), C.c_int(s1), _p(p), C.c_double(x2),
                             C.c_int(s2), C.byref(prm), _p(po), _p(J), _p(d1), _p(d2))
    if rc != 0:
        return None
    return po, J.reshape(5, 5), d1, d2


def bruteforce_chains(y, z, row, sector, params=None, chi2ndf_max=5.0,
                      cap_chains=100000, cap_hits=5000000):
    y, z, row = _c(y, np.float32), _c(z, np.float32), _c(row, np.uint16)
    prm = params or default_params()
    off = np.empty(cap_chains + 1, np.int32)
    hits = np.empty(cap_hits, np.int32)
    k = lib().orc_bruteforce_chains(_p(y), _p(z), _p(row), C.c_int64(y.shape[0]),
                                    C.c_int32(sector), C.byref(prm), C.c_double(chi2ndf_max),
                                    C.c_int64(cap_chains), C.c_int64(cap_hits), _p(off), _p(hits))
    if k < 0:
        raise RuntimeError("brute-force capacity too small")
    return [hits[off[i]:off[i + 1]].copy() for i in range(k)]


def seed(y, z, row, sector_of, hits, first_is_outer=True, params=None, f64=False):
    """The fit seed: (x0, frame, p[5]) of a hit list in fit order.  With f64
    the points are passed in FP64 (pins with exact helix points)."""
    dt = np.float64 if f64 else np.float32
    y, z, row = _c(y, dt), _c(z, dt), _c(row, np.uint16)
    sec = _c(sector_of, np.int32)
    hits = _c(hits, np.int32)
    prm = params or default_params()
    x0 = C.c_double(0.0); fr = C.c_int32(0); p = np.empty(5)
    fn = lib().orc_seed_f64 if f64 else lib().orc_seed
    rc = fn(_p(y), _p(z), _p(row), _p(sec), _p(hits), C.c_int32(hits.shape[0]),
                        C.c_int(1 if first_is_outer else 0), C.byref(prm), C.byref(x0),
                        C.byref(fr), _p(p))
    if rc != 0:
        raise ValueError("seed needs >= 3 clusters")
    return x0.value, fr.value, p


def tracklet(y, z, row, beg, end, sector, seg_hits, params=None):
    """S3b of one segment (hits outermost first) inside the group [beg, end)
    of one sector: the tracklet the find builds from it, outermost first."""
    y, z, row = _c(y, np.float32), _c(z, np.float32), _c(row, np.uint16)
    seg = _c(seg_hits, np.int32)
    prm = params or default_params()
    cap = 4 * 152
    out = np.empty(cap, np.int32)
    k = lib().orc_tracklet(_p(y), _p(z), _p(row), C.c_int64(beg), C.c_int64(end), C.c_int32(sector),
                           _p(seg), C.c_int32(seg.shape[0]), C.byref(prm), _p(out), C.c_int32(cap))
    if k < 0:
        raise ValueError("orc_tracklet refused its arguments")
    return out[:k].copy()


def merge_chi2(y, z, row, hits_a, sec_a, hits_b, sec_b, params=None):
    """S4 of an inner segment A and an outer segment B (hits outermost
    first): (chi2_5, accepted by the merge's gates and cut), or None when a
    fit or the move fails."""
    y, z, row = _c(y, np.float32), _c(z, np.float32), _c(row, np.uint16)
    a, b = _c(hits_a, np.int32), _c(hits_b, np.int32)
    prm = params or default_params()
    c2 = C.c_double(0.0)
    ok = C.c_int32(0)
    rc = lib().orc_merge_chi2(_p(y), _p(z), _p(row), _p(a), C.c_int32(a.shape[0]), C.c_int32(sec_a),
                              _p(b), C.c_int32(b.shape[0]), C.c_int32(sec_b), C.byref(prm),
                              C.byref(c2), C.byref(ok))
    if rc == 1:
        raise ValueError("orc_merge_chi2 refused its arguments")
    return None if rc != 0 else (c2.value, bool(ok.value))


def kf_ops(y, z, row, sector_of, trk_off, trk_hits, params=None):
    """(operations, Kalman steps) of the FP64 fit of the given tracks; see
    orc_kf_ops (structural zeros and ones of the Jacobians not counted)."""
    y, z, row = _c(y, np.float32), _c(z, np.float32), _c(row, np.uint16)
    sec = _c(sector_of, np.int32)
    off, hits = _c(trk_off, np.int32), _c(trk_hits, np.int32)
    prm = params or default_params()
    ops = C.c_double(0.0)
    steps = C.c_int64(0)
    lib().orc_kf_ops(_p(y), _p(z), _p(row), _p(sec), _p(off), _p(hits), C.c_int32(off.shape[0] - 1),
                     C.byref(prm), C.byref(ops), C.byref(steps))
    return ops.value, steps.value


def smooth_tracks(y, z, row, sector_of, trk_off, trk_hits, params=None):
    """Inward fit plus Rauch-Tung-Striebel smoother: (smoothed[n_hits, 20]
    (state 5 + covariance 15 per hit of the lists, list order), chi2[T],
    ndf[T])."""
    y, z, row = _c(y, np.float32), _c(z, np.float32), _c(row, np.uint16)
    sec = _c(sector_of, np.int32)
    off, hits = _c(trk_off, np.int32), _c(trk_hits, np.int32)
    T = off.shape[0] - 1
    prm = params or default_params()
    out = np.zeros((max(int(off[-1]), 1), 20))
    chi2 = np.empty(T)
    ndf = np.empty(T, np.int32)
    lib().orc_smooth_tracks(_p(y), _p(z), _p(row), _p(sec), _p(off), _p(hits), C.c_int32(T),
                            C.byref(prm), _p(out), _p(chi2), _p(ndf))
    return out[:int(off[-1])], chi2, ndf


def find_clusters(digits, n_events, q_peak=8):
    """Clusters of pad-time digits u16 [n_events*36*152, n_time, 160]:
    (y, z, row, charge, evt_sector_off)."""
    d = _c(digits, np.uint16)
    n_time = d.shape[1]
    cap = max(int(np.count_nonzero(d)), 1)
    y = np.empty(cap, np.float32); z = np.empty(cap, np.float32)
    row = np.empty(cap, np.uint16); ch = np.empty(cap, np.uint16)
    off = np.empty(n_events * N_SECTORS + 1, np.int64)
    k = lib().orc_find_clusters(_p(d), C.c_int32(n_events), C.c_int32(n_time), C.c_int32(q_peak),
                                _p(y), _p(z), _p(row), _p(ch), _p(off), C.c_int64(cap))
    if k < 0:
        raise RuntimeError("cluster capacity too small")
    return y[:k], z[:k], row[:k], ch[:k], off


# --- NEXT-4: t0 as a sixth state parameter ------------------------------------

def default_sides_params(**kw) -> SidesParams:
    p = SidesParams()
    lib().orc_default_sides_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def fit_t0(y, z, row, sector_of, hits, n_outer, t0_seed, params=None, sides=None):
    """Six-parameter fit (y, z, sin phi, tan lambda, q/pT, t0) of hits
    (outermost first; the first n_outer the outer segment).  Returns
    (params6[6], cov6[21], chi2) or None when the fit fails."""
    y, z, row = _c(y, np.float32), _c(z, np.float32), _c(row, np.uint16)
    sec, h = _c(sector_of, np.int32), _c(hits, np.int32)
    prm = params or default_params()
    sp = sides or default_sides_params()
    p6 = np.empty(6)
    c6 = np.empty(21)
    c2 = np.empty(1)
    rc = lib().orc_fit_t0(_p(y), _p(z), _p(row), _p(sec), _p(h), len(h), int(n_outer), float(t0_seed),
                          C.byref(prm), C.byref(sp), _p(p6), _p(c6), _p(c2))
    return None if rc else (p6, c6, float(c2[0]))


def match_sides(y, z, row, evt_sector_off, n_events, trk_off, trk_hits, params=None, sides=None):
    """A/C-side association with t0.  Returns a dict of per-track arrays:
    partner, t0, params6 [T,6], cov6 [T,21], chi2, ndf, dchi2, margin;
    and n_pairs."""
    y, z, row = _c(y, np.float32), _c(z, np.float32), _c(row, np.uint16)
    off = _c(evt_sector_off, np.int64)
    to, th = _c(trk_off, np.int32), _c(trk_hits, np.int32)
    T = to.shape[0] - 1
    prm = params or default_params()
    sp = sides or default_sides_params()
    out = dict(partner=np.empty(T, np.int32), t0=np.empty(T), params6=np.empty((T, 6)),
               cov6=np.empty((T, 21)), chi2=np.empty(T), ndf=np.empty(T, np.int32),
               dchi2=np.empty(T), margin=np.empty(T))
    npairs = lib().orc_match_sides(_p(y), _p(z), _p(row), C.c_int64(y.shape[0]), _p(off),
                                   C.c_int32(n_events), _p(to), _p(th), C.c_int32(T), C.byref(prm),
                                   C.byref(sp), *[_p(out[k]) for k in ("partner", "t0", "params6", "cov6",
                                                                        "chi2", "ndf", "dchi2", "margin")])
    if npairs < 0:
        raise ValueError("oracle rejected the input")
    out["n_pairs"] = int(npairs)
    return out
