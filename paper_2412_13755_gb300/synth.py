"""Seeded synthetic TPC events: primary helices from the origin in a uniform Bz.

This module is simulation only.  It draws charged tracks, intersects each
helix with the pad-row planes of the 36 sectors in the *global* frame
(circle / straight-line intersection of the transverse projection), smears
the crossings, adds uniformly distributed noise clusters and lays the result
out as the (event, sector)-grouped structure-of-arrays that the tracking
library consumes.  It contains none of the reconstruction arithmetic (no
neighbour rule, no chaining, no Kalman transport or update); the oracle and
the CUDA path both read its output as plain data.

Workload shapes follow the five benchmark configurations of the build
(one sector; one central Pb-Pb-like event; a 50 kHz pile-up time frame;
512 uneven events; the alignment sample).  The paper measures on ALICE Run-3
Pb-Pb / pp time frames (Sec. 4, Sec. 4.3), which are not available here; these
seeded events stand in for them.

Geometry (the paper gives none; this is the build's stated reading):
  * sector s in [0,36): phi-index i = s mod 18, side A (z>0) for s<18, C below;
    sector centre angle alpha_i = (i + 1/2) * 20 deg;
  * local frame x = X cos a + Y sin a, y = -X sin a + Y cos a, z = Z;
  * pad row r in [0,152) is the plane x = 85 + r * 162/151 cm, accepted
    |y| <= x tan(10 deg), |z| < 250 cm;
  * curvature k = K * Bz * q/pT with K = 2.99792458e-3 (cm T GeV/c)^-1 and
    the direction angle obeying dphi/ds = -k (positive charges bend clockwise
    in +Bz).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

N_SECTORS = 36
N_PHI = 18
N_ROWS = 152
X_FIRST = 85.0
X_LAST = 247.0
ROW_PITCH = (X_LAST - X_FIRST) / (N_ROWS - 1)
SECTOR_WIDTH = math.radians(20.0)
TAN_HALF_SECTOR = math.tan(math.radians(10.0))
BZ = 0.5
KAPPA = 2.99792458e-3
Z_MAX = 250.0
SIGMA_Y = 0.1
SIGMA_Z = 0.15
ROW_DROP = 0.05
V_DRIFT = 2.58          # cm / us
FRAME_US = 2000.0       # 100 collisions at 50 kHz
SEED_BASE = 241213755

ROW_X = X_FIRST + np.arange(N_ROWS, dtype=np.float64) * ROW_PITCH


def sector_alpha(sector):
    """Centre angle (rad) of a sector (array or scalar)."""
    return ((np.asarray(sector) % N_PHI) + 0.5) * SECTOR_WIDTH


def rotation_matrix(a, b, g):
    """R = Rz(g) Ry(b) Rx(a) about the sector-local axes."""
    ca, sa, cb, sb, cg, sg = (math.cos(a), math.sin(a), math.cos(b),
                              math.sin(b), math.cos(g), math.sin(g))
    rx = np.array([[1, 0, 0], [0, ca, -sa], [0, sa, ca]])
    ry = np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
    rz = np.array([[cg, -sg, 0], [sg, cg, 0], [0, 0, 1]])
    return rz @ ry @ rx


@dataclasses.dataclass
class Events:
    """A batch of events, clusters grouped by (event, sector).

    Cluster arrays are in *input order*: grouped by event*36+sector
    (offsets in ``evt_sector_off``), shuffled inside each group.
    """
    y: np.ndarray               # f32 [n] local y (cm)
    z: np.ndarray               # f32 [n] local z (cm), drift-shifted in frames
    row: np.ndarray             # u16 [n]
    charge: np.ndarray          # u16 [n]
    evt_sector_off: np.ndarray  # i64 [E*36+1]
    n_events: int
    mc_track: np.ndarray        # i32 [n] global track id, -1 = noise
    trk_q: np.ndarray           # f64 [T] charge sign
    trk_pt: np.ndarray          # f64 [T]
    trk_tgl: np.ndarray         # f64 [T]
    trk_phi0: np.ndarray        # f64 [T]
    trk_event: np.ndarray       # i32 [T]
    trk_t0: np.ndarray          # f64 [T] drift-time offset (us), 0 outside frames
    # per-cluster truth at the crossing (noise: NaN); only when truth=True
    y_true: np.ndarray | None = None
    z_true: np.ndarray | None = None
    snp_true: np.ndarray | None = None
    arc_true: np.ndarray | None = None
    align: np.ndarray | None = None  # f64 [216] true correction parameters
    trk_vz: np.ndarray | None = None  # f64 [T] vertex z (cm)

    @property
    def n(self) -> int:
        return int(self.y.shape[0])

    def sector_of_cluster(self) -> np.ndarray:
        grp = np.repeat(np.arange(self.n_events * N_SECTORS),
                        np.diff(self.evt_sector_off))
        return (grp % N_SECTORS).astype(np.int32)

    def truth_tracks(self, n_min: int = 10):
        """Truth hit lists: (trk_off, trk_hits, track ids) for tracks with
        >= n_min clusters, hits in input-order indices, outermost first
        (descending arc length along the helix)."""
        sig = np.nonzero(self.mc_track >= 0)[0]
        if self.arc_true is not None:
            arc = self.arc_true[sig]
        else:
            arc = ROW_X[self.row[sig]]
        order = np.lexsort((-arc, self.mc_track[sig]))
        sig = sig[order]
        tid = self.mc_track[sig]
        ids, start, cnt = np.unique(tid, return_index=True, return_counts=True)
        keep = cnt >= n_min
        parts = [sig[s:s + c] for s, c, k in zip(start, cnt, keep) if k]
        hits = np.concatenate(parts).astype(np.int32) if parts else np.zeros(0, np.int32)
        off = np.zeros(int(keep.sum()) + 1, np.int32)
        off[1:] = np.cumsum(cnt[keep])
        return off, hits, ids[keep]

    def truth_segments(self, n_min: int = 10):
        """Truth hit lists split by side: one segment per (track, side) with
        >= n_min clusters, outermost first.  Returns (trk_off, trk_hits,
        track ids, sides (0 = A, 1 = C)); a track that crosses the central
        membrane gives two segments."""
        sig = np.nonzero(self.mc_track >= 0)[0]
        side = (self.sector_of_cluster()[sig] >= N_PHI).astype(np.int64)
        arc = self.arc_true[sig] if self.arc_true is not None else ROW_X[self.row[sig]]
        order = np.lexsort((-arc, side, self.mc_track[sig]))
        sig, side = sig[order], side[order]
        key = self.mc_track[sig].astype(np.int64) * 2 + side
        keys, start, cnt = np.unique(key, return_index=True, return_counts=True)
        keep = cnt >= n_min
        parts = [sig[s_:s_ + c] for s_, c, k in zip(start, cnt, keep) if k]
        hits = np.concatenate(parts).astype(np.int32) if parts else np.zeros(0, np.int32)
        off = np.zeros(int(keep.sum()) + 1, np.int32)
        off[1:] = np.cumsum(cnt[keep])
        return off, hits, (keys[keep] // 2).astype(np.int64), (keys[keep] % 2).astype(np.int32)


def _grid_voxel(sector, row, y, z, grid):
    """Voxel of the distortion model (grid as in FIELD_GRID) at local (y, z)
    on pad row `row` of `sector`, binned in FP64: the detector model's own
    piecewise-constant field, independent of the reconstruction's binning."""
    nb, ny, nz = grid["n_band"], grid["n_y"], grid["n_z"]
    band = row * nb // N_ROWS
    iy = np.clip(np.floor((y / ROW_X[row] - grid["u_lo"]) * grid["u_inv"]), 0, ny - 1).astype(np.int64)
    iz = np.clip(np.floor(np.abs(z) * grid["z_inv"]), 0, nz - 1).astype(np.int64)
    return ((sector * nb + band) * ny + iy) * nz + iz


def _crossings(phi0, k, tgl, wedge, misalign, want_truth, distortion=None, vz=None):
    """Intersect each helix with every accepted (sector, row) plane.

    vz: None (every track from z = 0, its side fixed by the sign of tan
    lambda), or the vertex z of each track: z = vz + tan(lambda) s, and each
    crossing goes to the sector of the side its own z lies on (a track can
    cross the central membrane and leave clusters on both sides).

    Works in the global transverse plane: the track circle has centre
    C = (sin phi0, -cos phi0)/k and passes through the origin; the outgoing
    crossing of the line n.P = x_r (n = (cos a, sin a)) has direction angle
    psi = a - asin(k (x_r - n.C)).
    Returns per-crossing arrays (track, sector, row, y, z, snp, arc).
    """
    T = phi0.shape[0]
    cx = np.sin(phi0) / k
    cy = -np.cos(phi0) / k
    r_hi = X_LAST / math.cos(SECTOR_WIDTH / 2) + 1.0
    th_a = phi0 - np.arcsin(np.clip(k * X_FIRST / 2, -1, 1))
    th_b = phi0 - np.arcsin(np.clip(k * r_hi / 2, -1, 1))
    i_lo = np.floor(np.minimum(th_a, th_b) / SECTOR_WIDTH).astype(np.int64)
    i_hi = np.floor(np.maximum(th_a, th_b) / SECTOR_WIDTH).astype(np.int64)
    side = np.where(tgl >= 0, 0, N_PHI)
    out = []
    xr = ROW_X[None, :]
    for slot in range(6):
        iphi = i_lo + slot
        valid = iphi <= i_hi
        if wedge is not None:
            valid &= (iphi % N_PHI) == wedge
        if not valid.any():
            continue
        t_idx = np.nonzero(valid)[0]
        a = (iphi[t_idx] + 0.5) * SECTOR_WIDTH
        ca, sa = np.cos(a)[:, None], np.sin(a)[:, None]
        kk = k[t_idx][:, None]
        nc = ca * cx[t_idx][:, None] + sa * cy[t_idx][:, None]
        q = kk * (xr - nc)
        ok = np.abs(q) < 1.0
        qc = np.clip(q, -0.999999, 0.999999)
        psi = a[:, None] - np.arcsin(qc)
        dphi = phi0[t_idx][:, None] - psi
        two_pi = 2 * math.pi
        dpos = np.mod(dphi, two_pi)
        dneg = -np.mod(-dphi, two_pi)
        dd = np.where(kk > 0, dpos, dneg)
        s = dd / kk
        ok &= (s > 0) & (np.abs(dd) <= math.pi)
        px = cx[t_idx][:, None] + (-np.sin(psi)) / kk
        py = cy[t_idx][:, None] + np.cos(psi) / kk
        yl = -sa * px + ca * py
        zl = tgl[t_idx][:, None] * s
        snp = np.sin(psi - a[:, None])
        sector = (iphi[t_idx] % N_PHI + side[t_idx])[:, None] + np.zeros_like(s, dtype=np.int64)
        if vz is not None:
            zl = zl + vz[t_idx][:, None]
            sector = (iphi[t_idx] % N_PHI)[:, None] + np.where(zl >= 0.0, 0, N_PHI)
        if (misalign is not None or distortion is not None) and vz is not None:
            raise ValueError("a vertex spread is not combined with misalignment or distortion")
        if misalign is not None or distortion is not None:
            # measured point on the displaced plane: x of R^T (P - D) = x_r,
            # solved only where the nominal crossing exists
            ti0, ri0 = np.nonzero(ok)
            args = (phi0[t_idx][ti0], kk[ti0, 0], tgl[t_idx][ti0], a[ti0], cx[t_idx][ti0],
                    cy[t_idx][ti0], s[ti0, ri0], ROW_X[ri0])
            sec0 = sector[ti0, ri0]
            if misalign is not None:
                par = misalign.reshape(N_SECTORS, 6)
                Rs = np.stack([rotation_matrix(*par[i, 3:6]) for i in range(N_SECTORS)])
                ym, zm, sm = _displaced_crossing(*args, Rs[sec0], par[sec0, 0:3])
            else:
                # distortion: the measured cluster is the true one moved by
                # -F[v], v the voxel of the measured position (found from
                # the nominal crossing, then once more from the result)
                grid, field = distortion
                eye = np.broadcast_to(np.eye(3), (len(ti0), 3, 3))
                v = _grid_voxel(sec0, ri0, yl[ti0, ri0], zl[ti0, ri0], grid)
                ym, zm, sm = _displaced_crossing(*args, eye, field[v])
                v2 = _grid_voxel(sec0, ri0, ym, zm, grid)
                moved = v2 != v
                if moved.any():
                    a2 = tuple(x[moved] for x in args)
                    y2, z2, s2 = _displaced_crossing(*a2, eye[moved], field[v2[moved]])
                    ym, zm, sm = ym.copy(), zm.copy(), sm.copy()
                    ym[moved], zm[moved], sm[moved] = y2, z2, s2
            yl = np.zeros_like(s)
            zl = np.zeros_like(s)
            yl[ti0, ri0] = ym
            zl[ti0, ri0] = zm
            s = s.copy()
            s[ti0, ri0] = sm
        ok &= np.abs(yl) <= xr * TAN_HALF_SECTOR
        ok &= np.abs(zl) < Z_MAX
        ti, ri = np.nonzero(ok)
        out.append((t_idx[ti], sector[ti, ri], ri, yl[ti, ri], zl[ti, ri],
                    snp[ti, ri], s[ti, ri]))
    if not out:
        e = np.zeros(0)
        return (e.astype(np.int64),) * 3 + (e,) * 4
    return tuple(np.concatenate([o[j] for o in out]) for j in range(7))


def _displaced_crossing(phi0, k, tgl, a, cx, cy, s, xr, R, D):
    """Newton solve (1-d arrays, one entry per crossing) for the arc length
    where the helix meets the displaced row plane {R (x_r, y, z) + D}
    (R [m, 3, 3], D [m, 3] per crossing); returns the measured (y, z) in
    that plane and the arc length."""
    ca, sa = np.cos(a), np.sin(a)
    s = s.copy()

    def rt(v0, v1, v2):  # R^T v, component-wise
        return (R[:, 0, 0] * v0 + R[:, 1, 0] * v1 + R[:, 2, 0] * v2,
                R[:, 0, 1] * v0 + R[:, 1, 1] * v1 + R[:, 2, 1] * v2,
                R[:, 0, 2] * v0 + R[:, 1, 2] * v1 + R[:, 2, 2] * v2)

    def measured(s):
        psi = phi0 - k * s
        px = cx + (-np.sin(psi)) / k
        py = cy + np.cos(psi) / k
        m = rt(ca * px + sa * py - D[:, 0], -sa * px + ca * py - D[:, 1], tgl * s - D[:, 2])
        return np.stack(m, -1), psi

    for _ in range(4):
        meas, psi = measured(s)
        d0 = rt(np.cos(psi - a), np.sin(psi - a), tgl)[0]
        s = s - (meas[:, 0] - xr) / d0
    meas, _ = measured(s)
    return meas[:, 1], meas[:, 2], s


def _draw_tracks(rng, n, pt_min, pt_slope, wedge):
    pt = pt_min + rng.exponential(pt_slope, n)
    eta = rng.uniform(-0.9, 0.9, n)
    tgl = np.sinh(eta)
    if wedge is None:
        phi0 = rng.uniform(0.0, 2 * math.pi, n)
    else:
        phi0 = rng.uniform(wedge * SECTOR_WIDTH, (wedge + 1) * SECTOR_WIDTH, n)
    q = np.where(rng.uniform(size=n) < 0.5, 1.0, -1.0)
    return q, pt, tgl, phi0


def _one_collision(rng, n_tracks, noise_frac, wedge, pt_min, pt_slope,
                   misalign, want_truth, t0_us, tid0, distortion=None, vz_sigma=0.0):
    q, pt, tgl, phi0 = _draw_tracks(rng, n_tracks, pt_min, pt_slope, wedge)
    # vertex z spread: drawn only when asked for, so that every other
    # workload keeps its random stream
    vz = rng.normal(0.0, vz_sigma, n_tracks) if vz_sigma > 0 else None
    k = KAPPA * BZ * q / pt
    parts = []
    CH = 8192
    for c0 in range(0, n_tracks, CH):
        sl = slice(c0, min(n_tracks, c0 + CH))
        tr, sec, row, y, z, snp, arc = _crossings(phi0[sl], k[sl], tgl[sl], wedge,
                                                  misalign, want_truth, distortion,
                                                  None if vz is None else vz[sl])
        parts.append((tr + c0, sec, row, y, z, snp, arc))
    tr, sec, row, yt, zt, snp, arc = (np.concatenate([p[j] for p in parts]) for j in range(7))
    keep = rng.uniform(size=tr.shape[0]) >= ROW_DROP
    tr, sec, row, yt, zt, snp, arc = (v[keep] for v in (tr, sec, row, yt, zt, snp, arc))
    ym = yt + rng.normal(0.0, SIGMA_Y, yt.shape[0])
    zm = zt + rng.normal(0.0, SIGMA_Z, zt.shape[0])
    chg = np.minimum(20 + np.round(rng.exponential(60.0, yt.shape[0])), 65535)
    n_sig = tr.shape[0]
    n_noise = int(round(noise_frac / (1.0 - noise_frac) * n_sig)) if noise_frac > 0 else 0
    if wedge is None:
        nsec = rng.integers(0, N_SECTORS, n_noise)
    else:
        nsec = wedge + N_PHI * rng.integers(0, 2, n_noise)
    nrow = rng.integers(0, N_ROWS, n_noise)
    half = ROW_X[nrow] * TAN_HALF_SECTOR
    ny = rng.uniform(-1.0, 1.0, n_noise) * half
    nz = rng.uniform(0.0, Z_MAX, n_noise) * np.where(nsec < N_PHI, 1.0, -1.0)
    nchg = rng.integers(1, 101, n_noise)
    # drift-time shift (frames): A side z' = z - v t0, C side z' = z + v t0
    if t0_us != 0.0:
        shift = V_DRIFT * t0_us
        zm = zm - np.where(sec < N_PHI, shift, -shift)
        nz = nz - np.where(nsec < N_PHI, shift, -shift)
    cl = dict(
        sector=np.concatenate([sec, nsec]).astype(np.int64),
        row=np.concatenate([row, nrow]).astype(np.uint16),
        y=np.concatenate([ym, ny]),
        z=np.concatenate([zm, nz]),
        charge=np.concatenate([chg, nchg]).astype(np.uint16),
        mc=np.concatenate([tr + tid0, np.full(n_noise, -1)]).astype(np.int32),
        y_true=np.concatenate([yt, np.full(n_noise, np.nan)]),
        z_true=np.concatenate([zt, np.full(n_noise, np.nan)]),
        snp_true=np.concatenate([snp, np.full(n_noise, np.nan)]),
        arc_true=np.concatenate([arc, np.full(n_noise, np.nan)]),
    )
    trk = dict(q=q, pt=pt, tgl=tgl, phi0=phi0, vz=np.zeros(n_tracks) if vz is None else vz)
    return cl, trk


def generate(events, seed, wedge=None, pt_min=0.2, pt_slope=0.5,
             misalign=None, truth=False, frame=None, distortion=None, vz_sigma=0.0):
    """Generate a batch.

    vz_sigma: the Gaussian spread (cm) of the tracks' vertex z (0: every
            track from z = 0, none crossing the central membrane).

    distortion: None, or (grid, field[n_voxels, 3]): each signal cluster is
            measured displaced by -field[v] from the helix crossing (the
            plane moved by field[v][0]), v its voxel; exclusive with
            misalign.
    events: list of (n_tracks, noise_frac) per event.
    frame:  None, or a list of (n_tracks, noise_frac) per collision; all
            collisions then share one event with uniform drift-time offsets
            over FRAME_US (z shifted by V_DRIFT * t0).
    """
    if misalign is not None and distortion is not None:
        raise ValueError("misalign and distortion are exclusive")
    rng = np.random.default_rng(seed)
    if frame is not None:
        specs = [[(nt, nf, rng.uniform(0.0, FRAME_US)) for nt, nf in frame]]
    else:
        specs = [[(nt, nf, 0.0)] for nt, nf in events]
    cls, trks = [], []
    tid0 = 0
    for ev, colls in enumerate(specs):
        for nt, nf, t0 in colls:
            cl, trk = _one_collision(rng, nt, nf, wedge, pt_min, pt_slope,
                                     misalign, truth, t0, tid0, distortion, vz_sigma)
            cl['event'] = np.full(cl['row'].shape[0], ev, np.int64)
            trk['event'] = np.full(nt, ev, np.int32)
            trk['t0'] = np.full(nt, t0)
            tid0 += nt
            cls.append(cl)
            trks.append(trk)
    cat = {key: np.concatenate([c[key] for c in cls]) for key in cls[0]}
    E = len(specs)
    key = cat['event'] * N_SECTORS + cat['sector']
    if E == 1:
        perm = rng.permutation(key.shape[0])
        order = perm[np.argsort(key[perm], kind='stable')]
    else:
        # events are contiguous in generation order: group and shuffle each
        bounds = np.searchsorted(cat['event'], np.arange(E + 1))
        parts = []
        for e in range(E):
            b0, b1 = bounds[e], bounds[e + 1]
            perm = rng.permutation(b1 - b0)
            parts.append(b0 + perm[np.argsort(cat['sector'][b0:b1][perm], kind='stable')])
        order = np.concatenate(parts)
    counts = np.bincount(key, minlength=E * N_SECTORS)
    off = np.zeros(E * N_SECTORS + 1, np.int64)
    off[1:] = np.cumsum(counts)
    trk = {key_: np.concatenate([t[key_] for t in trks]) for key_ in trks[0]}
    ev = Events(
        y=cat['y'][order].astype(np.float32),
        z=cat['z'][order].astype(np.float32),
        row=cat['row'][order],
        charge=cat['charge'][order],
        evt_sector_off=off, n_events=E,
        mc_track=cat['mc'][order],
        trk_q=trk['q'], trk_pt=trk['pt'], trk_tgl=trk['tgl'],
        trk_phi0=trk['phi0'], trk_event=trk['event'], trk_t0=trk['t0'],
    )
    ev.trk_vz = trk['vz']
    ev.arc_true = cat['arc_true'][order]
    if truth:
        ev.y_true = cat['y_true'][order]
        ev.z_true = cat['z_true'][order]
        ev.snp_true = cat['snp_true'][order]
    if misalign is not None:
        ev.align = np.asarray(misalign, np.float64).copy()
    if distortion is not None:
        ev.field = np.asarray(distortion[1], np.float64).copy()
    return ev


# --- parallel generation ---------------------------------------------------------

def _unit(args):
    """One independently seeded generation unit (an event, a collision of a
    frame, or a chunk of the tracks of one event) for generate_parallel."""
    seed, n_tracks, noise, wedge, pt_min, pt_slope, misalign, t0, vz_sigma = args
    rng = np.random.default_rng(seed)
    cl, trk = _one_collision(rng, n_tracks, noise, wedge, pt_min, pt_slope, misalign, False, t0, 0,
                             vz_sigma=vz_sigma)
    keep = ("sector", "row", "y", "z", "charge", "mc", "arc_true")
    cl = {k: cl[k] for k in keep}
    cl["y"] = cl["y"].astype(np.float32)
    cl["z"] = cl["z"].astype(np.float32)
    return cl, trk


def generate_parallel(units, seed, workers=None, wedge=None, pt_min=0.2, pt_slope=0.5,
                      misalign=None, vz_sigma=0.0):
    """Like generate() for many units, in a spawn-context process pool.

    units: list of (event index, n_tracks, noise_frac[, t0_us]); units of
    one event are merged into that event (t0_us: drift-time offset of a
    collision in a frame).  Unit u draws from PCG64 seeded with
    (seed, u), so the result does not depend on the number of workers (it
    differs from generate() with the same seed)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    if workers is None:
        workers = max(1, len(os.sched_getaffinity(0)))
    units = [tuple(u) + (0.0,) * (4 - len(u)) for u in units]
    jobs = [((seed, u), nt, nf, wedge, pt_min, pt_slope, misalign, t0, vz_sigma)
            for u, (_, nt, nf, t0) in enumerate(units)]
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_unit, jobs, chunksize=max(1, len(jobs) // (4 * workers))))
    E = max(u[0] for u in units) + 1
    tid0 = 0
    cls, trks = [], []
    for (ev, nt, _, t0), (cl, trk) in zip(units, res):
        cl["mc"] = np.where(cl["mc"] >= 0, cl["mc"] + tid0, -1).astype(np.int32)
        cl["event"] = np.full(cl["row"].shape[0], ev, np.int64)
        trk["event"] = np.full(nt, ev, np.int32)
        trk["t0"] = np.full(nt, t0)
        tid0 += nt
        cls.append(cl)
        trks.append(trk)
    cat = {key: np.concatenate([c[key] for c in cls]) for key in cls[0]}
    key = cat["event"] * N_SECTORS + cat["sector"]
    rng = np.random.default_rng((seed, len(units)))
    order = np.argsort(key * (1 << 31) + rng.integers(0, 1 << 31, key.shape[0]), kind="stable")
    counts = np.bincount(key, minlength=E * N_SECTORS)
    off = np.zeros(E * N_SECTORS + 1, np.int64)
    off[1:] = np.cumsum(counts)
    trk = {k: np.concatenate([t[k] for t in trks]) for k in trks[0]}
    ev = Events(y=cat["y"][order], z=cat["z"][order], row=cat["row"][order],
                charge=cat["charge"][order], evt_sector_off=off, n_events=E,
                mc_track=cat["mc"][order], trk_q=trk["q"], trk_pt=trk["pt"], trk_tgl=trk["tgl"],
                trk_phi0=trk["phi0"], trk_event=trk["event"], trk_t0=trk["t0"])
    ev.trk_vz = trk["vz"]
    ev.arc_true = cat["arc_true"][order]
    if misalign is not None:
        ev.align = np.asarray(misalign, np.float64).copy()
    return ev


def pileup_frame_parallel(n_collisions=100, n_tracks=10000, noise=0.20, seed=SEED_BASE + 2,
                          workers=None):
    """The 50 kHz frame generated in parallel (one unit per collision)."""
    rng = np.random.default_rng(seed + 2000003)
    t0 = rng.uniform(0.0, FRAME_US, n_collisions)
    return generate_parallel([(0, n_tracks, noise, float(t0[i])) for i in range(n_collisions)],
                             seed, workers=workers)


def uneven_batch_parallel(n_events=512, lo=10, hi=10000, seed=SEED_BASE + 3, workers=None):
    """The uneven 512-event batch, generated in parallel (one unit per event)."""
    rng = np.random.default_rng(seed + 1000003)
    nt = np.exp(rng.uniform(math.log(lo), math.log(hi), n_events)).round().astype(int)
    nf = rng.uniform(0.05, 0.30, n_events)
    return generate_parallel([(e, int(nt[e]), float(nf[e])) for e in range(n_events)], seed,
                             workers=workers)


def alignment_sample_parallel(n_tracks=200000, seed=SEED_BASE + 4, misalign=None, chunk=5000,
                              workers=None):
    """The alignment sample (one event) generated in parallel track chunks."""
    if misalign is None:
        misalign = draw_misalignment(seed)
    units = []
    left = n_tracks
    while left > 0:
        units.append((0, min(chunk, left), 0.0))
        left -= chunk
    return generate_parallel(units, seed, workers=workers, pt_min=1.0, pt_slope=0.5,
                             misalign=misalign)


# --- the five workload shapes -------------------------------------------------

def one_sector(n_tracks=200, noise=0.10, seed=SEED_BASE + 0, truth=False):
    """One 20-degree wedge (sectors 0 and 18), 200 tracks, 10% noise."""
    return generate([(n_tracks, noise)], seed, wedge=0, truth=truth)


def central_event(n_tracks=10000, noise=0.20, seed=SEED_BASE + 1, truth=False):
    """One central Pb-Pb-like event over 36 sectors, 1e4 tracks, 20% noise."""
    return generate([(n_tracks, noise)], seed, truth=truth)


def pileup_frame(n_collisions=100, n_tracks=10000, noise=0.20,
                 seed=SEED_BASE + 2, truth=False):
    """50 kHz frame: collisions at uniform drift-time offsets over 2 ms."""
    return generate(None, seed, frame=[(n_tracks, noise)] * n_collisions,
                    truth=truth)


VZ_SIGMA = 6.0   # cm, vertex z spread of the membrane-crossing frames


def membrane_frame(n_collisions=20, n_tracks=2000, noise=0.20, vz_sigma=VZ_SIGMA,
                   seed=SEED_BASE + 8, truth=False):
    """A pile-up frame whose collisions have a vertex z spread: tracks of
    small |tan lambda| cross the central membrane and leave one segment on
    each side, seen shifted in opposite directions by the collision's
    drift-time offset."""
    return generate(None, seed, frame=[(n_tracks, noise)] * n_collisions, truth=truth,
                    vz_sigma=vz_sigma)


def membrane_frame_parallel(n_collisions=100, n_tracks=10000, noise=0.20, vz_sigma=VZ_SIGMA,
                            seed=SEED_BASE + 8, workers=None):
    """The 50 kHz frame with a vertex z spread, generated in parallel."""
    rng = np.random.default_rng(seed + 2000003)
    t0 = rng.uniform(0.0, FRAME_US, n_collisions)
    return generate_parallel([(0, n_tracks, noise, float(t0[i])) for i in range(n_collisions)],
                             seed, workers=workers, vz_sigma=vz_sigma)


def uneven_batch(n_events=512, lo=10, hi=10000, seed=SEED_BASE + 3, truth=False):
    """Events with log-uniform multiplicity in [lo, hi] and noise U[5%,30%]."""
    rng = np.random.default_rng(seed + 1000003)
    nt = np.exp(rng.uniform(math.log(lo), math.log(hi), n_events)).round().astype(int)
    nf = rng.uniform(0.05, 0.30, n_events)
    return generate(list(zip(nt.tolist(), nf.tolist())), seed, truth=truth)


def draw_misalignment(seed=SEED_BASE + 4, shift_sigma=0.01, rot_sigma=1e-4):
    """36 x (dx, dy, dz, a, b, g): shifts sigma 100 um, rotations 0.1 mrad."""
    rng = np.random.default_rng(seed + 7777)
    m = np.empty((N_SECTORS, 6))
    m[:, 0:3] = rng.normal(0.0, shift_sigma, (N_SECTORS, 3))
    m[:, 3:6] = rng.normal(0.0, rot_sigma, (N_SECTORS, 3))
    return m.reshape(-1)


# Voxel grid of the distortion map (the build's reading of the space-charge
# distortion map of Sec. 4.2; the paper gives no grid): 8 bands of 19 pad
# rows, 4 bins of y/x over the sector acceptance, 5 bins of |z| over the
# drift length.  Plain numbers; each side builds its own grid record.
FIELD_GRID = dict(n_band=8, n_y=4, n_z=5, u_lo=-TAN_HALF_SECTOR,
                  u_inv=4 / (2 * TAN_HALF_SECTOR), z_inv=5 / Z_MAX)


def n_voxels(grid=FIELD_GRID):
    return N_SECTORS * grid["n_band"] * grid["n_y"] * grid["n_z"]


def draw_field(seed=SEED_BASE + 5, sigma=0.02, grid=FIELD_GRID):
    """A random displacement field [n_voxels, 3]: each (x, y, z) component of
    each voxel N(0, sigma) cm."""
    rng = np.random.default_rng(seed + 5555)
    return rng.normal(0.0, sigma, (n_voxels(grid), 3))


def distortion_sample(n_tracks=2000, seed=SEED_BASE + 5, field=None, grid=FIELD_GRID):
    """pT > 1 GeV/c tracks, no noise, clusters displaced by a voxel field
    (default: draw_field(seed)); the field is kept as ev.field."""
    if field is None:
        field = draw_field(seed, grid=grid)
    return generate([(n_tracks, 0.0)], seed, pt_min=1.0, pt_slope=0.5, distortion=(grid, field))


def alignment_sample(n_tracks=200000, seed=SEED_BASE + 4, misalign=None,
                     n_events=1):
    """pT > 1 GeV/c tracks, no noise, clusters on misaligned row planes."""
    if misalign is None:
        misalign = draw_misalignment(seed)
    per = [(n_tracks // n_events + (1 if i < n_tracks % n_events else 0), 0.0)
           for i in range(n_events)]
    return generate(per, seed, pt_min=1.0, pt_slope=0.5, misalign=misalign)


CONFIG_NAMES = ("one_sector", "central_event", "pileup_frame", "uneven_batch",
                "alignment_sample")


# --- tracks through material (Kalman-filter variants) ---------------------------

PION_MASS = 0.13957      # GeV/c^2
MAT_X_X0_ROW = 1e-4      # radiation lengths of one pad-row layer at normal incidence
MAT_ELOSS_ROW = 2e-6     # GeV lost in one pad-row layer at normal incidence


def highland_theta0(p, beta, x_x0):
    """Width (rad) of the projected multiple-scattering angle after x_x0
    radiation lengths for a unit-charge particle of momentum p (GeV/c) and
    velocity beta (the Highland formula, PDG Review of Particle Physics)."""
    x = np.maximum(x_x0, 1e-300)
    return np.where(x_x0 > 0, 0.0136 / (beta * p) * np.sqrt(x) * (1.0 + 0.038 * np.log(x)), 0.0)


def material_tracks(n_tracks=2000, seed=SEED_BASE + 6, x_x0_row=MAT_X_X0_ROW,
                    eloss_row=MAT_ELOSS_ROW, mass=PION_MASS, pt_min=0.3, pt_slope=0.5,
                    sector=0):
    """Pions from the origin through the pad rows of one sector, with
    material concentrated in the row planes: each plane the track crosses
    deflects it by two independent Gaussian angles of width theta0 (Highland,
    x/X0 = x_x0_row times the path factor 1/(cos phi cos lambda)) and takes
    eloss_row times the same factor off its energy, after the crossing is
    recorded.  Between planes the track is an exact helix in Bz.

    Returns an Events batch of one event (clusters smeared as everywhere
    else, no noise) whose truth arrays hold, per cluster, the state arriving
    at its plane (before that plane's deflection and loss): y_true, z_true,
    snp_true and, as attributes, tgl_true and qpt_true."""
    rng = np.random.default_rng(seed)
    q = np.where(rng.uniform(size=n_tracks) < 0.5, 1.0, -1.0)
    pt = pt_min + rng.exponential(pt_slope, n_tracks)
    lam = np.arctan(np.sinh(rng.uniform(-0.9, 0.9, n_tracks)))
    phi = rng.uniform(-0.06, 0.06, n_tracks)           # local direction at the origin
    lam0, phi0 = lam.copy(), phi.copy()
    p = pt / np.cos(lam)
    e = np.sqrt(p * p + mass * mass)
    xs, ys, zs = np.zeros(n_tracks), np.zeros(n_tracks), np.zeros(n_tracks)
    alive = np.ones(n_tracks, bool)
    rec = []
    for r in range(N_ROWS):
        xr = ROW_X[r]
        k = KAPPA * BZ * q / (p * np.cos(lam))
        s0 = np.sin(phi)
        s1 = s0 - k * (xr - xs)
        alive &= np.abs(s1) < 0.9
        s1 = np.clip(s1, -0.9, 0.9)
        c0, c1 = np.sqrt(1 - s0 * s0), np.sqrt(1 - s1 * s1)
        y1 = ys + (c1 - c0) / k
        arc = (np.arcsin(s0) - np.arcsin(s1)) / k
        z1 = zs + np.tan(lam) * arc
        alive &= (np.abs(y1) <= xr * TAN_HALF_SECTOR) & (np.abs(z1) < Z_MAX)
        idx = np.nonzero(alive)[0]
        if idx.size == 0:
            break
        rec.append((idx, np.full(idx.size, r), y1[idx], z1[idx], s1[idx], np.tan(lam[idx]),
                    (q / (p * np.cos(lam)))[idx]))
        # the plane's material: deflection, then energy loss
        phi = np.arcsin(s1)
        path = 1.0 / (c1 * np.cos(lam))
        beta = p / e
        th0 = highland_theta0(p, beta, x_x0_row * path)
        phi = phi + rng.normal(0.0, 1.0, n_tracks) * th0 / np.cos(lam)
        lam = lam + rng.normal(0.0, 1.0, n_tracks) * th0
        e = e - eloss_row * path
        alive &= e > mass * 1.001
        p = np.sqrt(np.maximum(e * e - mass * mass, 1e-12))
        xs, ys, zs = np.full(n_tracks, xr), y1, z1
    tr, row, yt, zt, st, tt, wt = (np.concatenate([a[j] for a in rec]) for j in range(7))
    keep = rng.uniform(size=tr.shape[0]) >= ROW_DROP
    tr, row, yt, zt, st, tt, wt = (v[keep] for v in (tr, row, yt, zt, st, tt, wt))
    ym = yt + rng.normal(0.0, SIGMA_Y, yt.shape[0])
    zm = zt + rng.normal(0.0, SIGMA_Z, zt.shape[0])
    # a track's clusters go to the sector of its side at the origin (a
    # scattering that carries a flat track across z = 0 does not move them)
    sec = sector % N_PHI + N_PHI * (lam0[tr] < 0)
    order = np.lexsort((tr, sec))
    counts = np.bincount(sec, minlength=N_SECTORS)
    off = np.zeros(N_SECTORS + 1, np.int64)
    off[1:] = np.cumsum(counts)
    ev = Events(y=ym[order].astype(np.float32), z=zm[order].astype(np.float32),
                row=row[order].astype(np.uint16), charge=np.full(len(order), 50, np.uint16),
                evt_sector_off=off, n_events=1, mc_track=tr[order].astype(np.int32),
                trk_q=q, trk_pt=pt, trk_tgl=np.tan(lam0),
                trk_phi0=phi0 + float(sector_alpha(sector)), trk_event=np.zeros(n_tracks, np.int32),
                trk_t0=np.zeros(n_tracks))
    ev.arc_true = ROW_X[row[order]]
    ev.y_true, ev.z_true, ev.snp_true = yt[order], zt[order], st[order]
    ev.tgl_true, ev.qpt_true = tt[order], wt[order]
    return ev


# --- pad-time digits (clusterization input) ----------------------------------------

# The build's digit format (the paper gives none): per (event, sector, pad
# row) a dense array of 10-bit ADC counts, u16 [N_TIME][N_PAD], pads
# contiguous.  Pad p covers y in [(p - 80) PAD_W, (p - 79) PAD_W); time bin t
# covers |z| in [t T_W, (t + 1) T_W) (z < 0 on the C side).
N_PAD = 160
N_TIME = 512
PAD_W = 0.6          # cm
T_W = 0.5            # cm of drift per time bin
DIGIT_SIGMA_PAD = 0.7    # charge spread, pads
DIGIT_SIGMA_TIME = 0.8   # charge spread, time bins
DIGIT_GAIN = 4.0     # ADC counts per unit of cluster charge
DIGIT_NOISE = 1.0    # ADC noise on digits with signal
DIGIT_ZS = 3         # zero suppression: counts below are dropped
ADC_MAX = 1023


def _bin_fraction(c, sigma, k):
    """Fraction of a Gaussian (centre c, width sigma, in bin units) inside
    bin k = [k, k + 1)."""
    from scipy.special import erf
    a = (k - c) / (sigma * math.sqrt(2.0))
    b = (k + 1 - c) / (sigma * math.sqrt(2.0))
    return 0.5 * (erf(b) - erf(a))


def digitize(ev, seed=SEED_BASE + 7, n_time=N_TIME):
    """Pad-time digits of an Events batch: every cluster deposits
    DIGIT_GAIN x its charge as a 2-d Gaussian over the 5 x 5 bins around its
    (pad, time) centre; digits with signal get N(0, DIGIT_NOISE) noise, are
    rounded down to integers, clamped to [0, ADC_MAX] and dropped below
    DIGIT_ZS (zero suppression; digits without signal stay 0).  Returns
    u16 [n_events * 36 * 152, n_time, N_PAD]."""
    rng = np.random.default_rng(seed)
    n_planes = ev.n_events * N_SECTORS * N_ROWS
    grp = np.repeat(np.arange(ev.n_events * N_SECTORS), np.diff(ev.evt_sector_off))
    plane = grp.astype(np.int64) * N_ROWS + ev.row.astype(np.int64)
    cp = ev.y.astype(np.float64) / PAD_W + 80.0
    ct = np.abs(ev.z.astype(np.float64)) / T_W
    q = ev.charge.astype(np.float64) * DIGIT_GAIN
    p0 = np.floor(cp).astype(np.int64)
    t0 = np.floor(ct).astype(np.int64)
    idxs, ws = [], []
    for dp in range(-2, 3):
        kp = p0 + dp
        fp = _bin_fraction(cp, DIGIT_SIGMA_PAD, kp)
        for dt in range(-2, 3):
            kt = t0 + dt
            ft = _bin_fraction(ct, DIGIT_SIGMA_TIME, kt)
            ok = (kp >= 0) & (kp < N_PAD) & (kt >= 0) & (kt < n_time)
            idxs.append((plane[ok] * n_time + kt[ok]) * N_PAD + kp[ok])
            ws.append((q * fp * ft)[ok])
    idx = np.concatenate(idxs)
    w = np.concatenate(ws)
    order = np.argsort(idx, kind="stable")
    idx, w = idx[order], w[order]
    start = np.flatnonzero(np.r_[True, idx[1:] != idx[:-1]])
    uniq = idx[start]
    acc = np.add.reduceat(w, start)
    val = np.floor(acc + rng.normal(0.0, DIGIT_NOISE, uniq.size))
    val = np.clip(val, 0, ADC_MAX)
    val[val < DIGIT_ZS] = 0
    out = np.zeros(n_planes * n_time * N_PAD, np.uint16)
    out[uniq] = val.astype(np.uint16)
    return out.reshape(n_planes, n_time, N_PAD)
