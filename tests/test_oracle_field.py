"""Pins of the oracle's distortion-map gradient: the TPC space-charge
distortion evaluation (Sec. 4.2) read as a piecewise-constant displacement
per voxel of the sector frames, estimated from the summed track chi2.

* Voxel membership: every index is in range and names the cluster's sector
  and pad-row band; a cluster well inside a bin (y/x and |z| at least 1% of
  a bin width from its edges, beyond any FP32 rounding) lies in the bin that
  contains it in exact arithmetic; coordinates beyond the grid go to the
  edge bins.
* A field constant over each sector is a rigid translation of that sector:
  its chi2 equals the alignment chi2 with the same shifts and no rotation,
  bit for bit (the two corrected positions are the same FP64 numbers), and
  the field gradient summed over a sector's voxels equals the alignment
  gradient's shift components (the alignment gradient is itself pinned to
  finite differences).
* FP64 central finite differences of the summed chi2 with respect to
  sampled voxel components (h = 1e-6 cm).
* Voxels without clusters have zero gradient; a zero field gives the plain
  fit sum; a rigid alignment and a field combine.
"""
import numpy as np
import pytest

from paper_2412_13755_gb300 import synth

G = synth.FIELD_GRID


@pytest.fixture(scope="module")
def grid(orc):
    return orc.field_grid(**G)


def _sample(n_tracks=150, seed=41):
    ev = synth.alignment_sample(n_tracks=n_tracks, seed=seed, misalign=np.zeros(216))
    off, hits, _ = ev.truth_tracks(n_min=10)
    return ev, ev.sector_of_cluster(), off, hits


def test_voxel_membership(orc, grid):
    ev = synth.central_event(n_tracks=2000, seed=42)
    sec = ev.sector_of_cluster()
    vox, nv = orc.voxel_of(ev.y, ev.z, ev.row, sec, grid)
    nb, ny, nz = G["n_band"], G["n_y"], G["n_z"]
    assert nv == 36 * nb * ny * nz
    assert vox.min() >= 0 and vox.max() < nv
    iz = vox % nz
    iy = (vox // nz) % ny
    band = (vox // (nz * ny)) % nb
    s = vox // (nz * ny * nb)
    assert np.array_equal(s, sec)
    assert np.array_equal(band, ev.row.astype(np.int64) // (152 // nb))
    # exact-arithmetic bins of the clusters well inside one
    x = synth.ROW_X[ev.row]
    fy = (ev.y.astype(np.float64) / x - G["u_lo"]) * G["u_inv"]
    fz = np.abs(ev.z.astype(np.float64)) * G["z_inv"]
    inside = (np.abs(fy - np.floor(fy) - 0.5) < 0.49) & (np.abs(fz - np.floor(fz) - 0.5) < 0.49)
    inside &= (fy > 0) & (fy < ny) & (fz < nz)
    assert inside.mean() > 0.9
    assert np.array_equal(iy[inside], np.floor(fy[inside]).astype(np.int64))
    assert np.array_equal(iz[inside], np.floor(fz[inside]).astype(np.int64))


def test_out_of_range_coordinates_go_to_the_edge_bins(orc, grid):
    row = np.array([0, 151, 75, 75, 10, 10], np.uint16)
    x = synth.ROW_X[row]
    y = np.array([-2.0, 2.0, 0.0, 0.0, np.nan, 0.0]) * x
    z = np.array([0.0, 1e4, -1e4, 0.0, 0.0, np.inf])
    sec = np.array([0, 35, 17, 18, 3, 3], np.int32)
    vox, _ = orc.voxel_of(y.astype(np.float32), z.astype(np.float32), row, sec, grid)
    ny, nz = G["n_y"], G["n_z"]
    iz, iy = vox % nz, (vox // nz) % ny
    assert list(iy[:2]) == [0, ny - 1] and list(iz[1:3]) == [nz - 1, nz - 1]
    assert iy[4] == 0 and iz[5] == nz - 1


@pytest.mark.parametrize("g", [None, dict(n_band=4, n_y=2, n_z=3, u_lo=-0.2, u_inv=5.0, z_inv=0.012)])
def test_constant_field_is_a_rigid_translation(orc, grid, g):
    ev, sec, off, hits = _sample()
    rng = np.random.default_rng(5)
    shift = rng.normal(0.0, 0.02, (36, 3))
    align = np.zeros((36, 6))
    align[:, :3] = shift
    if g is not None:
        grid = orc.field_grid(**g)
    nv = synth.n_voxels(G if g is None else g)
    field = np.repeat(shift, nv // 36, axis=0)
    c_f, g_f = orc.field_adjoint(ev.y, ev.z, ev.row, sec, off, hits, grid, field)
    c_a, g_a = orc.fit_adjoint(ev.y, ev.z, ev.row, sec, off, hits, align.reshape(-1))
    assert c_f == c_a
    per_sector = g_f.reshape(36, nv // 36, 3).sum(axis=1)
    want = g_a.reshape(36, 6)[:, :3]
    np.testing.assert_allclose(per_sector, want, rtol=1e-9, atol=1e-9 * np.abs(want).max())
    assert np.abs(want).max() > 1.0


def test_gradient_matches_central_differences(orc, grid):
    ev, sec, off, hits = _sample(n_tracks=120, seed=43)
    field = synth.draw_field(seed=43, sigma=0.02)
    c, g = orc.field_adjoint(ev.y, ev.z, ev.row, sec, off, hits, grid, field)
    vox, nv = orc.voxel_of(ev.y, ev.z, ev.row, sec, grid)
    used = np.unique(vox[hits])
    rng = np.random.default_rng(6)
    pick = [(int(v), int(c_)) for v in rng.choice(used, 24, replace=False) for c_ in range(3)]
    h = 1e-6
    scale = np.abs(g).max()
    assert scale > 1.0
    for v, k in pick:
        fp, fm = field.copy(), field.copy()
        fp[v, k] += h
        fm[v, k] -= h
        cp = orc.field_adjoint(ev.y, ev.z, ev.row, sec, off, hits, grid, fp, want_grad=False)
        cm = orc.field_adjoint(ev.y, ev.z, ev.row, sec, off, hits, grid, fm, want_grad=False)
        fd = (cp - cm) / (2 * h)
        assert abs(g[v, k] - fd) <= 1e-6 * abs(fd) + 1e-6 * scale, (v, k, g[v, k], fd)


def test_empty_voxels_zero_field_and_combination(orc, grid):
    ev, sec, off, hits = _sample(n_tracks=100, seed=44)
    nv = synth.n_voxels()
    vox, _ = orc.voxel_of(ev.y, ev.z, ev.row, sec, grid)
    empty = np.setdiff1d(np.arange(nv), vox[hits])
    field = synth.draw_field(seed=44)
    c, g = orc.field_adjoint(ev.y, ev.z, ev.row, sec, off, hits, grid, field)
    assert len(empty) > 0 and np.all(g[empty] == 0.0)
    # zero field: the plain fit sum
    c0 = orc.field_adjoint(ev.y, ev.z, ev.row, sec, off, hits, grid, np.zeros((nv, 3)), want_grad=False)
    par, cov, c2, ndf = orc.fit_tracks(ev.y, ev.z, ev.row, sec, off, hits)
    assert c0 == c2[ndf > 0].sum() or abs(c0 - c2[ndf > 0].sum()) <= 1e-12 * c0
    # alignment and field together: a sector's rigid shift moves into the
    # field without changing chi2
    mis = synth.draw_misalignment(44)
    al = mis.copy().reshape(36, 6)
    moved = al[:, :3].copy()
    al[:, :3] = 0.0
    f2 = field + np.repeat(moved, nv // 36, axis=0)
    c_both = orc.field_adjoint(ev.y, ev.z, ev.row, sec, off, hits, grid, field, align=mis,
                               want_grad=False)
    c_moved = orc.field_adjoint(ev.y, ev.z, ev.row, sec, off, hits, grid, f2, align=al.reshape(-1),
                                want_grad=False)
    assert abs(c_both - c_moved) <= 1e-9 * c_both


def test_generated_distortion_lies_on_the_helix_once_undone():
    """The generator's distortion model: a noiseless distorted cluster moved
    back by +F[v] (v its voxel) lies on its track's helix: on the circle of
    radius 1/|k| through the origin and at z = tan(lambda) times the arc
    length."""
    F = synth.draw_field(seed=61, sigma=0.05)
    ev = synth.generate([(150, 0.0)], 61, pt_min=1.0, distortion=(G, F), truth=True)
    sec = ev.sector_of_cluster().astype(np.int64)
    row = ev.row.astype(np.int64)
    v = synth._grid_voxel(sec, row, ev.y_true, ev.z_true, G)
    x = synth.ROW_X[row] + F[v, 0]
    y = ev.y_true + F[v, 1]
    z = ev.z_true + F[v, 2]
    a = synth.sector_alpha(sec)
    X, Y = x * np.cos(a) - y * np.sin(a), x * np.sin(a) + y * np.cos(a)
    t = ev.mc_track
    k = synth.KAPPA * synth.BZ * ev.trk_q[t] / ev.trk_pt[t]
    phi0 = ev.trk_phi0[t]
    cx, cy = np.sin(phi0) / k, -np.cos(phi0) / k
    r_err = np.abs(np.hypot(X - cx, Y - cy) * np.abs(k) - 1.0)
    psi = np.arctan2(-(X - cx) * k, (Y - cy) * k)
    d = np.where(k > 0, np.mod(phi0 - psi, 2 * np.pi), -np.mod(psi - phi0, 2 * np.pi))
    z_err = np.abs(z - ev.trk_tgl[t] * d / k)
    on = (r_err < 1e-9) & (z_err < 1e-7)
    # within one displacement of a y or |z| bin edge the voxel can flip
    # between the nominal and the displaced crossing, and the cluster keep
    # the other voxel's displacement; everywhere else it must be exact
    fy = (ev.y_true / synth.ROW_X[row] - G["u_lo"]) * G["u_inv"]
    fz = np.abs(ev.z_true) * G["z_inv"]
    edge = (np.abs(fy - np.round(fy)) * synth.ROW_X[row] / G["u_inv"] < 0.5) | \
           (np.abs(fz - np.round(fz)) / G["z_inv"] < 0.5)
    assert np.all(on[~edge]), (r_err[~edge].max(), z_err[~edge].max())
    assert edge.mean() < 0.15 and on.mean() > 0.99
    assert np.abs(F[v]).max() > 0.1


def test_field_that_undoes_the_distortion_minimises_chi2(orc, grid):
    """Along the line t F from no correction to the generated field, the
    summed chi2 is smallest at t = 1, and the field gradient there is small
    along F compared with its value at t = 0."""
    F = synth.draw_field(seed=62, sigma=0.05)
    ev = synth.distortion_sample(n_tracks=300, seed=62, field=F)
    off, hits, _ = ev.truth_tracks(n_min=10)
    sec = ev.sector_of_cluster()
    ts = np.array([0.0, 0.5, 1.0, 1.5, 2.0])
    c = np.array([orc.field_adjoint(ev.y, ev.z, ev.row, sec, off, hits, grid, t * F, want_grad=False)
                  for t in ts])
    a2, a1, _ = np.polyfit(ts, c, 2)
    t_min = -a1 / (2 * a2)
    print(f"chi2 along t F: {c.round(1)}, vertex t = {t_min:.4f}")
    assert a2 > 0 and abs(t_min - 1.0) < 0.05
    assert c[2] == c.min()
    _, g0 = orc.field_adjoint(ev.y, ev.z, ev.row, sec, off, hits, grid, 0 * F)
    _, g1 = orc.field_adjoint(ev.y, ev.z, ev.row, sec, off, hits, grid, F)
    d0, d1 = float(np.sum(g0 * F)), float(np.sum(g1 * F))
    assert d0 < 0 and abs(d1) < 0.05 * abs(d0), (d0, d1)


def test_gn_blocks_are_the_exact_hessian_in_the_linear_case(orc, grid):
    """With Bz = 0 and the sin phi and q/pT priors at zero the fit is linear
    in the measurements, so the chi2 is exactly quadratic in a voxel's
    (dy, dz): its (y, z) Gauss-Newton block equals the Hessian, here from
    central differences of the exact gradient."""
    prm = orc.default_params(bz=0.0, prior=[4.0, 4.0, 0.0, 0.25, 0.0])
    ev, sec, off, hits = _sample(n_tracks=40, seed=45)
    field = synth.draw_field(seed=45, sigma=0.02)
    B = orc.field_gn_blocks(ev.y, ev.z, ev.row, sec, off, hits, grid, field, params=prm)
    vox, nv = orc.voxel_of(ev.y, ev.z, ev.row, sec, grid)
    cnt = np.bincount(vox[hits], minlength=nv)
    h = 1e-3
    for v in np.argsort(cnt)[::-1][:4]:
        for c in (1, 2):
            fp, fm = field.copy(), field.copy()
            fp[v, c] += h
            fm[v, c] -= h
            _, gp = orc.field_adjoint(ev.y, ev.z, ev.row, sec, off, hits, grid, fp, params=prm)
            _, gm = orc.field_adjoint(ev.y, ev.z, ev.row, sec, off, hits, grid, fm, params=prm)
            hess = (gp[v, 1:] - gm[v, 1:]) / (2 * h)
            np.testing.assert_allclose(B[v, c, 1:], hess, rtol=1e-8, atol=1e-8 * np.abs(hess).max())
            assert B[v, c, c] > 100.0


def test_gn_blocks_symmetric_psd_and_empty_voxels_zero(orc, grid):
    ev, sec, off, hits = _sample(n_tracks=100, seed=46)
    B = orc.field_gn_blocks(ev.y, ev.z, ev.row, sec, off, hits, grid, synth.draw_field(seed=46))
    vox, nv = orc.voxel_of(ev.y, ev.z, ev.row, sec, grid)
    used = np.bincount(vox[hits], minlength=nv) > 0
    assert np.allclose(B, B.transpose(0, 2, 1), rtol=1e-12, atol=1e-9)
    w = np.linalg.eigvalsh(B[used])
    assert w.min() > -1e-9 * w.max()
    assert np.all(B[~used] == 0.0)


def test_damped_block_descent_recovers_the_field(orc, grid):
    """Calibration from the adjoint: on clusters generated with a y, z
    distortion, three damped block-Gauss-Newton steps (each voxel's (y, z)
    block from the oracle at the start, plus a tenth of its mean diagonal)
    lower the chi2 at every step and cut the rms error of the (y, z)
    field over voxels with >= 30 clusters by at least 40%, toward the
    statistical floor of about 0.1 cm / sqrt(clusters per voxel)."""
    F = synth.draw_field(seed=63, sigma=0.05)
    F[:, 0] = 0.0
    ev = synth.distortion_sample(n_tracks=2000, seed=63, field=F)
    off, hits, _ = ev.truth_tracks(n_min=10)
    sec = ev.sector_of_cluster()
    vox, nv = orc.voxel_of(ev.y, ev.z, ev.row, sec, grid)
    used = np.bincount(vox[hits], minlength=nv) >= 30
    B = orc.field_gn_blocks(ev.y, ev.z, ev.row, sec, off, hits, grid, np.zeros_like(F))[used][:, 1:, 1:]
    B = B + 0.05 * np.trace(B, axis1=1, axis2=2)[:, None, None] * np.eye(2)
    theta = np.zeros_like(F)
    chi2s, errs = [], []
    for _ in range(4):
        c, g = orc.field_adjoint(ev.y, ev.z, ev.row, sec, off, hits, grid, theta)
        chi2s.append(c)
        errs.append(np.sqrt(np.mean((theta - F)[used][:, 1:] ** 2)))
        theta[used, 1:] -= np.linalg.solve(B, g[used][:, 1:, None])[..., 0]
    print(f"chi2 {np.round(chi2s, 1)}, rms (y, z) error {np.round(errs, 4)}")
    assert all(b < a for a, b in zip(chi2s, chi2s[1:]))
    assert errs[-1] < 0.6 * errs[0]
