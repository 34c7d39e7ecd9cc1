"""GPU distortion-map gradient (the space-charge distortion evaluation of
Sec. 4.2, read as a piecewise-constant displacement per voxel of the sector
frames) against the oracle.

* chi2 total and d chi2 / d field: the hand-written reverse sweep, scattered
  per run of clusters in one voxel, vs the oracle's exact gradient (dual
  numbers): chi2 within 1e-5 relative, the gradient within 1e-4
  norm-relative, voxels without clusters exactly 0.
* The field gradient summed over a sector's voxels equals the alignment
  gradient's shift components of the same call (both sum the same
  per-cluster position adjoints).
* A zero field reproduces tpc_fit_adjoint: the same chi2 and alignment
  gradient.
* On clusters generated with a distortion F, the field that undoes it
  minimises the GPU chi2 along t F.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2412_13755_gb300 import synth, tpc  # noqa: E402
from gpu_util import to_dev  # noqa: E402

G = synth.FIELD_GRID


def _setup(n_tracks, seed):
    ev = synth.alignment_sample(n_tracks=n_tracks, seed=seed, misalign=synth.draw_misalignment(seed))
    off, hits, _ = ev.truth_tracks(n_min=10)
    tr = tpc.Tracker(ev.n, 1)
    keep = to_dev(ev)
    tr.load(*keep, 1)
    tr._keep = keep
    return ev, off, hits, tr


def test_field_gradient_matches_oracle(orc):
    ev, off, hits, tr = _setup(2000, 51)
    sec = ev.sector_of_cluster()
    field = synth.draw_field(seed=51, sigma=0.02)
    align = 0.5 * synth.draw_misalignment(51)
    d_off, d_hits = torch.from_numpy(off).cuda(), torch.from_numpy(hits).cuda()
    chi2, g_al, g_f = tr.adjoint_field(d_off, d_hits, len(off) - 1, tpc.field_grid(**G),
                                       torch.from_numpy(field).cuda(),
                                       align=torch.from_numpy(align).cuda())
    torch.cuda.synchronize()
    tr.check()
    o_chi2, o_g = orc.field_adjoint(ev.y, ev.z, ev.row, sec, off, hits, orc.field_grid(**G), field,
                                    align=align)
    g = g_f.cpu().numpy()
    rel_chi2 = abs(chi2.item() - o_chi2) / o_chi2
    rel_g = np.linalg.norm(g - o_g) / np.linalg.norm(o_g)
    print(f"chi2 rel {rel_chi2:.2e}  field grad norm-rel {rel_g:.2e}  |g| {np.linalg.norm(o_g):.3e}")
    assert rel_chi2 < 1e-5
    assert rel_g < 1e-4
    empty = np.all(o_g == 0, axis=1)
    assert empty.any() and np.all(g[empty] == 0)
    # per sector, the voxels' shift gradients add up to the alignment's
    per_sector = g.reshape(36, -1, 3).sum(axis=1)
    want = g_al.cpu().numpy().reshape(36, 6)[:, :3]
    np.testing.assert_allclose(per_sector, want, rtol=1e-9, atol=1e-9 * np.abs(want).max())


def test_zero_field_is_the_alignment_adjoint():
    ev, off, hits, tr = _setup(1000, 52)
    align = torch.from_numpy(0.5 * synth.draw_misalignment(52)).cuda()
    d_off, d_hits = torch.from_numpy(off).cuda(), torch.from_numpy(hits).cuda()
    T = len(off) - 1
    zero = torch.zeros(synth.n_voxels(), 3, dtype=torch.float64, device="cuda")
    chi2_f, g_al, g_f = tr.adjoint_field(d_off, d_hits, T, tpc.field_grid(**G), zero, align=align)
    chi2_a, g_a = tr.adjoint(d_off, d_hits, T, align)
    torch.cuda.synchronize()
    tr.check()
    assert abs(chi2_f.item() - chi2_a.item()) <= 1e-12 * chi2_a.item()
    a = g_a.cpu().numpy()
    np.testing.assert_allclose(g_al.cpu().numpy(), a, rtol=1e-9, atol=1e-9 * np.abs(a).max())
    # forward only: the same chi2, no gradients
    chi2_o, none_a, none_f = tr.adjoint_field(d_off, d_hits, T, tpc.field_grid(**G), zero, align=align,
                                              want_grad=False)
    assert none_a is None and none_f is None
    assert abs(chi2_o.item() - chi2_a.item()) <= 1e-12 * chi2_a.item()


def test_field_buffers_and_grid_refused():
    ev, off, hits, tr = _setup(50, 53)
    d_off, d_hits = torch.from_numpy(off).cuda(), torch.from_numpy(hits).cuda()
    T = len(off) - 1
    short = torch.zeros(synth.n_voxels() - 1, 3, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError, match="field"):
        tr.adjoint_field(d_off, d_hits, T, tpc.field_grid(**G), short)
    bad = dict(G, n_band=7)
    with pytest.raises(ValueError, match="grid"):
        tr.adjoint_field(d_off, d_hits, T, tpc.field_grid(**bad),
                         torch.zeros(synth.n_voxels(), 3, dtype=torch.float64, device="cuda"))
    tr.check()


def test_field_that_undoes_the_distortion_on_gpu():
    """On clusters generated with a distortion F, the GPU chi2 along t F is
    smallest at t = 1, and the GPU field gradient along F is negative at
    t = 0 and below 5% of that at t = 1."""
    F = synth.draw_field(seed=54, sigma=0.05)
    ev = synth.distortion_sample(n_tracks=3000, seed=54, field=F)
    off, hits, _ = ev.truth_tracks(n_min=10)
    tr = tpc.Tracker(ev.n, 1)
    keep = to_dev(ev)
    tr.load(*keep, 1)
    d_off, d_hits = torch.from_numpy(off).cuda(), torch.from_numpy(hits).cuda()
    T = len(off) - 1
    res = {}
    for t in (0.0, 1.0, 2.0):
        chi2, _, g = tr.adjoint_field(d_off, d_hits, T, tpc.field_grid(**G),
                                      torch.from_numpy(t * F).cuda())
        res[t] = (chi2.item(), float(np.sum(g.cpu().numpy() * F)))
    torch.cuda.synchronize()
    tr.check()
    print({t: (round(c, 1), round(d, 1)) for t, (c, d) in res.items()})
    assert res[1.0][0] < res[0.0][0] and res[1.0][0] < res[2.0][0]
    assert res[0.0][1] < 0 and abs(res[1.0][1]) < 0.05 * abs(res[0.0][1])


def test_field_descent_on_gpu(orc):
    """Three damped block Gauss-Newton steps driven by the GPU field
    gradient (blocks from the oracle at the start) cut the (y, z) field
    error by at least 40% on generated distortions, and end where the same
    steps driven by the oracle's gradient end."""
    F = synth.draw_field(seed=63, sigma=0.05)
    F[:, 0] = 0.0
    ev = synth.distortion_sample(n_tracks=2000, seed=63, field=F)
    off, hits, _ = ev.truth_tracks(n_min=10)
    sec = ev.sector_of_cluster()
    og = orc.field_grid(**G)
    vox, nv = orc.voxel_of(ev.y, ev.z, ev.row, sec, og)
    used = np.bincount(vox[hits], minlength=nv) >= 30
    B = orc.field_gn_blocks(ev.y, ev.z, ev.row, sec, off, hits, og, np.zeros_like(F))[used][:, 1:, 1:]
    B = B + 0.05 * np.trace(B, axis1=1, axis2=2)[:, None, None] * np.eye(2)
    tr = tpc.Tracker(ev.n, 1)
    keep = to_dev(ev)
    tr.load(*keep, 1)
    d_off, d_hits = torch.from_numpy(off).cuda(), torch.from_numpy(hits).cuda()
    T = len(off) - 1

    def descend(grad_of):
        theta = np.zeros_like(F)
        errs = []
        for _ in range(3):
            g = grad_of(theta)
            errs.append(np.sqrt(np.mean((theta - F)[used][:, 1:] ** 2)))
            theta[used, 1:] -= np.linalg.solve(B, g[used][:, 1:, None])[..., 0]
        errs.append(np.sqrt(np.mean((theta - F)[used][:, 1:] ** 2)))
        return theta, errs

    def gpu_grad(theta):
        _, _, g = tr.adjoint_field(d_off, d_hits, T, tpc.field_grid(**G), torch.from_numpy(theta).cuda())
        return g.cpu().numpy()

    th_g, errs = descend(gpu_grad)
    torch.cuda.synchronize()
    tr.check()
    th_o, _ = descend(lambda th: orc.field_adjoint(ev.y, ev.z, ev.row, sec, off, hits, og, th)[1])
    d = np.sqrt(np.mean((th_g - th_o)[used] ** 2)) / np.sqrt(np.mean(th_o[used] ** 2))
    print(f"rms (y, z) error {np.round(errs, 4)}; GPU vs oracle end point {d:.2e}")
    assert errs[-1] < 0.6 * errs[0]
    assert d < 1e-3


def test_field_calibration_without_the_oracle():
    """The calibration driver (limited-memory BFGS over the GPU adjoint's
    exact gradient, a Tikhonov term for the undetermined directions) needs
    no CPU reference: on generated (y, z) distortions of sigma 0.5 mm it
    lowers the objective at every iteration and cuts the rms (y, z) field
    error over the voxels with >= 30 clusters to below 0.6 of the
    distortion, the bar the block Gauss-Newton descent meets (the field
    patterns along a track that its own parameters absorb stay
    undetermined).  The Tikhonov weight is the generator's prior, 1/sigma^2:
    the minimum is then the posterior mode (a weight of 1 leaves the weakly
    determined directions to fit noise, and the converged error grows to
    0.66 of the distortion)."""
    from paper_2412_13755_gb300 import calib
    F = synth.draw_field(seed=63, sigma=0.05)
    F[:, 0] = 0.0
    ev = synth.distortion_sample(n_tracks=2000, seed=63, field=F)
    off, hits, _ = ev.truth_tracks(n_min=10)
    tr = tpc.Tracker(ev.n, 1)
    keep = to_dev(ev)
    tr.load(*keep, 1)
    sec = ev.sector_of_cluster()
    # voxels with enough clusters, counted with the generator's binning
    # (plain bookkeeping for the mask; the calibration itself uses none)
    g = synth.FIELD_GRID
    vox = synth._grid_voxel(sec, ev.row, ev.y.astype(np.float64), ev.z.astype(np.float64), g)
    used = np.bincount(vox[hits], minlength=synth.n_voxels(g)) >= 30
    mask = np.zeros((synth.n_voxels(g), 3), bool)
    mask[used, 1:] = True
    d_off, d_hits = torch.from_numpy(off).cuda(), torch.from_numpy(hits).cuda()
    errs = {}

    def err_of(it, est, f):
        if it % 20 == 0:
            errs[it] = round(float(np.sqrt(np.mean((est - F)[used][:, 1:] ** 2))), 4)

    est, hist = calib.calibrate_field(tr, d_off, d_hits, len(off) - 1, tpc.field_grid(**G), iters=200,
                                      lam=1.0 / 0.05 ** 2, mask=mask, callback=err_of)
    tr.check()
    e0 = np.sqrt(np.mean(F[used][:, 1:] ** 2))
    e1 = np.sqrt(np.mean((est - F)[used][:, 1:] ** 2))
    print(f"objective {hist[0]:.6e} -> {hist[-1]:.6e} in {len(hist) - 1} iterations; "
          f"rms (y, z) error {e0:.4f} -> {e1:.4f} cm; by iteration {errs}")
    assert all(b <= a for a, b in zip(hist, hist[1:]))
    assert e1 < 0.6 * e0
