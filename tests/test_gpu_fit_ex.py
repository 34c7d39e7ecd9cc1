"""NEXT-3 on the GPU through the C ABI: the Kalman-filter variants
(material in the pad-row planes, outward refit, Rauch-Tung-Striebel
smoother) against the FP64 oracle on tracks generated through material,
with the bars of the host check (tests/test_fit_ex_host.py): parameters and
chi2 within 1e-9, covariances within 1e-7 (smoothed 1e-6) of their scale,
ndf equal; and the GPU's pulls with material are unit-width."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2412_13755_gb300 import synth, tpc  # noqa: E402
from gpu_util import to_dev  # noqa: E402

SCALE = np.array([1.0, 1.0, 0.1, 0.1, 0.1])
DIAG = [0, 5, 9, 12, 14]
IU = [(i, j) for i in range(5) for j in range(i, 5)]


def _rel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), SCALE)


def _crel(c, oc):
    d = oc[:, DIAG]
    cs = np.stack([np.sqrt(np.abs(d[:, i] * d[:, j])) for i, j in IU], 1)
    return np.abs(c - oc) / np.maximum(cs, 1e-300)


def _setup(seed=91, n=2000, eloss=3e-5):
    ev = synth.material_tracks(n, seed=seed, eloss_row=eloss)
    off, hits, _ = ev.truth_tracks(n_min=10)
    tr = tpc.Tracker(ev.n, 1)
    tr.load(*to_dev(ev), 1)
    return ev, off, hits, tr


def _orc_prm(orc, x0, el, m):
    return orc.default_params(mat_x_x0=float(np.float32(x0)), mat_eloss=float(np.float32(el)),
                              mass=float(np.float32(m)))


@pytest.mark.parametrize("outward", [False, True])
def test_material_fit_parity(orc, outward):
    ev, off, hits, tr = _setup()
    x0, el, m = synth.MAT_X_X0_ROW, 3e-5, synth.PION_MASS
    o = tpc.fit_options(x0, el, m, outward=outward)
    T = len(off) - 1
    par, cov, chi2, ndf, _ = tr.fit_ex(torch.from_numpy(off).cuda(), torch.from_numpy(hits).cuda(), T, o)
    torch.cuda.synchronize()
    tr.check()
    opar, ocov, ochi2, ondf = orc.fit_tracks(ev.y, ev.z, ev.row, ev.sector_of_cluster(), off, hits,
                                             params=_orc_prm(orc, x0, el, m), reverse=outward)
    par, cov = par.cpu().numpy().astype(np.float64), cov.cpu().numpy().astype(np.float64)
    chi2, ndf = chi2.cpu().numpy().astype(np.float64), ndf.cpu().numpy()
    assert np.array_equal(ndf <= 0, ondf <= 0)
    ok = ondf > 0
    assert np.array_equal(ndf[ok], ondf[ok])
    # the outputs are FP32 (the state is FP64 inside): the bar is FP32 rounding
    rel, crel = _rel(par, opar)[ok], _crel(cov, ocov)[ok]
    chrel = (np.abs(chi2 - ochi2) / np.maximum(ochi2, 1.0))[ok]
    print(f"{ok.sum()} tracks: params {rel.max():.2e} cov {crel.max():.2e} chi2 {chrel.max():.2e}")
    assert rel.max() <= 1e-6 and crel.max() <= 1e-6 and chrel.max() <= 1e-6
    # pulls against the generator's truth at the fit's end cluster
    end = hits[off[:-1]] if outward else hits[off[1:] - 1]
    truth = np.stack([ev.y_true[end], ev.z_true[end], ev.snp_true[end], ev.tgl_true[end], ev.qpt_true[end]], 1)
    pull = ((par - truth) / np.sqrt(cov[:, DIAG]))[ok]
    print("pull mean", np.round(pull.mean(0), 3), "std", np.round(pull.std(0), 3))
    assert np.all(np.abs(pull.mean(0)) < 0.07) and np.all((pull.std(0) > 0.94) & (pull.std(0) < 1.06))


def test_smoother_parity(orc):
    ev, off, hits, tr = _setup(seed=92, n=1000)
    x0, el, m = synth.MAT_X_X0_ROW, 3e-5, synth.PION_MASS
    T = len(off) - 1
    out = tr.fit_ex(torch.from_numpy(off).cuda(), torch.from_numpy(hits).cuda(), T,
                    tpc.fit_options(x0, el, m), smooth=True)
    torch.cuda.synchronize()
    tr.check()
    sm = out[4].cpu().numpy()[:off[-1]]
    osm, _, ondf = orc.smooth_tracks(ev.y, ev.z, ev.row, ev.sector_of_cluster(), off, hits,
                                     params=_orc_prm(orc, x0, el, m))
    ok = np.repeat(ondf > 0, np.diff(off))
    rel = _rel(sm[:, :5], osm[:, :5])[ok]
    crel = _crel(sm[:, 5:], osm[:, 5:])[ok]
    print(f"{ok.sum()} smoothed states: params {rel.max():.2e} cov {crel.max():.2e}")
    assert rel.max() <= 1e-9 and crel.max() <= 1e-6
    assert np.all(sm[~ok] == 0)


def test_smoother_refused_for_outward_fits():
    ev, off, hits, tr = _setup(seed=93, n=50)
    T = len(off) - 1
    with pytest.raises(tpc.TPCError, match="TPC_ERR_ARG"):
        tr.fit_ex(torch.from_numpy(off).cuda(), torch.from_numpy(hits).cuda(), T,
                  tpc.fit_options(1e-4, 0.0, 0.13957, outward=True), smooth=True)
