"""Calibration drivers over the library's adjoint (NEXT-1, the space-charge
distortion map of Sec. 4.2, read as a per-voxel displacement field).

The heavy part of every iteration, the summed chi2 of all tracks and its
exact gradient with respect to the 3 n_voxels field components, runs in the
library's adjoint kernel on the GPU (tpc_fit_adjoint_field).  The driver
only combines those gradients: limited-memory BFGS (two-loop recursion over
the last `memory` steps, Armijo backtracking), so the descent needs no
second-derivative blocks and no CPU reference.  A Tikhonov term
lam * |F|^2 pins the directions the tracks do not determine (the field's
rigid modes, and x, which trades against the track parameters).
"""
from __future__ import annotations

import numpy as np
import torch

from . import tpc


def calibrate_field(tracker: tpc.Tracker, trk_off, trk_hits, n_tracks: int, grid: tpc.FieldGrid,
                    iters: int = 30, lam: float = 1.0, memory: int = 10, mask=None, field0=None,
                    align=None, callback=None):
    """Field minimising sum(chi2) + lam |F|^2 over the components where
    `mask` (bool [n_voxels, 3], default all) is set, from field0 (default 0).
    callback(iteration, field, objective), when given, sees every accepted
    iterate.  Returns (field [n_voxels, 3] float64 numpy, list of objective
    values)."""
    nv = tpc.tpc_field_voxels(grid)
    dev = tracker.device
    F = np.zeros((nv, 3)) if field0 is None else np.array(field0, np.float64).reshape(nv, 3)
    m = np.ones((nv, 3), bool) if mask is None else np.asarray(mask, bool).reshape(nv, 3)
    if align is None:
        align = torch.zeros(216, dtype=torch.float64, device=dev)

    def objective(x):
        chi2, _, g = tracker.adjoint_field(trk_off, trk_hits, n_tracks, grid,
                                           torch.from_numpy(x).to(dev), align=align)
        g = g.cpu().numpy() + 2.0 * lam * x
        return float(chi2.item()) + lam * float(np.sum(x * x)), np.where(m, g, 0.0)

    f, g = objective(F)
    hist = [f]
    S, Y = [], []
    for _ in range(iters):
        # two-loop recursion: d = -H g
        q = g.copy()
        alphas = []
        for s, y in reversed(list(zip(S, Y))):
            rho = 1.0 / float(np.sum(y * s))
            a = rho * float(np.sum(s * q))
            alphas.append((a, rho))
            q -= a * y
        if S:
            s, y = S[-1], Y[-1]
            q *= float(np.sum(s * y)) / float(np.sum(y * y))
        else:
            q *= 1e-3 / max(float(np.max(np.abs(g))), 1e-300)   # first step: at most 10 um
        for (s, y), (a, rho) in zip(zip(S, Y), reversed(alphas)):
            b = rho * float(np.sum(y * q))
            q += (a - b) * s
        d = -q
        slope = float(np.sum(g * d))
        if slope >= 0:  # not a descent direction: restart from the gradient
            S, Y = [], []
            d = -g * (1e-3 / max(float(np.max(np.abs(g))), 1e-300))
            slope = float(np.sum(g * d))
        t = 1.0
        while True:
            Fn = F + t * d
            fn, gn = objective(Fn)
            if fn <= f + 1e-4 * t * slope:
                break
            t *= 0.5
            if t < 1e-6:  # no decrease left to resolve: converged
                return F, hist
        s, y = Fn - F, gn - g
        if float(np.sum(s * y)) > 1e-12 * float(np.sum(y * y)):
            S.append(s)
            Y.append(y)
            if len(S) > memory:
                S.pop(0)
                Y.pop(0)
        F, f, g = Fn, fn, gn
        hist.append(f)
        if callback is not None:
            callback(len(hist) - 1, F, f)
    return F, hist
