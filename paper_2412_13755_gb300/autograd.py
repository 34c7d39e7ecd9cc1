"""torch.autograd wrapper of the alignment chi2 (tpc_fit_adjoint).

TPCChi2.apply(align, tracker, trk_off, trk_hits, n_tracks) returns the total
fit chi2 of the given tracks (FP64 scalar) as a function of the 216
per-sector corrections; backward() runs the library's hand-written reverse
sweep and scales it by the incoming gradient.
"""
from __future__ import annotations

import torch

from . import tpc


class TPCChi2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, align, tracker, trk_off, trk_hits, n_tracks):
        if align.dtype != torch.float64 or align.numel() != 216:
            raise TypeError("align must be a float64 tensor of 216 corrections")
        a = align.detach().contiguous()
        chi2, _ = tracker.adjoint(trk_off, trk_hits, n_tracks, a, want_grad=False)
        ctx.save_for_backward(a)
        ctx.tracker, ctx.trk_off, ctx.trk_hits, ctx.n_tracks = tracker, trk_off, trk_hits, n_tracks
        return chi2.reshape(())

    @staticmethod
    def backward(ctx, g):
        (a,) = ctx.saved_tensors
        _, grad = ctx.tracker.adjoint(ctx.trk_off, ctx.trk_hits, ctx.n_tracks, a, want_grad=True)
        return g * grad, None, None, None, None


def total_chi2(align, tracker, trk_off, trk_hits, n_tracks):
    return TPCChi2.apply(align, tracker, trk_off, trk_hits, n_tracks)
