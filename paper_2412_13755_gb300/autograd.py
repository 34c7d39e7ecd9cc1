"""torch.autograd wrapper of the alignment chi2 (tpc_fit_adjoint).

TPCChi2.apply(align, tracker, trk_off, trk_hits, n_tracks) returns the total
fit chi2 of the given tracks (FP64 scalar) as a function of the 216
per-sector corrections.  When align requires a gradient, forward() runs the
library's forward and hand-written reverse sweep in one call (each track is
recomputed inside the kernel, nothing is stored per cluster) and keeps the
216 gradient values; backward() only scales them by the incoming gradient.
Without a gradient, forward() runs the forward sweep alone.
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
        want = bool(ctx.needs_input_grad[0])
        chi2, grad = tracker.adjoint(trk_off, trk_hits, n_tracks, a, want_grad=want)
        if want:
            ctx.save_for_backward(grad)
        return chi2.reshape(())

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None, None, None, None


def total_chi2(align, tracker, trk_off, trk_hits, n_tracks):
    return TPCChi2.apply(align, tracker, trk_off, trk_hits, n_tracks)
