"""Helpers for the GPU parity tests: run the CUDA path through the C ABI on
synthetic events, and compare track assignments canonically."""
import numpy as np
import torch

from paper_2412_13755_gb300 import tpc


def to_dev(ev, dev="cuda"):
    y = torch.from_numpy(np.ascontiguousarray(ev.y)).to(dev)
    z = torch.from_numpy(np.ascontiguousarray(ev.z)).to(dev)
    row = torch.from_numpy(np.ascontiguousarray(ev.row).view(np.int16)).to(dev).view(torch.uint16)
    off = torch.from_numpy(np.ascontiguousarray(ev.evt_sector_off)).to(dev)
    return y, z, row, off


def gpu_find(ev, tracker=None, params=None):
    tr = tracker or tpc.Tracker(max(ev.n, 1), ev.n_events, params=params)
    y, z, row, off = to_dev(ev)
    tr.load(y, z, row, off, ev.n_events)
    toc, trk_off, hits, ntd = tr.find()
    torch.cuda.synchronize()
    st = tr.check()
    T = int(ntd.item())
    o = trk_off[:T + 1].cpu().numpy()
    return toc.cpu().numpy()[:ev.n], o, hits[:o[-1]].cpu().numpy(), st, tr


def canon_of_cluster(toc, trk_off, hits, n):
    """Per cluster: the smallest input index of its track (-1 = none)."""
    out = np.full(n, -1, np.int64)
    for k in range(len(trk_off) - 1):
        h = hits[trk_off[k]:trk_off[k + 1]]
        out[h] = h.min()
    return out
