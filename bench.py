#!/usr/bin/env python3
"""Benchmark of the TPC tracking path on GB300.

One step = the whole tracking path over one central Pb-Pb-like event
(36 sectors, 1e4 primary tracks, 20% noise, ~1.8e6 clusters): register the
clusters (S0), bin (S1), neighbours (S2), chains and Kalman-guided tracklets
(S3), merge (S4), and the Kalman fit of every found track (S5).  Metric:
clusters per second.  The inputs (~22 MB) are smaller than L2, so L2 is
flushed (512 MB write) between timed steps.  Synthetic seeded events stand in
for ALICE Run-3 data.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle (the paper publishes no code to
compare with) on the same workload, on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TPC clusters/s tracked (CA+Kalman), 1 GB300"
WORKLOAD = ("central_event: 1 event x 36 sectors, 1e4 primary tracks (pT exp slope 0.5 GeV/c "
            "min 0.2, |eta|<0.9), 20% noise, ~1.8e6 clusters, Bz 0.5 T")
FP32_LANES_PER_SM = 128                 # Blackwell SM: 4 partitions x 32 FP32 lanes
FP64_NOMINAL_TFLOPS = 1.25   # GB300 dense FP64, nominal (no FP64 figure is measured on this machine)
# algorithmic traffic / work per unit, fixed before measuring
# the whole find + fit path, every intermediate product written once and read
# once: binning 22, neighbours 16, chains and tracks 16, fit 12.7, scatter 12
PATH_BYTES_PER_CLUSTER = 78.7
# the fused lower bound: read y, z, row once (10), write each cluster's track
# (4) and the per-track fit outputs (88 B per ~120 clusters, 0.7)
PATH_FUSED_BYTES_PER_CLUSTER = 14.7
# the neighbour stage alone: binned (y, z) read (8), the two choices (8) and
# D^2 (4) written
NB_BYTES_PER_CLUSTER = 20.0
FIT_BYTES_PER_HIT = 14.0                # hit index (4) + y, z (8) + row (2)
FIT_BYTES_PER_TRACK = 88.0              # 5 params + 15 cov + chi2 + ndf

def kf_ops_per_step():
    """Arithmetic operations of one Kalman step (transport, covariance
    transport, update, chi2) as counted by the FP64 oracle over the central
    event's truth tracks; stored in tests/golden/kf_ops_per_step.json by
    tests/golden/make_kf_ops.py."""
    with open(os.path.join(ROOT, "tests", "golden", "kf_ops_per_step.json")) as f:
        return float(json.load(f)["ops_per_step"])


def fp32_peak_tflops(torch, dev, sm_max_mhz):
    """FP32 issue peak: SMs (queried) x 128 lanes x 2 (FMA) x max SM clock."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return sms * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12, sms
# DRAM bytes (read + write) of one build launch of k_tracklet_lanes on the
# central event, from an ncu capture of this kernel (dram__bytes_read.sum +
# dram__bytes_write.sum); None for a kernel without a capture
TRAFFIC_BYTES_PER_LAUNCH = {"k_tracklet_lanes": 38.144e6 + 2.447e6, "k_fit": 23.837e6}


def batched_vs_plain(torch, tpc, dev, steps):
    """512 events of log-uniform multiplicity (10..1e4 tracks, noise 5-30%):
    the whole batch as one autotuned call captured in the library's CUDA
    graph (tpc_graph_capture / tpc_graph_launch) vs the plain path (one load
    + find + fit per event).  Both give identical tracks."""
    from paper_2412_13755_gb300 import synth
    t0 = time.perf_counter()
    ev = synth.uneven_batch_parallel()
    gen_s = time.perf_counter() - t0
    n, E = ev.n, ev.n_events
    off = ev.evt_sector_off
    y = torch.from_numpy(ev.y).to(dev)
    z = torch.from_numpy(ev.z).to(dev)
    row = torch.from_numpy(ev.row.view(np.int16)).to(dev).view(torch.uint16)
    d_off = torch.from_numpy(off).to(dev)
    cap = n // 10 + 16
    # batched: one context over all events
    trb = tpc.Tracker(n, E, device=dev)
    outb = (torch.empty(n, dtype=torch.int32, device=dev), torch.empty(cap + 1, dtype=torch.int32, device=dev),
            torch.empty(n, dtype=torch.int32, device=dev), torch.empty(1, dtype=torch.int32, device=dev))
    fitb = (torch.empty(cap, 5, dtype=torch.float32, device=dev), torch.empty(cap, 15, dtype=torch.float32, device=dev),
            torch.empty(cap, dtype=torch.float32, device=dev), torch.empty(cap, dtype=torch.int32, device=dev))
    trb.load(y, z, row, d_off, E)
    tune = trb.autotune(out=outb)
    # the library's own graph of the whole batch call (load, find, fit)
    trb.capture(y, z, row, d_off, E, outb, fitb)
    l0 = trb.stats().n_launches
    trb.replay()
    torch.cuda.synchronize()
    graph_kernels = int(trb.stats().n_launches - l0)  # kernels of one replay
    stb = trb.check()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        trb.replay()
    e1.record()
    torch.cuda.synchronize()
    batched_s = e0.elapsed_time(e1) / 1e3 / steps
    # plain: one context sized for the largest event, one call sequence per event
    sizes = off[36::36] - off[0:-1:36]
    nmax = int(sizes.max())
    trp = tpc.Tracker(nmax, 1, device=dev)
    capp = nmax // 10 + 16
    outp = (torch.empty(nmax, dtype=torch.int32, device=dev), torch.empty(capp + 1, dtype=torch.int32, device=dev),
            torch.empty(nmax, dtype=torch.int32, device=dev), torch.empty(1, dtype=torch.int32, device=dev))
    fitp = (torch.empty(capp, 5, dtype=torch.float32, device=dev), torch.empty(capp, 15, dtype=torch.float32, device=dev),
            torch.empty(capp, dtype=torch.float32, device=dev), torch.empty(capp, dtype=torch.int32, device=dev))
    ev_offs = [d_off[36 * e:36 * e + 37] - int(off[36 * e]) for e in range(E)]
    starts = [int(off[36 * e]) for e in range(E)]
    plain_toc = torch.empty(n, dtype=torch.int32, device=dev)

    def step_p(record=False):
        for e in range(E):
            b, m = starts[e], int(sizes[e])
            trp.load(y[b:b + m], z[b:b + m], row[b:b + m], ev_offs[e], 1)
            trp.find(out=outp)
            trp.fit(outp[1], outp[2], capp, outp[3], out=fitp)
            if record:
                plain_toc[b:b + m] = outp[0][:m]

    step_p(record=True)
    torch.cuda.synchronize()
    trp.check()
    # equal accuracy: per event, the plain track ids equal the batched ones
    # shifted by the number of batched tracks of earlier events
    bt = outb[0]
    first = torch.full((E,), 0, dtype=torch.int32, device=dev)
    for e in range(E):
        b, m = starts[e], int(sizes[e])
        seg = bt[b:b + m]
        first[e] = seg[seg >= 0].min() if bool((seg >= 0).any()) else 0
    ev_of = torch.repeat_interleave(torch.arange(E, device=dev), torch.from_numpy(sizes).to(dev))
    shifted = torch.where(bt >= 0, bt - first[ev_of], bt)
    identical = bool(torch.equal(shifted, plain_toc))
    e0.record()
    for _ in range(steps):
        step_p()
    e1.record()
    torch.cuda.synchronize()
    plain_s = e0.elapsed_time(e1) / 1e3 / steps
    return {
        "workload": f"uneven_batch: {E} events, log-uniform 10..1e4 tracks, noise U[5%,30%], {n} clusters",
        "batched_clusters_per_s": n / batched_s, "plain_clusters_per_s": n / plain_s,
        "speedup": plain_s / batched_s, "batched_ms": 1e3 * batched_s, "plain_ms": 1e3 * plain_s,
        "identical_tracks": identical, "tracks": int(stb.n_tracks),
        "tune": {"lane_blocks_per_sm": tune.lane_blocks_per_sm, "lane_tile": tune.lane_tile,
                 "nb_sub_lanes": tune.nb_sub_lanes},
        "graph_kernels_per_step": graph_kernels, "generation_s": gen_s,
        "inputs_vs_l2": "1.5 GB of inputs, larger than L2 (no flush needed)",
    }


def adjoint_bench(torch, tpc, dev, steps):
    """Alignment sample: 2e5 tracks pT > 1 GeV/c; chi2 + gradient per step."""
    from paper_2412_13755_gb300 import synth
    ev = synth.alignment_sample_parallel()
    off_h, hits_h, _ = ev.truth_tracks(n_min=10)
    T = len(off_h) - 1
    tr = tpc.Tracker(ev.n, 1, device=dev)
    y = torch.from_numpy(ev.y).to(dev)
    z = torch.from_numpy(ev.z).to(dev)
    row = torch.from_numpy(ev.row.view(np.int16)).to(dev).view(torch.uint16)
    d_off = torch.from_numpy(ev.evt_sector_off).to(dev)
    tr.load(y, z, row, d_off, 1)
    trk_off = torch.from_numpy(off_h).to(dev)
    trk_hits = torch.from_numpy(hits_h).to(dev)
    align = torch.from_numpy(0.5 * ev.align).to(dev)
    for _ in range(2):
        tr.adjoint(trk_off, trk_hits, T, align)
    torch.cuda.synchronize()
    tr.check()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        chi2, grad = tr.adjoint(trk_off, trk_hits, T, align)
    e1.record()
    torch.cuda.synchronize()
    s_grad = e0.elapsed_time(e1) / 1e3 / steps
    e0.record()
    for _ in range(steps):
        tr.adjoint(trk_off, trk_hits, T, align, want_grad=False)
    e1.record()
    torch.cuda.synchronize()
    s_fwd = e0.elapsed_time(e1) / 1e3 / steps
    # lower-bound roofline: the two forward Kalman sweeps per cluster (the
    # checkpointing pass and the recompute of each segment) at the oracle's
    # counted operations per step; the reverse step's own operations have
    # no independent count and are left out
    n_hits = int(off_h[-1])
    ops = kf_ops_per_step()
    peak_tf, sms = fp32_peak_tflops(torch, dev, measured_sm_max_mhz())
    ach = 2 * n_hits * ops / s_grad / 1e12
    return {"workload": f"alignment_sample: {T} tracks pT>1 GeV/c, {ev.n} clusters, 216 parameters",
            "tracks_per_s": T / s_grad, "forward_only_tracks_per_s": T / s_fwd,
            "ms_per_step": 1e3 * s_grad, "chi2": float(chi2.item()),
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak_tf, "unit": "TFLOP/s",
                         "frac": ach / peak_tf, "kernel": "k_adjoint",
                         "work": f"2 forward Kalman steps per cluster x {ops:.1f} counted operations "
                                 "(the reverse step not counted: a lower bound)"}}


def pileup_bench(torch, tpc, dev, steps):
    """50 kHz frame: 100 central-like collisions over 2 ms, one event, one
    pass (find + fit)."""
    from paper_2412_13755_gb300 import synth
    t0 = time.perf_counter()
    ev = synth.pileup_frame_parallel()
    gen_s = time.perf_counter() - t0
    n = ev.n
    cap = n // 10 + 16
    tr = tpc.Tracker(n, 1, device=dev)
    y = torch.from_numpy(ev.y).to(dev)
    z = torch.from_numpy(ev.z).to(dev)
    row = torch.from_numpy(ev.row.view(np.int16)).to(dev).view(torch.uint16)
    d_off = torch.from_numpy(ev.evt_sector_off).to(dev)
    tr.load(y, z, row, d_off, 1)
    out = tr.alloc_find_outputs(cap)
    fit = (torch.empty(cap, 5, dtype=torch.float32, device=dev), torch.empty(cap, 15, dtype=torch.float32, device=dev),
           torch.empty(cap, dtype=torch.float32, device=dev), torch.empty(cap, dtype=torch.int32, device=dev))

    def step():
        tr.load(y, z, row, d_off, 1)
        tr.find(out=out)
        tr.fit(out[1], out[2], cap, out[3], out=fit)

    step()
    torch.cuda.synchronize()
    st = tr.check()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3 / steps
    return {"workload": f"pileup_frame: 100 collisions x 1e4 tracks over 2 ms, {n} clusters, one event",
            "clusters_per_s": n / sec, "ms_per_step": 1e3 * sec, "tracks": int(st.n_tracks),
            "workspace_gb": tr.workspace.numel() / 1e9, "generation_s": gen_s}


def kf_variants_bench(torch, tpc, dev, steps):
    """NEXT-3: the Kalman-filter variants on 2e4 pions through material (one
    sector, material in every pad-row plane): the inward fit with material,
    the outward refit and the fit with the Rauch-Tung-Striebel smoother,
    FP64 per track (tpc_fit_tracks_ex)."""
    from paper_2412_13755_gb300 import synth
    ev = synth.material_tracks(n_tracks=20000)
    off_h, hits_h, _ = ev.truth_tracks(n_min=10)
    T = len(off_h) - 1
    tr = tpc.Tracker(ev.n, 1, device=dev)
    y = torch.from_numpy(ev.y).to(dev)
    z = torch.from_numpy(ev.z).to(dev)
    row = torch.from_numpy(ev.row.view(np.int16)).to(dev).view(torch.uint16)
    d_off = torch.from_numpy(ev.evt_sector_off).to(dev)
    tr.load(y, z, row, d_off, 1)
    trk_off = torch.from_numpy(off_h).to(dev)
    trk_hits = torch.from_numpy(hits_h).to(dev)
    out = {}
    for name, outward, smooth in (("material_fit", False, False), ("outward_refit", True, False),
                                  ("fit_and_smoother", False, True)):
        o = tpc.fit_options(synth.MAT_X_X0_ROW, synth.MAT_ELOSS_ROW, synth.PION_MASS, outward=outward)
        tr.fit_ex(trk_off, trk_hits, T, o, smooth=smooth)
        torch.cuda.synchronize()
        tr.check()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            tr.fit_ex(trk_off, trk_hits, T, o, smooth=smooth)
        e1.record()
        torch.cuda.synchronize()
        out[name] = {"tracks_per_s": T * steps / (e0.elapsed_time(e1) / 1e3),
                     "ms_per_step": e0.elapsed_time(e1) / steps}
    # FP64 roofline of the material fit: the oracle's counted operations per
    # cluster through material (tests/golden/kf_ops_per_step.json) against
    # the nominal FP64 rate (no FP64 figure is measured on this machine)
    with open(os.path.join(ROOT, "tests", "golden", "kf_ops_per_step.json")) as f:
        ops_hit = float(json.load(f)["material"]["ops_per_hit"])
    ach = int(off_h[-1]) * ops_hit / (out["material_fit"]["ms_per_step"] * 1e-3) / 1e12
    out["roofline"] = {"bound": "fp64", "achieved": ach, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                       "frac": ach / FP64_NOMINAL_TFLOPS, "kernel": "k_fit_ex (material fit)",
                       "peak_source": "nominal GB300 FP64 (not measured)", "ops_per_hit": ops_hit}
    out["workload"] = f"material_tracks: {T} pions pT > 0.3 GeV/c in one sector, {int(off_h[-1])} clusters"
    return out


def sides_bench(torch, tpc, dev, steps):
    """NEXT-4: a 20-collision frame with a vertex z spread (sigma 6 cm),
    found once; the timed step is the A/C-side association with t0 over all
    found tracks (tpc_match_sides), candidates, end fits and joint fits."""
    from paper_2412_13755_gb300 import synth
    t0 = time.perf_counter()
    ev = synth.membrane_frame_parallel(n_collisions=20)
    gen_s = time.perf_counter() - t0
    n = ev.n
    cap = n // 10 + 16
    tr = tpc.Tracker(n, 1, device=dev)
    y = torch.from_numpy(ev.y).to(dev)
    z = torch.from_numpy(ev.z).to(dev)
    row = torch.from_numpy(ev.row.view(np.int16)).to(dev).view(torch.uint16)
    d_off = torch.from_numpy(ev.evt_sector_off).to(dev)
    tr.load(y, z, row, d_off, 1)
    out = tr.alloc_find_outputs(cap)
    tr.find(out=out)
    torch.cuda.synchronize()
    tr.check()
    T = int(out[3].item())
    r = tr.match_sides(out[1], out[2], T)
    torch.cuda.synchronize()
    tr.check()
    pairs = int(r["n_pairs"].item())
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        r = tr.match_sides(out[1], out[2], T)
    e1.record()
    torch.cuda.synchronize()
    tr.check()
    sec = e0.elapsed_time(e1) / 1e3 / steps
    p = r["partner"][:T]
    sel = torch.nonzero(p >= 0).flatten()
    sig = torch.sqrt(r["cov6"][sel, 20])
    return {"workload": f"membrane_frame: 20 collisions x 1e4 tracks over 2 ms, vertex z sigma 6 cm, {n} clusters, "
                        f"{T} found tracks", "tracks_per_s": T / sec, "ms_per_step": 1e3 * sec, "pairs": pairs,
            "t0_sigma_median_us": float(sig.median().item()) if len(sel) else None, "generation_s": gen_s}


def field_adjoint_bench(torch, tpc, dev, steps):
    """NEXT-1: chi2 and its gradient with respect to the voxel displacement
    field (36 x 160 voxels x 3) plus the alignment, on 2e5 pT > 1 GeV/c
    tracks, at a drawn field (sigma 0.5 mm) added to every cluster in the
    fit: tracks/s, forward + reverse sweep."""
    from paper_2412_13755_gb300 import synth
    grid = synth.FIELD_GRID
    F = synth.draw_field(seed=synth.SEED_BASE + 5, sigma=0.05)
    units = [(0, 5000, 0.0)] * 40
    ev = synth.generate_parallel(units, synth.SEED_BASE + 5, pt_min=1.0, pt_slope=0.5, misalign=None)
    off_h, hits_h, _ = ev.truth_tracks(n_min=10)
    T = len(off_h) - 1
    tr = tpc.Tracker(ev.n, 1, device=dev)
    y = torch.from_numpy(ev.y).to(dev)
    z = torch.from_numpy(ev.z).to(dev)
    row = torch.from_numpy(ev.row.view(np.int16)).to(dev).view(torch.uint16)
    d_off = torch.from_numpy(ev.evt_sector_off).to(dev)
    tr.load(y, z, row, d_off, 1)
    trk_off, trk_hits = torch.from_numpy(off_h).to(dev), torch.from_numpy(hits_h).to(dev)
    g = tpc.field_grid(**grid)
    field = torch.from_numpy(F).to(dev)
    for _ in range(2):
        tr.adjoint_field(trk_off, trk_hits, T, g, field)
    torch.cuda.synchronize()
    tr.check()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        tr.adjoint_field(trk_off, trk_hits, T, g, field)
    e1.record()
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3 / steps
    # lower-bound roofline as for the alignment adjoint
    ops = kf_ops_per_step()
    peak_tf, _ = fp32_peak_tflops(torch, dev, measured_sm_max_mhz())
    ach = 2 * int(trk_off[-1].item()) * ops / sec / 1e12
    return {"workload": f"distortion map: {T} tracks pT>1 GeV/c, {ev.n} clusters, "
                        f"{synth.n_voxels(grid)} voxels x 3 + 216 alignment parameters",
            "tracks_per_s": T / sec, "ms_per_step": 1e3 * sec,
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak_tf, "unit": "TFLOP/s",
                         "frac": ach / peak_tf, "kernel": "k_adjoint<true>",
                         "work": f"2 forward Kalman steps per cluster x {ops:.1f} counted operations "
                                 "(the reverse step not counted: a lower bound)"}}


def fit_precision_bench(torch, tr, find_out, track_cap, dev, steps):
    """The central event's found tracks fitted by the two precision modes of
    the fit: float-float covariance (tpc_fit_tracks, the path's fit) and FP32
    covariance with FP64 redos of cancelling updates (tpc_fit_tracks_fp32);
    CUDA events around each launch, after warm-up."""
    T = int(find_out[3].item())
    out = (torch.empty(max(T, 1), 5, dtype=torch.float32, device=dev),
           torch.empty(max(T, 1), 15, dtype=torch.float32, device=dev),
           torch.empty(max(T, 1), dtype=torch.float32, device=dev),
           torch.empty(max(T, 1), dtype=torch.int32, device=dev))
    res = {"tracks": T}
    for name, prec in (("float_float_ms", "ff"), ("fp32_fp64_redo_ms", "fp32")):
        for _ in range(3):
            tr.fit(find_out[1], find_out[2], T, out=out, precision=prec)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            tr.fit(find_out[1], find_out[2], T, out=out, precision=prec)
        e1.record()
        torch.cuda.synchronize()
        res[name] = e0.elapsed_time(e1) / steps
    tr.check()
    res["parity_bars"] = "float-float: 1e-5 of the FP64 oracle; FP32 with FP64 redos: 1e-4 (tests/test_gpu_parity.py)"
    return res


def clusterize_bench(torch, tpc, dev, steps, ev):
    """NEXT-2: clusterization of the central event's pad-time digits
    (36 x 152 planes x 512 time bins x 160 pads, u16: 0.9 GB, larger than
    L2): digits/s and the HBM fraction of the clusterizer kernel, whose
    algorithmic bytes are the digits read once plus 12 B per cluster
    written (y, z, row, charge)."""
    from paper_2412_13755_gb300 import synth
    d = synth.digitize(ev)
    d_dev = torch.from_numpy(d.view(np.int16)).to(dev).view(torch.uint16)
    cap = int(np.count_nonzero(d))
    cl = tpc.Clusterizer(1, d.shape[1], cap, device=dev)
    for _ in range(3):
        out = cl.run(d_dev)
    torch.cuda.synchronize()
    st = out[6].cpu().numpy()
    if st[0] != 0:
        raise RuntimeError(f"clusterizer status {st}")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        cl.run(d_dev)
    e1.record()
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3 / steps
    n_cl = int(out[5].item())
    algo = d.nbytes + 12 * n_cl
    hbm_peak, src = measured_peaks()
    return {"workload": f"central_event digits: {d.shape[0]} planes x {d.shape[1]} time bins x {d.shape[2]} pads "
                        f"(u16, {d.nbytes / 1e9:.2f} GB), {n_cl} clusters",
            "digits_per_s": d.size / sec, "clusters_per_s": n_cl / sec, "ms_per_step": 1e3 * sec,
            "roofline": {"bound": "hbm", "achieved": algo / sec / 1e9, "peak": hbm_peak, "unit": "GB/s",
                         "frac": algo / sec / 1e9 / hbm_peak, "algorithmic_bytes": algo,
                         "peak_source": src + " (MEASURED_PEAKS.json hbm_gbs)"},
            "inputs_vs_l2": "0.9 GB of digits, larger than L2 (no flush needed)"}


EXTRA_NAMES = ("batched_vs_plain", "adjoint", "clusterize", "field_adjoint", "kf_variants", "sides",
               "pileup_frame", "fit_precision")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-profiler", action="store_true", help="(kept for compatibility)")
    ap.add_argument("--pileup", action="store_true",
                    help="(kept for compatibility: the pile-up frame is timed by default)")
    ap.add_argument("--no-pileup", action="store_true",
                    help="skip the 100-collision pile-up frame (~1.8e8 clusters)")
    ap.add_argument("--tune", default="",
                    help="LANE_BLOCKS_PER_SM,LANE_TILE,NB_SUB_LANES: use this tuning of the central "
                         "event instead of autotuning it (for profiler runs)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched-vs-plain and adjoint measurements")
    ap.add_argument("--only", choices=sorted(EXTRA_NAMES),
                    help="run one of the extra measurements alone and print its JSON (for profiling)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, dist, device):
    """The largest of the ranks' values of x (the job's time is its slowest
    rank's); x itself when there is one rank."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(units_per_rank, world, steps, total_s):
    """Whole-job throughput: the units every rank processed over the
    slowest rank's time (weak scaling: per-rank work is fixed)."""
    return units_per_rank * world * steps / total_s


def rank_seed_offset(rank):
    """Each rank tracks its own event (seed offset = rank)."""
    return rank


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ----------------------------------------------------------------- clocks --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def wait_first(self, timeout_s=3.0):
        """Blocks until the sampler has written its first line (or gives up),
        so that the samples that follow cover the timed region."""
        t0 = time.perf_counter()
        while self.proc is not None and time.perf_counter() - t0 < timeout_s:
            try:
                if os.path.getsize(self.path) > 0:
                    return
            except OSError:
                return
            time.sleep(0.01)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm, mx, reasons = [], [], set()
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                    "sw_power_cap"), f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- workload --
def make_event(seed_offset=0):
    from paper_2412_13755_gb300 import synth
    return synth.central_event(seed=synth.SEED_BASE + 1 + seed_offset)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def measured_sm_max_mhz():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"])
    except (OSError, KeyError, ValueError):
        return 2070.0


def cpu_baseline(ev, target_s=12.0):
    """The oracle, as it stands, on the host cores: find + fit of the event."""
    import oracle
    cores = host_cores()
    oracle.set_threads(cores)
    sec = ev.sector_of_cluster()
    done, t0 = 0, time.perf_counter()
    while True:
        toc, off, hits = oracle.find_tracks(ev.y, ev.z, ev.row, ev.evt_sector_off, ev.n_events)
        oracle.fit_tracks(ev.y, ev.z, ev.row, sec, off, hits)
        done += 1
        el = time.perf_counter() - t0
        if el >= target_s:
            break
    return {"value": done * ev.n / el, "unit": "clusters/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} x the full central event ({ev.n} clusters), find + FP64 fit, "
                      f"OpenMP over groups/tracks, {el:.1f} s"}


# -------------------------------------------------------------- reference --
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    ev = make_event()
    cores = host_cores()
    oracle.set_threads(cores)
    sec = ev.sector_of_cluster()

    def step():
        toc, off, hits = oracle.find_tracks(ev.y, ev.z, ev.row, ev.evt_sector_off, ev.n_events)
        oracle.fit_tracks(ev.y, ev.z, ev.row, sec, off, hits)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    v = args.steps * ev.n / el
    line = {"metric": METRIC, "value": v, "unit": "clusters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": "clusters/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} x the full central event ({ev.n} clusters), "
                                       f"find + FP64 fit"},
            "e2e": {"value": v, "unit": "clusters/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------- ours --
def run_ours(args):
    import torch

    from paper_2412_13755_gb300 import tpc

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    ev = make_event(seed_offset=rank_seed_offset(rank))
    n = ev.n
    track_cap = 32768
    tr = tpc.Tracker(n, 1, device=dev)
    stream = torch.cuda.current_stream(dev)

    # host (pinned) and device copies of the inputs
    h_y = torch.from_numpy(ev.y).pin_memory()
    h_z = torch.from_numpy(ev.z).pin_memory()
    h_row = torch.from_numpy(ev.row.view(np.int16)).pin_memory()
    h_off = torch.from_numpy(ev.evt_sector_off).pin_memory()
    d_y, d_z = h_y.to(dev), h_z.to(dev)
    d_row = h_row.to(dev).view(torch.uint16)
    d_off = h_off.to(dev)
    find_out = (torch.empty(n, dtype=torch.int32, device=dev),
                torch.empty(track_cap + 1, dtype=torch.int32, device=dev),
                torch.empty(n, dtype=torch.int32, device=dev),
                torch.empty(1, dtype=torch.int32, device=dev))
    fit_out = (torch.empty(track_cap, 5, dtype=torch.float32, device=dev),
               torch.empty(track_cap, 15, dtype=torch.float32, device=dev),
               torch.empty(track_cap, dtype=torch.float32, device=dev),
               torch.empty(track_cap, dtype=torch.int32, device=dev))
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def step(y=d_y, z=d_z, row=d_row, off=d_off):
        tr.load(y, z, row, off, 1)
        tr.find(out=find_out)
        tr.fit(find_out[1], find_out[2], track_cap, find_out[3], out=fit_out)

    sync = torch.cuda.synchronize
    # clocks: sampled from the warm-up through the timed steps
    clocks = ClockSampler(local)
    clocks.start()
    clocks.wait_first()
    step()
    sync()
    # the work-queue tiles tuned on this event, then the whole step (load,
    # find, fit) recorded once as the library's CUDA graph: the timed steps
    # replay it, as a server does for every event of a fixed-size stream
    if args.tune:
        # a fixed tuning (for profiler runs, where the autotuner's timings
        # would be those of the profiler)
        lb, tile, nb = (int(v) for v in args.tune.split(","))
        tune = tpc.Tune()
        tune.lane_blocks_per_sm, tune.lane_tile, tune.nb_sub_lanes = lb, tile, nb
        tr.set_tune(tune)
    else:
        tune = tr.autotune(out=find_out)
    # stage events on at capture: they become event nodes of the graph, so
    # each timed replay carries its own stage times
    tr.stage_timing(True)
    tr.capture(d_y, d_z, d_row, d_off, 1, find_out, fit_out)
    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        tr.replay()
    sync()
    st = tr.check()
    l0 = tr.stats().n_launches
    tr.replay()
    sync()
    launches_per_step = tr.stats().n_launches - l0
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    sync()
    stage_sum = {}
    for k in range(args.steps):
        flush.zero_()
        e0[k].record(stream)
        tr.replay()
        e1[k].record(stream)
        sync()
        for name, ms in tr.stage_times().items():
            stage_sum[name] = stage_sum.get(name, 0.0) + ms
    sync()
    step_ms = [a.elapsed_time(b) for a, b in zip(e0, e1)]
    total_s = max_over_ranks(sum(step_ms) / 1e3, dist if world > 1 else None, dev)
    st = tr.check()
    T = int(find_out[3].item())
    value = weak_value(n, world, args.steps, total_s)
    # the same step through the per-call entry points (load, find, fit as
    # three calls)
    plain_ms = []
    for k in range(args.steps):
        flush.zero_()
        e0[k].record(stream)
        step()
        e1[k].record(stream)
        sync()
        plain_ms.append(e0[k].elapsed_time(e1[k]))
    sync()
    clk = clocks.stop()
    tr.stage_timing(False)
    if int(find_out[3].item()) != T:
        raise RuntimeError("the per-call step found a different number of tracks than the graph replay")

    # end to end: host buffers -> device, step, results back to the host.
    # Steps are pipelined as for a stream of events: while a step computes,
    # a copy stream uploads the next step's inputs and downloads the previous
    # step's results (two buffer sets, ordered by events); each set's step
    # is the library graph of load + find + fit over that set's buffers.
    main_s = torch.cuda.current_stream(dev)
    copy_s = torch.cuda.Stream(device=dev)

    def buffer_set():
        b = {
            "y": torch.empty_like(d_y), "z": torch.empty_like(d_z),
            "row": torch.empty(n, dtype=torch.int16, device=dev), "off": torch.empty_like(d_off),
            "find": tuple(torch.empty_like(t) for t in find_out),
            "fit": tuple(torch.empty_like(t) for t in fit_out),
            "h_toc": torch.empty(n, dtype=torch.int32).pin_memory(),
            "h_par": torch.empty(track_cap, 5, dtype=torch.float32).pin_memory(),
            "h_chi2": torch.empty(track_cap, dtype=torch.float32).pin_memory(),
            "h_nt": torch.empty(1, dtype=torch.int32).pin_memory(),
            "in": torch.cuda.Event(), "done": torch.cuda.Event(), "out": torch.cuda.Event(),
        }
        # each buffer set has its own context holding the graph of the step
        # over that set's buffers (the same call a server replays per event)
        b["tr"] = tpc.Tracker(n, 1, device=dev)
        b["y"].copy_(d_y)
        b["z"].copy_(d_z)
        b["row"].copy_(d_row.view(torch.int16))
        b["off"].copy_(d_off)
        b["tr"].load(b["y"], b["z"], b["row"].view(torch.uint16), b["off"], 1)
        b["tr"].set_tune(tune)
        b["tr"].capture(b["y"], b["z"], b["row"].view(torch.uint16), b["off"], 1, b["find"], b["fit"])
        return b

    sets = [buffer_set(), buffer_set()]

    def upload(b):
        with torch.cuda.stream(copy_s):
            copy_s.wait_event(b["done"])  # the inputs' previous step has finished
            b["y"].copy_(h_y, non_blocking=True)
            b["z"].copy_(h_z, non_blocking=True)
            b["row"].copy_(h_row, non_blocking=True)
            b["off"].copy_(h_off, non_blocking=True)
            b["in"].record(copy_s)

    def compute(b):
        main_s.wait_event(b["in"])
        main_s.wait_event(b["out"])  # the outputs' previous download has finished
        b["tr"].replay(stream=main_s)
        b["done"].record(main_s)

    def download(b):
        with torch.cuda.stream(copy_s):
            copy_s.wait_event(b["done"])
            b["h_toc"].copy_(b["find"][0], non_blocking=True)
            b["h_nt"].copy_(b["find"][3], non_blocking=True)
            b["h_par"].copy_(b["fit"][0], non_blocking=True)
            b["h_chi2"].copy_(b["fit"][2], non_blocking=True)
            b["out"].record(copy_s)

    def e2e_run(k_steps, flushes):
        upload(sets[0])
        for k in range(k_steps):
            b = sets[k % 2]
            if flushes:
                flush.zero_()
            compute(b)
            if k + 1 < k_steps:
                upload(sets[(k + 1) % 2])
            download(b)
        sync()

    e2e_run(3, False)
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    e2e_run(args.steps, True)
    e2e_s = time.perf_counter() - t0
    # the flushes are outside the metric: time them alone and subtract
    t1 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
    sync()
    e2e_s = max(e2e_s - (time.perf_counter() - t1), 1e-9)
    e2e_s = max_over_ranks(e2e_s, dist if world > 1 else None, dev)
    # the last step's results as read on the host agree with the device
    last = sets[(args.steps - 1) % 2]
    if int(last["h_nt"][0]) != T:
        raise RuntimeError("end-to-end results differ from the device-resident run")
    h2d = 4 * n + 4 * n + 2 * n + 8 * ev.evt_sector_off.size
    d2h = 4 * n + 4 + 20 * track_cap + 4 * track_cap

    # roofline of the dominant kernel: the longest launch among the stages
    # that are one kernel each (the tracklet build, the fit); the neighbour
    # stage is three kernels (first pass, later gap pairs, overflow)
    per_step = {k: v / args.steps for k, v in stage_sum.items()}
    hits_total = int(find_out[1][T].item()) if T > 0 else 0
    kernels = {
        "k_tracklet_lanes": per_step.get("tracklets", 0.0),
        "k_fit": per_step.get("fit", 0.0),
    }
    dom = max(kernels, key=kernels.get)
    hbm_peak, peak_src = measured_peaks()
    ms = kernels[dom]
    # Kalman kernels are FP32-ALU work: counted steps x operations per step
    work_steps = st.n_kf_steps if dom == "k_tracklet_lanes" else hits_total
    ops_step = kf_ops_per_step()
    sm_max = clk.get("sm_max_mhz") or measured_sm_max_mhz()
    peak_tf, sms = fp32_peak_tflops(torch, dev, sm_max)
    achieved = work_steps * ops_step / (ms * 1e-3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_tf,
            "unit": "TFLOP/s", "frac": achieved / peak_tf,
            "traffic": TRAFFIC_BYTES_PER_LAUNCH.get(dom), "kf_steps_per_launch": int(work_steps),
            "ops_per_kf_step": ops_step, "kernel": dom, "kernel_ms": ms,
            "peak_source": f"derived: {sms} SMs (queried) x {FP32_LANES_PER_SM} FP32 lanes x 2 (FMA) x "
                           f"{sm_max:.0f} MHz (max SM clock)"}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": "clusters/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "events_per_gpu": 1, "clusters_per_gpu": n,
                   "tracks_found": T, "l2": "flushed between timed steps (512 MB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "tracks_per_s": T * world * args.steps / total_s,
        "timed_step": "replay of the library's CUDA graph of load + find + fit (tpc_graph_capture, "
                      "tpc_graph_launch), work queues autotuned on this event",
        "tune": {"lane_blocks_per_sm": tune.lane_blocks_per_sm, "lane_tile": tune.lane_tile,
                 "nb_sub_lanes": tune.nb_sub_lanes},
        "per_call_ms_per_step": sum(plain_ms) / len(plain_ms),
        "stage_ms_per_step": per_step,
        "e2e": {"value": weak_value(n, world, args.steps, e2e_s), "unit": "clusters/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "roofline": roof,
        "path_roofline": {"bound": "hbm", "bytes_per_cluster": PATH_BYTES_PER_CLUSTER,
                          "achieved": value * PATH_BYTES_PER_CLUSTER / 1e9, "peak": hbm_peak,
                          "unit": "GB/s", "frac": value * PATH_BYTES_PER_CLUSTER / 1e9 / hbm_peak,
                          "fused_bytes_per_cluster": PATH_FUSED_BYTES_PER_CLUSTER,
                          "fused_frac": value * PATH_FUSED_BYTES_PER_CLUSTER / 1e9 / hbm_peak,
                          "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)"},
        "neighbours_roofline": {
            "bound": "hbm", "bytes_per_cluster": NB_BYTES_PER_CLUSTER,
            "achieved": n * NB_BYTES_PER_CLUSTER / (per_step.get("neighbours", 0.0) * 1e-3) / 1e9
            if per_step.get("neighbours", 0.0) > 0 else None,
            "peak": hbm_peak, "unit": "GB/s",
            "frac": n * NB_BYTES_PER_CLUSTER / (per_step.get("neighbours", 0.0) * 1e-3) / 1e9 / hbm_peak
            if per_step.get("neighbours", 0.0) > 0 else None,
            "stage_ms": per_step.get("neighbours", 0.0),
            "kernels": "k_neighbours_first, k_neighbours_sub, k_neighbours_warp (one stage)"},
        "status": {"fp64_updates": st.n_fp64_updates, "segments": st.n_segments,
                   "tracklets": st.n_tracklets, "merges": st.n_merges},
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(ev)
    # the extra measurements run after the headline is complete; a failing
    # one is reported in its own field and does not discard the headline
    extras = []
    if not args.no_extras:
        extras += [("batched_vs_plain", lambda: batched_vs_plain(torch, tpc, dev, max(3, args.steps // 4))),
                   ("adjoint", lambda: adjoint_bench(torch, tpc, dev, max(3, args.steps // 4))),
                   ("clusterize", lambda: clusterize_bench(torch, tpc, dev, max(3, args.steps // 2), ev)),
                   ("field_adjoint", lambda: field_adjoint_bench(torch, tpc, dev, max(3, args.steps // 4))),
                   ("kf_variants", lambda: kf_variants_bench(torch, tpc, dev, max(3, args.steps // 4))),
                   ("sides", lambda: sides_bench(torch, tpc, dev, max(3, args.steps // 4))),
                   ("fit_precision", lambda: fit_precision_bench(torch, tr, find_out, track_cap, dev,
                                                                 max(3, args.steps // 2)))]
    if not args.no_extras and not args.no_pileup:
        extras.append(("pileup_frame", lambda: pileup_bench(torch, tpc, dev, 2)))
    for name, fn in extras:
        try:
            line[name] = fn()
        except Exception as ex:  # noqa: BLE001  (reported, the headline stands)
            line[name] = {"error": f"{type(ex).__name__}: {ex}"[:400]}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_only(args):
    import torch

    from paper_2412_13755_gb300 import tpc
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    k = max(3, args.steps // 4)
    fns = {"batched_vs_plain": lambda: batched_vs_plain(torch, tpc, dev, k),
           "adjoint": lambda: adjoint_bench(torch, tpc, dev, k),
           "clusterize": lambda: clusterize_bench(torch, tpc, dev, max(3, args.steps // 2), make_event()),
           "field_adjoint": lambda: field_adjoint_bench(torch, tpc, dev, k),
           "sides": lambda: sides_bench(torch, tpc, dev, k),
           "kf_variants": lambda: kf_variants_bench(torch, tpc, dev, k),
           "pileup_frame": lambda: pileup_bench(torch, tpc, dev, 2),
           "fit_precision": lambda: central_fit_precision(torch, tpc, dev, k)}
    print(json.dumps({args.only: fns[args.only]()}), flush=True)


def central_fit_precision(torch, tpc, dev, steps):
    """fit_precision on its own: the central event is found once, then its
    tracks are fitted by both precision modes."""
    ev = make_event()
    tr = tpc.Tracker(ev.n, 1, device=dev)
    y = torch.from_numpy(ev.y).to(dev)
    z = torch.from_numpy(ev.z).to(dev)
    row = torch.from_numpy(ev.row.view(np.int16)).to(dev).view(torch.uint16)
    off = torch.from_numpy(ev.evt_sector_off).to(dev)
    tr.load(y, z, row, off, 1)
    track_cap = 32768
    find_out = tr.alloc_find_outputs(track_cap)
    tr.find(out=find_out)
    return fit_precision_bench(torch, tr, find_out, track_cap, dev, steps)


def main():
    args = parse()
    if args.only:
        run_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
