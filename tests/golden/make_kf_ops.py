"""Writes kf_ops_per_step.json: the arithmetic work of one Kalman step of
the fit (helix transport with its Jacobian, covariance transport, 2-d
update and chi2), counted by the FP64 oracle over the truth tracks of the
seeded central event (1e4 tracks).  Structural zeros and ones of the
Jacobians are not counted.  The benchmark reads the number to express its
Kalman kernels' throughput in operations per second.  A second count, per
cluster, is the fit through material (every pad-row plane crossed with its
multiple-scattering noise and energy loss) on the seeded material sample,
for the Kalman-filter variants.

    python tests/golden/make_kf_ops.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "kf_ops_per_step.json")


MATERIAL_SAMPLE = dict(n_tracks=2000)  # synth.material_tracks defaults otherwise


def count_material():
    import numpy as np
    import oracle
    from paper_2412_13755_gb300 import synth
    ev = synth.material_tracks(**MATERIAL_SAMPLE)
    off, hits, _ = ev.truth_tracks(n_min=10)
    f32 = lambda v: float(np.float32(v))  # the library's options are FP32
    prm = oracle.default_params(mat_x_x0=f32(synth.MAT_X_X0_ROW), mat_eloss=f32(synth.MAT_ELOSS_ROW),
                                mass=f32(synth.PION_MASS))
    ops, steps = oracle.kf_ops(ev.y, ev.z, ev.row, ev.sector_of_cluster(), off, hits, params=prm)
    return {"ops": ops, "hits": steps, "ops_per_hit": ops / steps,
            "sample": "truth tracks (>= 10 clusters) of synth.material_tracks(n_tracks=2000), "
                      "material in every pad-row plane (x/X0 1e-4, energy loss 2e-6 GeV)"}


def count():
    import oracle
    from paper_2412_13755_gb300 import synth
    ev = synth.central_event(seed=synth.SEED_BASE + 1, noise=0.0)
    off, hits, _ = ev.truth_tracks()
    ops, steps = oracle.kf_ops(ev.y, ev.z, ev.row, ev.sector_of_cluster(), off, hits)
    return {"ops": ops, "steps": steps, "ops_per_step": ops / steps,
            "sample": "truth tracks (>= 10 clusters) of the seeded central event, 1e4 primaries, no noise",
            "counted": "+ - * / sqrt asin sin cos of the FP64 fit; operations on exact zeros and "
                       "multiplications by exact ones not counted",
            "material": count_material()}


if __name__ == "__main__":
    d = count()
    with open(OUT, "w") as f:
        json.dump(d, f, indent=1)
        f.write("\n")
    print(json.dumps(d))
