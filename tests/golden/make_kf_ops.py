"""Writes kf_ops_per_step.json: the arithmetic work of one Kalman step of
the fit (helix transport with its Jacobian, covariance transport, 2-d
update and chi2), counted by the FP64 oracle over the truth tracks of the
seeded central event (1e4 tracks).  Structural zeros and ones of the
Jacobians are not counted.  The benchmark reads the number to express its
Kalman kernels' throughput in operations per second.

    python tests/golden/make_kf_ops.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "kf_ops_per_step.json")


def count():
    import oracle
    from paper_2412_13755_gb300 import synth
    ev = synth.central_event(seed=synth.SEED_BASE + 1, noise=0.0)
    off, hits, _ = ev.truth_tracks()
    ops, steps = oracle.kf_ops(ev.y, ev.z, ev.row, ev.sector_of_cluster(), off, hits)
    return {"ops": ops, "steps": steps, "ops_per_step": ops / steps,
            "sample": "truth tracks (>= 10 clusters) of the seeded central event, 1e4 primaries, no noise",
            "counted": "+ - * / sqrt asin sin cos of the FP64 fit; operations on exact zeros and "
                       "multiplications by exact ones not counted"}


if __name__ == "__main__":
    d = count()
    with open(OUT, "w") as f:
        json.dump(d, f, indent=1)
        f.write("\n")
    print(json.dumps(d))
