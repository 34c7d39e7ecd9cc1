"""The stored Kalman-step work (tests/golden/kf_ops_per_step.json, read by
the benchmark) is what the oracle counts now, and the counter counts what it
claims on a case counted by hand: a straight track in a field-free frame,
where the transport's arcsine branch, the curvature terms and most Jacobian
entries are structural zeros and ones."""
import json
import os

import numpy as np
import pytest

from paper_2412_13755_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.slow
def test_stored_count_is_current(orc):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_kf_ops", os.path.join(HERE, "golden", "make_kf_ops.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    stored = json.load(open(os.path.join(HERE, "golden", "kf_ops_per_step.json")))
    now = m.count()
    assert now["ops"] == stored["ops"] and now["steps"] == stored["steps"]
    assert 150 < stored["ops_per_step"] < 450
    # through material every plane between two clusters is crossed too
    assert now["material"] == stored["material"]
    assert stored["material"]["ops_per_hit"] > stored["ops_per_step"]


def test_count_grows_linearly_with_the_steps(orc):
    """Every step of a track in one frame costs the same work once the
    state is away from the special values of the seed: the count of n + m
    steps minus that of n steps is m times the per-step count, and the
    field-free case costs less than the curved one (its curvature terms are
    zeros)."""
    rows = np.arange(20, 120).astype(np.uint16)
    x = synth.ROW_X[rows]
    y = (0.5 + 0.05 * (x - 85.0)).astype(np.float32)
    z = (3.0 + 0.4 * (x - 85.0)).astype(np.float32)
    sec = np.zeros(len(rows), np.int32)
    res = {}
    for bz in (0.5, 0.0):
        prm = orc.default_params(bz=bz)
        per = []
        for n in (40, 70, 100):
            hits = np.arange(len(rows) - 1, len(rows) - 1 - n, -1, dtype=np.int32)
            ops, steps = orc.kf_ops(y, z, rows, sec, np.array([0, n], np.int32), hits, params=prm)
            assert steps == n
            per.append(ops)
        assert per[2] - per[1] == per[1] - per[0]
        res[bz] = (per[2] - per[1]) / 30
    assert 0 < res[0.0] < res[0.5]
