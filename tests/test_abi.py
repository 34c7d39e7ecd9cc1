"""The C-ABI library loads on a machine without a GPU, exports every entry
point declared in include/*.h, and its host-only calls behave (defaults,
workspace sizing, argument errors).  No kernel is launched here."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(tpc_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    import torch  # noqa: F401  (loads the CUDA runtime the library links against)

    from paper_2412_13755_gb300 import tpc
    return tpc.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert {"tpc_load_clusters", "tpc_find_tracks", "tpc_fit_tracks", "tpc_fit_adjoint"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2412_13755_gb300 import tpc
    assert set(tpc.EXPORTS) == declared_functions()


def test_host_only_calls(lib):
    from paper_2412_13755_gb300 import tpc
    p = tpc.default_params()
    assert p.chi2_link == 16.0 and p.max_gap == 3 and p.n_min == 10
    ctx = tpc.tpc_create(p)
    try:
        small = tpc.tpc_workspace_bytes(ctx, 1000, 1)
        big = tpc.tpc_workspace_bytes(ctx, 2_000_000, 1)
        assert 0 < small < big
        assert tpc.tpc_workspace_bytes(ctx, 1000, 0) == 0
        # calls out of order are rejected without touching the device
        rc = lib.tpc_find_tracks(ctx, None, None, None, None, 0, None)
        assert rc == tpc.TPC_ERR_STATE
        rc = lib.tpc_load_clusters(ctx, None, None, None, None, 10, None, 1, None)
        assert rc == tpc.TPC_ERR_STATE
    finally:
        tpc.tpc_destroy(ctx)
    bad = tpc.default_params(max_gap=7)
    with pytest.raises(tpc.TPCError):
        tpc.tpc_create(bad)
    assert lib.tpc_create(None, None) == tpc.TPC_ERR_ARG


def test_struct_sizes_match_header(lib):
    from paper_2412_13755_gb300 import tpc
    # 5 floats, 5 int32, 2 floats, 2 floats, int32, float, 5 floats, 6 floats
    assert C.sizeof(tpc.Params) == 108
    assert C.sizeof(tpc.Stats) == 56
