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


def test_struct_sizes_match_header(lib, tmp_path):
    # the binding's ctypes structures against the C header, compiled here
    import shutil
    import subprocess
    from paper_2412_13755_gb300 import tpc
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include "tpc_track.h"\n'
                   'int main(void) { printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(tpc_params), sizeof(tpc_stats), '
                   'sizeof(tpc_tune), sizeof(tpc_field_grid), sizeof(tpc_fit_options), '
                   'sizeof(tpc_sides_options)); return 0; }\n')
    exe = tmp_path / "sizes"
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    sizes = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                            text=True).stdout.split()]
    assert sizes == [C.sizeof(tpc.Params), C.sizeof(tpc.Stats), C.sizeof(tpc.Tune),
                     C.sizeof(tpc.FieldGrid), C.sizeof(tpc.FitOptions), C.sizeof(tpc.SidesOptions)]


def test_field_voxels(lib):
    """The voxel count of a field grid, and the refusal of invalid grids (host
    only; tpc_fit_adjoint_field refuses the same grids with TPC_ERR_ARG)."""
    from paper_2412_13755_gb300 import synth, tpc
    assert tpc.tpc_field_voxels(tpc.field_grid(**synth.FIELD_GRID)) == synth.n_voxels()
    assert tpc.tpc_field_voxels(tpc.field_grid(1, 1, 1, 0, 1, 1)) == 36
    assert tpc.tpc_field_voxels(tpc.field_grid(152, 2, 3, 0, 1, 1)) == 36 * 152 * 6
    for bad in ((0, 1, 1), (5, 1, 1), (8, 0, 1), (8, 1, 0), (8, -3, 2), (152, 1 << 13, 1 << 13),
                (8, 1 << 26, 1)):
        assert tpc.tpc_field_voxels(tpc.field_grid(*bad, 0, 1, 1)) == -1, bad
    assert lib.tpc_field_voxels(None) == -1


def test_workspace_capacities_refused_on_the_host(lib):
    """Capacities whose 32-bit keys or indices would overflow are refused
    before any device memory is touched: the workspace size is 0 and
    tpc_set_workspace returns TPC_ERR_ARG (the buffer is never used)."""
    from paper_2412_13755_gb300 import tpc
    ctx = tpc.tpc_create()
    try:
        keys = lambda n, e: 152 * 16 * 36 * e + n + 16  # noqa: E731  (cell keys of the layout)
        lim = (1 << 31) - 1
        e_max = (lim - 2 - 16 - 1000) // (152 * 16 * 36)
        assert keys(1000, e_max) + 1 < lim <= keys(1000, e_max + 1) + 1
        assert tpc.tpc_workspace_bytes(ctx, 1000, e_max) > 0
        assert tpc.tpc_workspace_bytes(ctx, 1000, e_max + 1) == 0
        assert tpc.tpc_workspace_bytes(ctx, 1 << 30, 1) > 0
        assert tpc.tpc_workspace_bytes(ctx, (1 << 30) + 1, 1) == 0
        assert tpc.tpc_workspace_bytes(ctx, 1 << 30, 13000) == 0
        assert tpc.tpc_workspace_bytes(ctx, -1, 1) == 0
        fake = C.c_void_p(256)  # aligned, never dereferenced: refused first
        rc = lib.tpc_set_workspace(ctx, fake, C.c_size_t(1 << 62), C.c_int64(1000), C.c_int32(e_max + 1))
        assert rc == tpc.TPC_ERR_ARG
    finally:
        tpc.tpc_destroy(ctx)


def test_batch_calls_refused_without_device_work(lib):
    """Host-side refusals of the S7 calls and the tuning knobs: nothing is
    launched."""
    from paper_2412_13755_gb300 import tpc
    ctx = tpc.tpc_create(tpc.default_params())
    try:
        assert lib.tpc_graph_launch(ctx, None) == tpc.TPC_ERR_STATE
        out = tpc.BatchOutputs()
        assert lib.tpc_track_batch(ctx, None, None, None, None, 0, None, 1, C.byref(out), None) == \
            tpc.TPC_ERR_STATE
        for bad in ((0, 1, 8), (8, 0, 8), (8, 1, 5), (8, 1, 32), (17, 1, 8)):
            assert lib.tpc_set_tune(ctx, C.byref(tpc.Tune(*bad))) == tpc.TPC_ERR_ARG, bad
        for good in ((4, 1, 4), (16, 4, 16), (8, 1, 8)):
            assert lib.tpc_set_tune(ctx, C.byref(tpc.Tune(*good))) == tpc.TPC_OK
        assert lib.tpc_set_tune(ctx, None) == tpc.TPC_OK
    finally:
        tpc.tpc_destroy(ctx)


def test_match_sides_refused_without_device_work(lib):
    """Host-side refusals of tpc_match_sides (NEXT-4): nothing is launched."""
    from paper_2412_13755_gb300 import tpc
    assert lib.tpc_match_sides(None, None, None, 0, None, None, None, 0, 0, *([None] * 8), None) == tpc.TPC_ERR_ARG
    ctx = tpc.tpc_create(tpc.default_params())
    try:
        # no workspace, no clusters
        assert lib.tpc_match_sides(ctx, None, None, 0, None, None, None, 0, 0, *([None] * 8), None) == \
            tpc.TPC_ERR_STATE
    finally:
        tpc.tpc_destroy(ctx)
    assert tpc.tpc_sides_workspace_bytes(10, 1, 0) > 0
    assert tpc.tpc_sides_workspace_bytes(10, 1 << 17, 0) == 0
