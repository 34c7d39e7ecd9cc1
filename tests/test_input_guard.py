"""The device-side guard against invalid input, checked without a GPU.

The load's validation marks a rejected batch in its own status slot; every
kernel that reads clusters, their offsets or anything derived from them
must test that mark before its first access (find kernels return at once,
the fit reports failed fits, the adjoint returns).  Here the kernel sources
are read and each such kernel's body is checked to open with the guard, so
that a kernel added later without it fails on CPU.  The validation
decisions themselves are tested bit for bit on the host in
kernel_helpers_host.cpp."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2412_13755_gb300", "csrc")

# kernels that touch only buffers sized on the host (fills, scans, tables,
# the status copy) and the validation itself
UNGUARDED = {"k_fill_u64", "k_fill_u32", "k_fill_i32", "k_scan_reduce", "k_scan_top", "k_scan_down",
             "k_init_geo", "k_validate", "k_adj_tables", "k_zero_f64", "k_copy_status", "k_multi_fill"}


def kernels(path):
    text = open(path).read()
    for m in re.finditer(r"__global__\s+void\s+(?:__\w+__\([^)]*\)\s*)*(\w+)\s*\(", text):
        name = m.group(1)
        # the brace after the parameter list: skip nested parentheses
        depth, i = 1, m.end()
        while depth:
            depth += {"(": 1, ")": -1}.get(text[i], 0)
            i += 1
        body = text.index("{", i)
        yield name, text[body + 1:body + 400]


def test_every_data_kernel_opens_with_the_guard():
    seen = set()
    for f in ("tpc_find.cu", "tpc_fit.cu", "tpc_adjoint.cu", "tpc_common.cu", "tpc_noalloc.cu"):
        for name, head in kernels(os.path.join(CSRC, f)):
            seen.add(name)
            if name in UNGUARDED:
                continue
            first = head.strip().splitlines()
            # the guard is the first statement (comments aside)
            stmts = [ln.strip() for ln in first if ln.strip() and not ln.strip().startswith("//")]
            assert "input_rejected(" in stmts[0], f"{f}: {name} does not open with the input guard"
    # the scan found the kernels of every stage
    assert {"k_zrange", "k_hist", "k_scatter", "k_neighbours_first", "k_tracklet_lanes", "k_match",
            "k_track_len", "k_track_write", "k_fit", "k_adjoint"} <= seen


def test_track_len_reports_no_tracks_on_rejected_input():
    text = open(os.path.join(CSRC, "tpc_find.cu")).read()
    i = text.index("k_track_len(")
    head = text[text.index("{", text.index(") {", i)):][:300]
    assert "input_rejected(st)" in head and "*n_tracks_dev = 0" in head
