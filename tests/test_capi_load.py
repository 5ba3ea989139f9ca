"""The C-ABI library builds for sm_103a, loads, and exports exactly what include/pagerank.h
declares; host-side argument checks return statuses (no GPU needed, no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2109_09527_gb300 as pr
from paper_2109_09527_gb300 import _build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "pagerank.h")


def declared_functions():
    src = open(HEADER).read()
    return set(re.findall(r"PR_API\s+[\w\s\*]+?\b(pr_\w+)\s*\(", src))


def test_header_declares_the_boundary():
    names = declared_functions()
    assert {"pr_create_graph", "pr_destroy_graph", "pr_solve", "pr_iterate", "pr_status_string",
            "pr_last_error", "pr_graph_get_stats", "pr_set_option"} <= names


def test_library_exports_every_declared_symbol():
    path = _build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert declared_functions() <= exported
    # nothing else leaks out of the library
    assert {s for s in exported if not s.startswith("_")} == declared_functions()
    lib = pr.load()
    for name in declared_functions():
        assert hasattr(lib, name)
        assert name in pr.SIGNATURES


def test_status_strings_and_no_error_yet():
    assert pr.pr_status_string(pr.PR_OK) == "PR_OK"
    assert pr.pr_status_string(pr.PR_NOT_CONVERGED) == "PR_NOT_CONVERGED"
    assert pr.pr_status_string(99) == "PR_UNKNOWN_STATUS"


def test_argument_errors_return_status_without_a_gpu():
    lib = pr.load()
    out = ctypes.c_void_p()
    # out == NULL, n out of range, nnz < 0, missing arrays, bad layout: rejected before any CUDA call
    assert lib.pr_create_graph(4, 0, None, 0, None, None, 0, None, None) == pr.PR_ERR_INVALID_ARG
    assert lib.pr_create_graph(0, 0, None, 0, None, None, 0, None, ctypes.byref(out)) == pr.PR_ERR_INVALID_ARG
    rp = (ctypes.c_int32 * 3)(0, 1, 2)
    assert lib.pr_create_graph(2, -1, rp, 0, None, None, 0, None, ctypes.byref(out)) == pr.PR_ERR_INVALID_ARG
    assert lib.pr_create_graph(2, 2, None, 0, None, None, 0, None, ctypes.byref(out)) == pr.PR_ERR_INVALID_ARG
    assert lib.pr_create_graph(2, 2, rp, 0, None, None, 0, None, ctypes.byref(out)) == pr.PR_ERR_INVALID_ARG
    ci = (ctypes.c_int32 * 2)(1, 0)
    assert lib.pr_create_graph(2, 2, rp, 0, ci, None, 7, None, ctypes.byref(out)) == pr.PR_ERR_INVALID_ARG
    # an out-edge CSR is transposed on the device with 32-bit edge positions
    assert lib.pr_create_graph(2, 1 << 31, rp, 1, ci, None, pr.PR_OUT_CSR, None,
                               ctypes.byref(out)) == pr.PR_ERR_UNSUPPORTED
    w = (ctypes.c_float * 2)(1.0, 1.0)
    assert lib.pr_create_graph(2, 2, rp, 0, ci, w, 0, None, ctypes.byref(out)) == pr.PR_ERR_UNSUPPORTED
    assert lib.pr_create_graph(2, 1 << 31, rp, 0, ci, None, 0, None,
                               ctypes.byref(out)) == pr.PR_ERR_INVALID_ARG
    assert out.value is None
    assert "layout" in pr.pr_last_error() or "weights" in pr.pr_last_error() or pr.pr_last_error()
    # solve on a NULL graph
    info = pr.pr_info()
    x = (ctypes.c_float * 2)()
    assert lib.pr_solve(None, 0.85, 1e-6, 10, 0, None, None, x, ctypes.byref(info), None) == pr.PR_ERR_INVALID_ARG
    assert lib.pr_iterate(None, 0.85, None, x, 1, x, ctypes.byref(info), None) == pr.PR_ERR_INVALID_ARG
    assert lib.pr_destroy_graph(None) == pr.PR_OK
    assert lib.pr_graph_get_stats(None, None) == pr.PR_ERR_INVALID_ARG
    # the gather-rate diagnostic checks every argument before touching CUDA
    res = (ctypes.c_double * 3)()
    bad = [(1 << 24, 1 << 20, 0, 4, 4, None),      # no output array
           (0, 1 << 20, 0, 4, 4, res),             # empty vector
           (1 << 24, 1000, 0, 4, 4, res),          # indices not a multiple of 512
           (1 << 24, 512, 0, 4, 4, res),           # fewer than two chunks
           (1 << 24, 1 << 20, 2, 4, 4, res),       # cached not 0/1
           (1 << 24, 1 << 20, 0, 0, 4, res),       # no blocks
           (1 << 24, 1 << 20, 0, 9, 4, res),       # more than 8 blocks per SM
           (1 << 24, 1 << 20, 0, 4, 0, res),       # no chunks
           (1 << 24, 1 << 20, 0, 4, 65537, res)]   # too many chunks
    for nv, ni, cached, bps, chunks, o in bad:
        assert lib.pr_measure_gather_rate(nv, ni, cached, bps, chunks, 1, o, None) == pr.PR_ERR_INVALID_ARG
        assert "pr_measure_gather_rate" in pr.pr_last_error()


def test_options_validate_host_side():
    with pytest.raises(pr.PageRankError):
        pr.set_heavy_degree(100)          # not a power of two
    with pytest.raises(pr.PageRankError):
        pr.set_heavy_degree(32)           # too small
    with pytest.raises(pr.PageRankError):
        pr.set_heavy_degree(8192)         # light tiles must fit their staging area
    pr.set_heavy_degree(pr.DEFAULT_HEAVY_DEGREE)
    with pytest.raises(pr.PageRankError):
        pr.pr_set_option(None, 99, 1)
    for key in (pr.PR_OPT_USE_GRAPH, pr.PR_OPT_STAGED_TILES, pr.PR_OPT_NB_HUBS,
                pr.PR_OPT_HOT_VERTICES, pr.PR_OPT_HOT_CACHE, pr.PR_OPT_CTAS_PER_SM,
                pr.PR_OPT_TMA_TILES, pr.PR_OPT_TEST_WITHHOLD_COPY, pr.PR_OPT_LIGHT_LANES,
                pr.PR_OPT_FUSED_SEGMENTS, pr.PR_OPT_BATCH_DC, pr.PR_OPT_BATCH_ASYNC,
                pr.PR_OPT_IMPLICIT_ZERO_ROWS, pr.PR_OPT_SYNC_DC, pr.PR_OPT_TMA_HOT_VERTICES,
                pr.PR_OPT_NB_PIPELINE):
        with pytest.raises(pr.PageRankError):
            pr.pr_set_option(None, key, 1)               # needs a graph
    pr.pr_set_option(None, pr.PR_OPT_INDEX64, 0)


def test_build_targets_sm103a_only():
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of pr_info and pr_graph_stats have the C layout (sizes and
    offsets printed by a C program compiled against include/pagerank.h)."""
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"pr_info": pr.pr_info, "pr_graph_stats": pr.pr_graph_stats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "pagerank.h"', "int main(void) {"]
    for sname, cls in structs.items():
        lines.append(f'printf("{sname} sizeof %zu\\n", sizeof({sname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{sname} {fname} %zu\\n", offsetof({sname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(line.split()[:2]): int(line.split()[2]) for line in out if line}
    for sname, cls in structs.items():
        assert got[(sname, "sizeof")] == ctypes.sizeof(cls), sname
        for fname, _ in cls._fields_:
            assert got[(sname, fname)] == getattr(cls, fname).offset, (sname, fname)


def test_binding_constants_match_the_header():
    """Every PR_OPT_* option key and pr_status value the header defines has the same value
    in the Python binding."""
    import re
    text = open(HEADER).read()
    defines = dict(re.findall(r"#define (PR_OPT_[A-Z0-9_]+) (\d+)", text))
    assert defines, "no option keys found in the header"
    for name, value in defines.items():
        assert getattr(pr, name) == int(value), name
    statuses = dict(re.findall(r"\b(PR_(?:OK|ERR_[A-Z_]+|NOT_CONVERGED)) = (\d+)", text))
    assert "PR_ERR_DEVICE_TIMEOUT" in statuses
    for name, value in statuses.items():
        assert getattr(pr, name) == int(value), name
