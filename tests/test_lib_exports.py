"""The CUDA library builds for sm_103a here (no GPU needed) and exports every
function include/sqr.h declares; the oracle is a separate library and the
product binding refuses to run without libsqr (no CPU fallback)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^\s*(?:size_t|sq_status_t|const char\*)\s+(sq_\w+)\s*\(", src, re.M)
    return names


def test_library_exports_every_declared_symbol():
    from paper_2511_17361_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 7
    for n in names:
        assert hasattr(lib, n), n
    nm = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}$", nm, re.M), n


def test_checked_build_exports_the_same_symbols():
    """The debug build with bounds checks (-DSQR_CHECK, libsqr_check.so) has the same
    boundary; the normal library answers sq_check_query with "not compiled" and
    makes no CUDA call doing so (it works without a GPU)."""
    from paper_2511_17361_gb300 import _build
    path = _build.build(check=True)
    assert os.path.basename(path) == "libsqr_check.so"
    nm = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    for n in _declared():
        assert re.search(rf"\bT {n}$", nm, re.M), n
    from paper_2511_17361_gb300 import sqr
    assert os.path.basename(sqr.LIB_PATH) == "libsqr.so"
    assert sqr.check_query() == (False, 0)


def test_library_is_sm103a_only():
    from paper_2511_17361_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)


def test_status_strings_and_host_validation_without_gpu():
    """Host-side argument checks run before any CUDA call, so they work without a GPU."""
    from paper_2511_17361_gb300 import sqr
    assert sqr.lib.sq_status_string(0) == b"SQ_OK"
    assert b"capacity" in sqr.lib.sq_status_string(2)
    g = sqr.SqGrid(0, 1, 1, (ctypes.c_float * 3)(0, 0, 0), (ctypes.c_float * 3)(1, 1, 1))
    assert sqr.lib.sq_workspace_size(sqr.SQ_OP_INDEX, None, ctypes.byref(g), None) == 0
    g2 = sqr.SqGrid(200, 200, 16, (ctypes.c_float * 3)(-40, -40, -1), (ctypes.c_float * 3)(0.4, 0.4, 0.4))
    assert sqr.lib.sq_workspace_size(sqr.SQ_OP_INDEX, None, ctypes.byref(g2), None) > 640000 * 4
    p = sqr.SqPrims(None, None, None, None, None, None, 10, 18)
    st = sqr.lib.sq_build_index(ctypes.byref(p), ctypes.byref(g2), None, None, None, 0, None)
    assert st == sqr.SQ_ERR_INVALID_ARG


def test_oracle_is_not_imported_by_the_product_package():
    pkg = os.path.join(ROOT, "paper_2511_17361_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src and "sqr_oracle" not in src, f


def test_saved_state_sizes_without_gpu():
    """sq_saved_size is the paged size of every sample's page; sizes grow with the
    page count; invalid page counts give 0 (host arithmetic only)."""
    from paper_2511_17361_gb300 import sqr
    dummy = (ctypes.c_float * 16)()
    p = ctypes.cast(dummy, ctypes.c_void_p)
    for (nc, H, W, L, C) in [(1, 1, 1, 40, 5), (6, 225, 400, 100, 18), (2, 3, 5, 7, 32)]:
        r = sqr.SqRays(nc, H, W, p, p, p, L, 0.0, 1.0)
        pages = nc * H * W * ((L + sqr.SQ_SAVE_PAGE - 1) // sqr.SQ_SAVE_PAGE)
        full = sqr.lib.sq_saved_size(ctypes.byref(r), C)
        assert full == sqr.lib.sq_saved_size_pages(ctypes.byref(r), C, pages)
        sizes = [sqr.lib.sq_saved_size_pages(ctypes.byref(r), C, q) for q in (1, 2, pages // 2 + 1, pages)]
        assert all(a <= b for a, b in zip(sizes, sizes[1:])) and sizes[0] > 0
        assert sqr.lib.sq_saved_size_pages(ctypes.byref(r), C, 0) == 0
