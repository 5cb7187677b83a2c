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
