"""CPU-only checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point include/wtri.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"WTRI_API\s+[^;(]*?\b(wtri_\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("wtri_build_csr", "wtri_topk", "wtri_sample_topk", "wtri_last_error"):
        assert must in names


def test_library_builds_and_exports_everything():
    from paper_1910_00692_gb300 import build_lib
    path = build_lib.build()
    assert os.path.exists(path)
    L = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing
    L.wtri_version.restype = ctypes.c_char_p
    assert b"sm_103a" in L.wtri_version()


def test_binding_reports_errors_without_gpu_work():
    import paper_1910_00692_gb300 as wt
    L = wt.lib()
    # NULL out-pointer is rejected before any CUDA call.
    rc = L.wtri_build_csr(1, 0, None, None, None, 0, None, None)
    assert rc == -1
    assert b"NULL" in L.wtri_last_error()


def test_oracle_and_product_are_independent():
    """Neither side imports or links the other."""
    pkg = os.path.join(ROOT, "paper_1910_00692_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.findall(r"(?:import|include)\s+\S*", text).__str__(), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_1910_00692_gb300" not in text, f
            assert "wtri.h" not in text, f
