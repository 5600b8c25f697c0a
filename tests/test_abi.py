"""The C-ABI library builds, loads and exports every function include/sss.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import paper_2404_16517_gb300 as sss
from paper_2404_16517_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(sss_\w+)\s*\(", txt):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_function():
    _build.build()
    h = ctypes.CDLL(_build.LIB)
    names = declared_functions()
    assert "sss_sort" in names and "sss_lcp_merge" in names and "sss_dist_prefix" in names
    for name in sorted(names):
        assert hasattr(h, name), name


def test_binding_covers_declared_functions():
    _build.build()
    assert set(sss.exported_symbols()) >= declared_functions() - {"sss_kernel_stat"}
    h = sss.lib()
    for name in sss.exported_symbols():
        getattr(h, name)


def test_status_strings_and_defaults():
    _build.build()
    h = sss.lib()
    assert h.sss_status_string(0) == b"ok"
    p = sss.params()
    assert p.v == 2 and p.kmax == sss.SSS_KMAX_AUTO and p.kmin == 0
    assert sss.workspace_bytes(1 << 20, 500 << 20, 16) > (1 << 20) * 8


def test_null_context_is_rejected():
    _build.build()
    h = sss.lib()
    assert h.sss_sync(None) == 1
    assert h.sss_destroy(None) == 0
