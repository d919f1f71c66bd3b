"""The C-ABI library loads and exports every symbol include/tnvan.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2504_12037_gb300 import tnvan as tv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names.update(re.findall(r"\b(tnvan_\w+)\s*\(", src))
    return names


def test_header_declares_the_boundary_calls():
    d = _declared()
    for name in ["tnvan_init_graph", "tnvan_set_width_set", "tnvan_sample_and_contract",
                 "tnvan_free_energy", "tnvan_backward"]:
        assert name in d


def test_library_exports_every_declared_symbol():
    if not os.path.exists(tv.LIB_PATH):
        import __graft_entry__

        __graft_entry__.build()
    L = ctypes.CDLL(tv.LIB_PATH)
    for name in sorted(_declared()):
        assert hasattr(L, name), name
    assert set(tv.SIGNATURES) == _declared()


def test_version_and_errors_without_gpu():
    L = tv.lib()
    assert L.tnvan_version() >= 100
    assert L.tnvan_destroy(None) == 0
    # creating a context on a machine without a usable device fails cleanly
    h = ctypes.c_void_p()
    rc = L.tnvan_create(ctypes.byref(h), 10 ** 6)
    assert rc in (tv.E_ARG, tv.E_CUDA)
    assert len(L.tnvan_last_error(None)) > 0
