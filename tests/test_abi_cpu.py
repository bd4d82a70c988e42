"""The C ABI library builds, loads and exports every entry point its header
declares (no GPU needed: nothing here computes)."""
import ctypes
import os
import re

from paper_2205_04550_gb300 import _dbq, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header, prefix="db_"):
    text = open(os.path.join(ROOT, "include", header)).read()
    return set(re.findall(r"^\s*(?:int|const char\*)\s+(" + prefix + r"\w+)\s*\(", text, re.M))


def test_libdbq_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.build())
    declared = _declared("dbq.h")
    assert declared, "no declarations parsed"
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared == set(_dbq.EXPORTED)
    rd = _declared("rd.h", "rd_")
    assert rd == {"rd_create", "rd_simulate", "rd_stats", "rd_destroy"}
    for name in sorted(rd):
        assert hasattr(lib, name), name
    assert rd == set(_dbq.EXPORTED_RD)


def test_binding_loads_and_reports_no_error():
    build.build()
    lib = _dbq.load()
    assert lib.db_last_error() in (b"", None)
    # argument checks that fail before any CUDA call
    h = ctypes.c_void_p()
    rc = lib.db_create(ctypes.byref(h), 0, 8, 8, 4, 0, 0.6, 0.25, 0, 0)
    assert rc == _dbq.DBQ_EINVAL and h.value is None
    assert b"grid" in lib.db_last_error()
    assert lib.db_destroy(None) == 0
