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


def test_binding_constants_match_the_header():
    """Every enumerator and DBQ_ flag of include/dbq.h has the same value in the
    binding (an option or mode renumbered on one side would be passed through
    silently as another)."""
    text = open(os.path.join(ROOT, "include", "dbq.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    consts = {m.group(1): int(m.group(2))
              for m in re.finditer(r"\b(DBQ_[A-Z0-9_]+)\s*=\s*(-?\d+)", text)}
    consts.update({m.group(1): int(m.group(2))
                   for m in re.finditer(r"#define\s+(DBQ_[A-Z0-9_]+)\s+(\d+)u?\b", text)})
    for name in ("DBQ_OK", "DBQ_ETIMEOUT", "DBQ_OPT_SPARSE", "DBQ_OPT_RERANK",
                 "DBQ_MODE_HASH", "DBQ_FLAG_SKETCH", "DBQ_PLAN_TC_MIN_QUERIES"):
        assert name in consts, name
    for name, value in sorted(consts.items()):
        assert getattr(_dbq, name) == value, name
