"""ctypes binding of libdbq (include/dbq.h) -- argument marshalling only.

Every function has the name of the C entry point it calls and raises
``DbqError`` when the call returns a non-zero status.  Array arguments may
be torch tensors (CUDA or CPU, contiguous), numpy arrays, or raw integer
addresses; the library itself decides whether a pointer is host or device
memory.  No computation of the query happens in Python.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

DBQ_OK = 0
DBQ_EINVAL = -1
DBQ_ENOMEM = -2
DBQ_ESTATE = -3
DBQ_ECUDA = -4
DBQ_ETIMEOUT = -5
DBQ_ERANGE = -6

DBQ_F32 = 0
DBQ_F16 = 1
DBQ_BITS = 2

DBQ_STORE_BITS = 0
DBQ_STORE_F16 = 1

DBQ_FLAG_EMBED = 1
DBQ_FLAG_SKETCH = 2
SKETCH_DIMS = 4096

DBQ_OPT_SPARSE = 1
DBQ_OPT_RERANK = 2

DBQ_PLAN_ITEMS_PER_SM = 1
DBQ_PLAN_TC_MIN_QUERIES = 2
DBQ_PLAN_TEST_STALL_NS = 3

DBQ_MODE_EXACT = 0
DBQ_MODE_EMBED_BF16 = 1
DBQ_MODE_EMBED_FP8 = 2
DBQ_MODE_HASH = 3

STATUS_NAMES = {0: "DBQ_OK", -1: "DBQ_EINVAL", -2: "DBQ_ENOMEM", -3: "DBQ_ESTATE",
                -4: "DBQ_ECUDA", -5: "DBQ_ETIMEOUT", -6: "DBQ_ERANGE"}


class DbqError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class dbq_hit(ctypes.Structure):
    _fields_ = [("index", ctypes.c_int64), ("score", ctypes.c_double),
                ("i1", ctypes.c_uint32), ("i2", ctypes.c_uint32),
                ("e1", ctypes.c_uint32), ("e2", ctypes.c_uint32),
                ("p1", ctypes.c_uint32), ("p2", ctypes.c_uint32)]


HIT_DTYPE = np.dtype([("index", "<i8"), ("score", "<f8"), ("i1", "<u4"), ("i2", "<u4"),
                      ("e1", "<u4"), ("e2", "<u4"), ("p1", "<u4"), ("p2", "<u4")])
assert HIT_DTYPE.itemsize == ctypes.sizeof(dbq_hit) == 40

_lib = None
_lock = threading.Lock()

# (name, restype, argtypes)
_P = ctypes.c_void_p
_SIGS = [
    ("db_create", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                 ctypes.c_int, ctypes.c_uint32]),
    ("db_load_volumes", ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int64, _P, ctypes.c_int, _P,
                                       _P]),
    ("db_build_masks", ctypes.c_int, [_P, _P]),
    ("db_query", ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                ctypes.c_int, _P, _P, _P]),
    ("db_query_async", ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                      ctypes.c_int, _P, _P]),
    ("db_prepare_patient", ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                          _P]),
    ("db_query_prepared", ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    ("db_scan_counts", ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_float, ctypes.c_float, _P,
                                      _P, _P]),
    ("db_get_masks", ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int64, _P, _P, _P]),
    ("db_info", ctypes.c_int, [_P, _P]),
    ("db_query_batch", ctypes.c_int, [_P, _P, ctypes.c_int, _P, ctypes.c_int, _P, _P,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P]),
    ("db_prefilter", ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, _P, _P, _P]),
    ("db_get_embeddings", ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int64, _P, _P, _P, _P, _P,
                                         _P]),
    ("db_get_codes", ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int64, _P, _P]),
    ("db_stage_times", ctypes.c_int, [_P, _P, ctypes.c_int]),
    ("db_set_option", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int64]),
    ("db_last_support", ctypes.c_int, [_P, _P]),
    ("db_plan_create", ctypes.c_int, [ctypes.POINTER(_P), _P, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int]),
    ("db_plan_set", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int64]),
    ("db_plan_set_for", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int64]),
    ("db_plan_query", ctypes.c_int, [_P, _P, ctypes.c_int, _P, ctypes.c_int, _P, _P, _P, _P]),
    ("db_plan_status", ctypes.c_int, [_P, _P]),
    ("db_plan_destroy", ctypes.c_int, [_P]),
    ("db_create_downsampled", ctypes.c_int, [ctypes.POINTER(_P), _P, ctypes.c_int]),
    ("db_scan_packed_noalloc", ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int64, _P, _P,
                                              ctypes.c_int, _P, _P]),
    ("db_destroy", ctypes.c_int, [_P]),
    ("db_last_error", ctypes.c_char_p, []),
]

# the forward model (include/rd.h)
_SIGS += [
    ("rd_create", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, ctypes.c_int, _P,
                                 ctypes.c_int]),
    ("rd_simulate", ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_float, ctypes.c_double, _P, _P,
                                   _P]),
    ("rd_stats", ctypes.c_int, [_P, _P]),
    ("rd_destroy", ctypes.c_int, [_P]),
]
EXPORTED = [name for name, _, _ in _SIGS if name.startswith("db_")]
EXPORTED_RD = [name for name, _, _ in _SIGS if name.startswith("rd_")]


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libdbq.so (built by ``paper_2205_04550_gb300.build.build()``).

    Raises RuntimeError if the library has not been built: there is no
    fallback implementation."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or _build.LIB
        if not os.path.exists(p):
            raise RuntimeError(f"libdbq.so not found at {p}; build it with "
                               "paper_2205_04550_gb300.build.build() (nvcc, sm_103a)")
        lib = ctypes.CDLL(p)
        for name, res, args in _SIGS:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(rc: int):
    if rc != DBQ_OK:
        msg = load().db_last_error()
        raise DbqError(rc, msg.decode() if msg else "")


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(s) -> int | None:
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:  # pragma: no cover
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _kind_of(x) -> int:
    dt = str(getattr(x, "dtype", ""))
    if "float32" in dt:
        return DBQ_F32
    if "float16" in dt or "uint16" in dt or "int16" in dt:
        return DBQ_F16
    if "uint32" in dt or "int32" in dt:
        return DBQ_BITS
    raise TypeError(f"unsupported dtype {dt}")


# ---------------------------------------------------------------- entry points
def db_create(nx: int, ny: int, nz: int, capacity: int, storage: int = DBQ_STORE_BITS,
              t1: float = 0.6, t2: float = 0.25, n_params: int = 0, flags: int = 0) -> int:
    h = _P()
    _check(load().db_create(ctypes.byref(h), nx, ny, nz, capacity, storage, t1, t2, n_params,
                            flags))
    return h.value


def db_load_volumes(db: int, first: int, count: int, vols, kind: int | None = None,
                    params=None, stream=None):
    if params is not None:
        params = np.ascontiguousarray(params, dtype=np.float64)
    _check(load().db_load_volumes(db, first, count, _ptr(vols),
                                  _kind_of(vols) if kind is None else kind, _ptr(params),
                                  _stream(stream)))


def db_build_masks(db: int, stream=None):
    _check(load().db_build_masks(db, _stream(stream)))


def db_query(db: int, patient, k: int, t1: float = float("nan"), t2: float = float("nan"),
             kind: int | None = None, n_params: int = 0, stream=None):
    """-> (hits structured numpy array [k] of HIT_DTYPE, params [k, n_params])."""
    hits = np.zeros(k, dtype=HIT_DTYPE)
    params = np.zeros((k, n_params), dtype=np.float64) if n_params else None
    _check(load().db_query(db, _ptr(patient), _kind_of(patient) if kind is None else kind,
                           t1, t2, k, hits.ctypes.data, _ptr(params), _stream(stream)))
    return hits, params


def db_query_async(db: int, patient_dev, k: int, hits_dev, t1: float = float("nan"),
                   t2: float = float("nan"), kind: int | None = None, stream=None):
    _check(load().db_query_async(db, _ptr(patient_dev),
                                 _kind_of(patient_dev) if kind is None else kind, t1, t2, k,
                                 _ptr(hits_dev), _stream(stream)))


def db_prepare_patient(db: int, patient_dev, t1: float = float("nan"), t2: float = float("nan"),
                       kind: int | None = None, stream=None):
    _check(load().db_prepare_patient(db, _ptr(patient_dev),
                                     _kind_of(patient_dev) if kind is None else kind, t1, t2,
                                     _stream(stream)))


def db_query_prepared(db: int, k: int, hits_dev, stream=None):
    _check(load().db_query_prepared(db, k, _ptr(hits_dev), _stream(stream)))


def db_scan_counts(db: int, patient, counts, pcount, t1: float = float("nan"),
                   t2: float = float("nan"), kind: int | None = None, stream=None):
    _check(load().db_scan_counts(db, _ptr(patient), _kind_of(patient) if kind is None else kind,
                                 t1, t2, _ptr(counts), _ptr(pcount), _stream(stream)))


def db_get_masks(db: int, first: int, count: int, planes, sizes=None, stream=None):
    _check(load().db_get_masks(db, first, count, _ptr(planes), _ptr(sizes), _stream(stream)))


def db_info(db: int) -> dict:
    out = np.zeros(8, dtype=np.int64)
    _check(load().db_info(db, out.ctypes.data))
    keys = ("n", "v", "words", "padded_words", "storage", "built", "n_params", "device_bytes")
    return dict(zip(keys, (int(x) for x in out)))


def _ptr_array(xs):
    arr = (ctypes.c_void_p * len(xs))()
    for i, x in enumerate(xs):
        arr[i] = _ptr(x)
    return arr


def db_query_batch(dbs, db_of_query, patients, k: int, mode: int = DBQ_MODE_EXACT,
                   n_candidates: int = 0, t1=None, t2=None, kind: int | None = None,
                   n_params: int = 0, stream=None):
    """-> (hits [nq, k] HIT_DTYPE, params [nq, k, n_params] or None)."""
    nq = len(patients)
    hits = np.zeros((nq, k), dtype=HIT_DTYPE)
    params = np.zeros((nq, k, n_params), dtype=np.float64) if n_params else None
    dba = (ctypes.c_void_p * len(dbs))(*dbs)
    dq = np.ascontiguousarray(db_of_query, dtype=np.int32)
    a1 = None if t1 is None else np.ascontiguousarray(t1, dtype=np.float32)
    a2 = None if t2 is None else np.ascontiguousarray(t2, dtype=np.float32)
    _check(load().db_query_batch(dba, dq.ctypes.data, nq, _ptr_array(patients),
                                 _kind_of(patients[0]) if kind is None else kind,
                                 _ptr(a1), _ptr(a2), k, mode, n_candidates,
                                 hits.ctypes.data, _ptr(params), _stream(stream)))
    return hits, params


def db_prefilter(db: int, patients, mode: int, n_candidates: int = 0, dist=None, cand=None,
                 kind: int | None = None, stream=None):
    _check(load().db_prefilter(db, len(patients), _ptr_array(patients),
                               _kind_of(patients[0]) if kind is None else kind, mode,
                               n_candidates, _ptr(dist), _ptr(cand), _stream(stream)))


def db_get_embeddings(db: int, first: int, count: int, bf16=None, e4m3=None, scale=None,
                      norm_bf16=None, norm_fp8=None, stream=None):
    _check(load().db_get_embeddings(db, first, count, _ptr(bf16), _ptr(e4m3), _ptr(scale),
                                    _ptr(norm_bf16), _ptr(norm_fp8), _stream(stream)))


def db_get_codes(db: int, first: int, count: int, codes, stream=None):
    _check(load().db_get_codes(db, first, count, _ptr(codes), _stream(stream)))


def db_set_option(db: int, option: int, value: int):
    _check(load().db_set_option(db, option, value))


def db_plan_create(dbs, max_queries: int, k: int) -> int:
    h = _P()
    arr = (ctypes.c_void_p * len(dbs))(*dbs)
    _check(load().db_plan_create(ctypes.byref(h), arr, len(dbs), max_queries, k))
    return h.value


def db_plan_set(plan: int, param: int, value: int):
    _check(load().db_plan_set(plan, param, value))


def db_plan_set_for(plan: int, db_index: int, param: int, value: int):
    _check(load().db_plan_set_for(plan, db_index, param, value))


def db_plan_query(plan: int, db_of_query, patients_dev, hits_dev, kind: int | None = None,
                  t1=None, t2=None, stream=None, _keep=None):
    """Enqueue the plan's persistent exact scan; patients and hits are device
    memory.  ``_keep`` (a list) receives the argument arrays so a caller that
    captures the call into a graph can keep them alive."""
    dq = np.ascontiguousarray(db_of_query, dtype=np.int32)
    a1 = None if t1 is None else np.ascontiguousarray(t1, dtype=np.float32)
    a2 = None if t2 is None else np.ascontiguousarray(t2, dtype=np.float32)
    pa = _ptr_array(patients_dev)
    if _keep is not None:
        _keep.extend([dq, a1, a2, pa])
    _check(load().db_plan_query(plan, dq.ctypes.data, len(patients_dev), pa,
                                _kind_of(patients_dev[0]) if kind is None else kind,
                                _ptr(a1), _ptr(a2), _ptr(hits_dev), _stream(stream)))


def db_create_downsampled(src: int, factor: int) -> int:
    h = _P()
    _check(load().db_create_downsampled(ctypes.byref(h), src, factor))
    return h.value


def db_plan_status(plan: int, stream=None):
    """Raises DbqError (DBQ_ETIMEOUT) if a tensor-core wait of the plan has
    timed out since the last check; synchronises the stream."""
    _check(load().db_plan_status(plan, _stream(stream)))


def db_plan_destroy(plan: int):
    _check(load().db_plan_destroy(plan))


def db_last_support(db: int):
    """Support-list lengths (16-byte words) of the last sparse patient."""
    out = np.zeros(2, dtype=np.int64)
    _check(load().db_last_support(db, out.ctypes.data))
    return int(out[0]), int(out[1])


def db_stage_times(db: int) -> dict:
    """GPU ms per stage of the handle's last embedding-mode batch."""
    ms = np.zeros(5, dtype=np.float32)
    _check(load().db_stage_times(db, ms.ctypes.data, 5))
    keys = ("patients", "query_embed", "distances", "select", "rerank")
    return dict(zip(keys, (float(x) for x in ms)))


def db_scan_packed_noalloc(planes, sizes, n: int, stride_words: int, patient_planes,
                           patient_sizes, k: int, hits_dev, stream=None):
    """Allocation-free exact query over caller-owned device buffers (see
    include/dbq.h); only enqueues work."""
    _check(load().db_scan_packed_noalloc(_ptr(planes), _ptr(sizes), n, stride_words,
                                         _ptr(patient_planes), _ptr(patient_sizes), k,
                                         _ptr(hits_dev), _stream(stream)))


def db_destroy(db: int):
    _check(load().db_destroy(db))


def db_last_error() -> str:
    msg = load().db_last_error()
    return msg.decode() if msg else ""


def hits_from_device(t) -> np.ndarray:
    """View a device buffer of dbq_hit records (copied to host) as HIT_DTYPE."""
    return t.cpu().numpy().view(HIT_DTYPE).reshape(-1)


# ---------------------------------------------------------------- forward model
def rd_create(nx: int, ny: int, nz: int, tissue, batch: int = 0) -> int:
    h = _P()
    _check(load().rd_create(ctypes.byref(h), nx, ny, nz, _ptr(tissue), batch))
    return h.value


def rd_simulate(rs: int, theta, out, u0: float = 1.0, cfl: float = 0.9, steps=None, stream=None):
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1, 6)
    _check(load().rd_simulate(rs, th.shape[0], th.ctypes.data, u0, cfl, _ptr(out), _ptr(steps),
                              _stream(stream)))


def rd_stats(rs: int) -> dict:
    out = np.zeros(4, dtype=np.float64)
    _check(load().rd_stats(rs, out.ctypes.data))
    return {"step_ms": float(out[0]), "step_launches": int(out[1]),
            "voxel_updates": int(out[2]), "slots": int(out[3])}


def rd_destroy(rs: int):
    if rs:
        load().rd_destroy(rs)
