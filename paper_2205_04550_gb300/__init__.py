"""GB300-native brute-force tumour-database query (Ezhov et al. 2022).

The compute path is the CUDA library ``libdbq.so`` (C ABI in
``include/dbq.h``, sources in ``csrc/``); ``_dbq`` is its thin ctypes
binding and ``Database`` a small owner of one handle.  ``synth`` makes the
seeded surrogate volumes used as inputs.
"""
from __future__ import annotations

import numpy as np

from . import _dbq
from ._dbq import (DBQ_BITS, DBQ_F16, DBQ_F32, DBQ_STORE_BITS, DBQ_STORE_F16, HIT_DTYPE,
                   DbqError, db_build_masks, db_create, db_destroy, db_get_masks, db_info,
                   db_last_error, db_load_volumes, db_prepare_patient, db_query,
                   db_query_async, db_query_prepared, db_scan_counts)

__all__ = ["Database", "DbqError", "HIT_DTYPE", "DBQ_F32", "DBQ_F16", "DBQ_BITS",
           "DBQ_STORE_BITS", "DBQ_STORE_F16", "db_create", "db_load_volumes",
           "db_build_masks", "db_query", "db_query_async", "db_prepare_patient",
           "db_query_prepared", "db_scan_counts", "db_get_masks",
           "db_info", "db_destroy", "db_last_error"]


class Database:
    """Owns one libdbq handle; methods map one-to-one onto the C calls."""

    def __init__(self, shape, capacity: int, storage: int = DBQ_STORE_BITS,
                 t1: float = 0.6, t2: float = 0.25, n_params: int = 0):
        nx, ny, nz = shape
        self.shape = (int(nx), int(ny), int(nz))
        self.capacity = int(capacity)
        self.storage = storage
        self.t1, self.t2 = float(np.float32(t1)), float(np.float32(t2))
        self.n_params = int(n_params)
        self.handle = db_create(nx, ny, nz, capacity, storage, t1, t2, n_params)

    def load(self, first: int, vols, params=None, stream=None):
        db_load_volumes(self.handle, first, int(vols.shape[0]), vols, params=params,
                        stream=stream)

    def build(self, stream=None):
        db_build_masks(self.handle, stream)

    def query(self, patient, k: int, t1=float("nan"), t2=float("nan"), kind=None, stream=None):
        return db_query(self.handle, patient, k, t1, t2, kind, self.n_params, stream)

    def query_async(self, patient_dev, k: int, hits_dev, t1=float("nan"), t2=float("nan"),
                    kind=None, stream=None):
        db_query_async(self.handle, patient_dev, k, hits_dev, t1, t2, kind, stream)

    def scan_counts(self, patient, t1=float("nan"), t2=float("nan"), kind=None, stream=None):
        counts = np.zeros((self.capacity, 4), dtype=np.uint32)
        pcount = np.zeros(2, dtype=np.uint32)
        db_scan_counts(self.handle, patient, counts, pcount, t1, t2, kind, stream)
        return counts, pcount

    def masks(self, first: int, count: int):
        info = self.info()
        planes = np.zeros((count, 2, info["words"]), dtype=np.uint32)
        sizes = np.zeros((count, 2), dtype=np.uint32)
        db_get_masks(self.handle, first, count, planes, sizes)
        return planes, sizes

    def info(self) -> dict:
        return db_info(self.handle)

    def close(self):
        if self.handle:
            db_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
