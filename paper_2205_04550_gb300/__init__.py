"""GB300-native brute-force tumour-database query (Ezhov et al. 2022).

The compute path is the CUDA library ``libdbq.so`` (C ABI in
``include/dbq.h``, sources in ``csrc/``); ``_dbq`` is its thin ctypes
binding and ``Database`` a small owner of one handle.  ``synth`` makes the
seeded surrogate volumes used as inputs.
"""
from __future__ import annotations

import numpy as np

from . import _dbq
from ._dbq import (DBQ_BITS, DBQ_F16, DBQ_F32, DBQ_FLAG_EMBED, DBQ_FLAG_SKETCH,
                   DBQ_MODE_EMBED_BF16, DBQ_MODE_EMBED_FP8, DBQ_MODE_EXACT, DBQ_MODE_HASH,
                   SKETCH_DIMS, db_get_codes, DBQ_STORE_BITS, DBQ_STORE_F16, HIT_DTYPE,
                   DbqError, db_build_masks, db_create, db_destroy, db_get_embeddings,
                   db_get_masks, db_info, db_last_error, db_load_volumes, db_prefilter,
                   db_prepare_patient, db_query, db_query_async, db_query_batch,
                   db_query_prepared, db_scan_counts, db_scan_packed_noalloc, db_set_option,
                   db_stage_times, DBQ_OPT_SPARSE, DBQ_OPT_RERANK, DBQ_PLAN_ITEMS_PER_SM, DBQ_PLAN_TC_MIN_QUERIES,
                   db_plan_create, db_plan_set, db_plan_query, db_plan_status, db_plan_destroy,
                   db_create_downsampled)

__all__ = ["Database", "ForwardModel", "DbqError", "HIT_DTYPE", "DBQ_F32", "DBQ_F16", "DBQ_BITS",
           "DBQ_STORE_BITS", "DBQ_STORE_F16", "DBQ_FLAG_EMBED", "DBQ_FLAG_SKETCH",
           "DBQ_MODE_EXACT", "DBQ_MODE_EMBED_BF16", "DBQ_MODE_EMBED_FP8", "DBQ_MODE_HASH",
           "SKETCH_DIMS", "db_get_codes", "db_query_batch", "db_prefilter",
           "db_get_embeddings", "db_scan_packed_noalloc", "db_set_option", "db_stage_times",
           "DBQ_OPT_SPARSE", "DBQ_OPT_RERANK", "DBQ_PLAN_ITEMS_PER_SM", "DBQ_PLAN_TC_MIN_QUERIES", "Plan",
           "db_plan_create", "db_plan_set", "db_plan_query", "db_plan_status", "db_plan_destroy", "db_create_downsampled", "db_create", "db_load_volumes",
           "db_build_masks", "db_query", "db_query_async", "db_prepare_patient",
           "db_query_prepared", "db_scan_counts", "db_get_masks",
           "db_info", "db_destroy", "db_last_error"]


class ForwardModel:
    """The tumour forward model of Section 2.1 (Eq. 1-2) on one grid and
    tissue map; ``simulate`` returns u(T_end) for rows of theta =
    (x, y, z, D_w, rho, T_end).  See include/rd.h for the scheme."""

    def __init__(self, tissue, batch: int = 0):
        t = tissue
        nz, ny, nx = (int(d) for d in t.shape)
        self.shape = (nx, ny, nz)
        self.handle = _dbq.rd_create(nx, ny, nz, t if not isinstance(t, np.ndarray)
                                     else np.ascontiguousarray(t, dtype=np.float32), batch)

    def simulate(self, theta, out=None, u0: float = 1.0, cfl: float = 0.9, stream=None):
        """-> (u [count, nz, ny, nx] float32 (``out`` if given: host array or
        device tensor), steps [count] int64)."""
        th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1, 6)
        nx, ny, nz = self.shape
        if out is None:
            out = np.zeros((th.shape[0], nz, ny, nx), dtype=np.float32)
        steps = np.zeros(th.shape[0], dtype=np.int64)
        _dbq.rd_simulate(self.handle, th, out, u0, cfl, steps, stream)
        return out, steps

    def stats(self) -> dict:
        return _dbq.rd_stats(self.handle)

    def close(self):
        if self.handle:
            _dbq.rd_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Database:
    """Owns one libdbq handle; methods map one-to-one onto the C calls."""

    def __init__(self, shape, capacity: int, storage: int = DBQ_STORE_BITS,
                 t1: float = 0.6, t2: float = 0.25, n_params: int = 0, embed: bool = False,
                 sketch: bool = False):
        nx, ny, nz = shape
        self.shape = (int(nx), int(ny), int(nz))
        self.sparse = False
        self.sparse_mode = 0
        self.capacity = int(capacity)
        self.storage = storage
        self.t1, self.t2 = float(np.float32(t1)), float(np.float32(t2))
        self.n_params = int(n_params)
        self.embed = bool(embed)
        self.sketch = bool(sketch)
        flags = (DBQ_FLAG_EMBED if embed else 0) | (DBQ_FLAG_SKETCH if sketch else 0)
        self.handle = db_create(nx, ny, nz, capacity, storage, t1, t2, n_params, flags)

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

    def downsampled(self, factor: int) -> "Database":
        """A nearest-neighbour downsampled copy (DS64 / DS32 of Section 2.3);
        it takes patients at this database's resolution."""
        obj = Database.__new__(Database)
        nx, ny, nz = self.shape
        obj.shape = (nx // factor, ny // factor, nz // factor)
        obj.capacity = self.capacity
        obj.storage = self.storage
        obj.t1, obj.t2 = self.t1, self.t2
        obj.n_params = self.n_params
        obj.embed = False
        obj.sparse = False
        obj.sparse_mode = 0
        obj.sketch = False
        obj.handle = db_create_downsampled(self.handle, factor)
        return obj

    def set_sparse(self, on=True):
        """Exact scans read only the patient's support (identical results):
        True / 1, or 2 for single-patient scans over a word-major copy of the
        planes (twice the planes' memory); False / 0 reads every word."""
        mode = 2 if on == 2 else (1 if on else 0)
        db_set_option(self.handle, DBQ_OPT_SPARSE, mode)
        self.sparse = bool(mode)
        self.sparse_mode = mode

    def set_rerank(self, mode):
        """How embedding batches re-rank their candidates on a dense database:
        2 reads each distinct candidate entry of the batch once, 1 reads each
        query's candidates separately, 0 (default) takes 2 for batches of 32
        queries or more, else 1 (the same hits)."""
        db_set_option(self.handle, DBQ_OPT_RERANK, int(mode))

    def embeddings(self, first: int, count: int):
        """-> dict of bf16 bits [count,2,d] uint16, e4m3 codes [count,2,d] uint8,
        scale, norm_bf16, norm_fp8 [count,2] float32."""
        nx, ny, nz = self.shape
        d = SKETCH_DIMS if self.sketch else (nx // 8) * (ny // 8) * (nz // 8)
        out = dict(bf16=np.zeros((count, 2, d), np.uint16), e4m3=np.zeros((count, 2, d), np.uint8),
                   scale=np.zeros((count, 2), np.float32),
                   norm_bf16=np.zeros((count, 2), np.float32),
                   norm_fp8=np.zeros((count, 2), np.float32))
        db_get_embeddings(self.handle, first, count, **out)
        return out

    def codes(self, first: int, count: int):
        """Sign codes of a sketch database -> uint32 [count, 2, SKETCH_DIMS/32]."""
        out = np.zeros((count, 2, SKETCH_DIMS // 32), np.uint32)
        db_get_codes(self.handle, first, count, out)
        return out

    def prefilter(self, patients, mode: int, n_candidates: int = 0, kind=None):
        """-> (dist [nq, N] float32, cand [nq, n_candidates] int32 or None)."""
        nq = len(patients)
        dist = np.zeros((nq, self.capacity), np.float32)
        cand = np.zeros((nq, n_candidates), np.int32) if n_candidates else None
        db_prefilter(self.handle, patients, mode, n_candidates, dist, cand, kind)
        return dist, cand

    def query_batch(self, patients, k: int, mode: int = DBQ_MODE_EXACT, n_candidates: int = 0,
                    t1=None, t2=None, kind=None):
        return db_query_batch([self.handle], [0] * len(patients), patients, k, mode,
                              n_candidates, t1, t2, kind, self.n_params)

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


class Plan:
    """Many exact queries against several bit-packed databases in one
    persistent launch (db_plan_*).  ``query`` only enqueues work and can be
    captured in a CUDA graph; outputs are device buffers of dbq_hit records."""

    def __init__(self, databases, max_queries: int, k: int):
        self.databases = list(databases)
        self.max_queries = int(max_queries)
        self.k = int(k)
        self.handle = db_plan_create([d.handle for d in self.databases], max_queries, k)

    def set_items_per_sm(self, value: int):
        db_plan_set(self.handle, DBQ_PLAN_ITEMS_PER_SM, int(value))

    def set_tc_min_queries(self, value: int, db: int | None = None):
        """Dense queries per database from which that database is scanned for
        all of them at once on the tensor cores (0 = never); for database
        ``db`` of the plan alone when given (-1 = back to the plan-wide value)."""
        if db is None:
            db_plan_set(self.handle, DBQ_PLAN_TC_MIN_QUERIES, int(value))
        else:
            _dbq.db_plan_set_for(self.handle, int(db), DBQ_PLAN_TC_MIN_QUERIES, int(value))

    def status(self, stream=None):
        db_plan_status(self.handle, stream)

    def query(self, db_of_query, patients_dev, hits_dev, kind=None, stream=None, keep=None):
        db_plan_query(self.handle, db_of_query, patients_dev, hits_dev, kind, stream=stream,
                      _keep=keep)

    def close(self):
        if self.handle:
            db_plan_destroy(self.handle)
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
