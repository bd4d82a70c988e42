"""Shared helpers of the GPU parity tests (inputs and oracle comparisons)."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2205_04550_gb300 import synth


def pack_bits_np(mask: np.ndarray) -> np.ndarray:
    """[2][V] 0/1 -> [2][ceil(V/32)] uint32 with bit b of word w = voxel 32w+b
    (numpy little-endian bit packing; an input format, not the method)."""
    v = mask.shape[-1]
    words = (v + 31) // 32
    pad = np.zeros((2, words * 32), dtype=np.uint8)
    pad[:, :v] = mask
    b = np.packbits(pad.reshape(2, words * 32), axis=1, bitorder="little")
    return b.view("<u4").reshape(2, words).copy()


def random_db(shape, n, seed=0, p_zero=0.5, plant=()):
    """Uniform random float32 volumes with many zeros; planted copies of the
    patient at the given indices.  Returns (db [n,*], patient)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    db = rng.random((n, nz, ny, nx), dtype=np.float32)
    db[rng.random(db.shape) < p_zero] = 0.0
    patient = rng.random((nz, ny, nx), dtype=np.float32)
    patient[rng.random(patient.shape) < p_zero] = 0.0
    for j in plant:
        db[j] = patient
    return db, patient


def surrogate_db(shape, n, seed=synth.DB_SEED, patient_q=1, plant=()):
    db, theta = synth.database_np(shape, n, seed)
    pat, _ = synth.patients_np(shape, [patient_q], seed)
    for j in plant:
        db[j] = pat[0]
    return db, pat[0], theta


def assert_hits_equal(hits, ref, k):
    """GPU hits (HIT_DTYPE) vs oracle.query result: index, score bits, counts."""
    assert hits.shape[0] == k
    np.testing.assert_array_equal(hits["index"], ref["index"][:k])
    np.testing.assert_array_equal(hits["score"].view(np.uint64),
                                  ref["score"][:k].view(np.uint64))
    got = np.stack([hits[f] for f in ("i1", "i2", "e1", "e2", "p1", "p2")], axis=1)
    np.testing.assert_array_equal(got, ref["counts"][:k])


def oracle_query(db, patient, t1, t2, k, patient_mask=None):
    return oracle.query(db, patient, t1, t2, k, patient_mask=patient_mask)
