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


def stream_oracle_counts(shape, n, queries, dtype="float32", chunk=256, seed=synth.DB_SEED,
                         entries=None):
    """The oracle's per-entry counts over a whole surrogate database that is
    too large to hold on the host: the same seeded volumes the database was
    built from are generated on the GPU chunk by chunk, copied into pinned
    host memory, and counted by ``oracle.counts`` on all host cores by one
    worker thread while the next chunk is generated and copied (ctypes
    releases the GIL during the oracle's C call).

    queries: list of (patient mask [2][V] uint8, t1, t2).  entries: the entry
    ids counted (default 0 .. n-1; n is then len(entries)).
    Returns one [n, 4] uint32 array (I1, I2, E1, E2) per query, row i for the
    i-th entry.
    """
    import queue
    import threading

    import torch

    nx, ny, nz = shape
    tdt = torch.float16 if dtype == "float16" else torch.float32
    if entries is not None:
        n = len(entries)
    gen = synth.DeviceGenerator(shape, seed, np.arange(n) if entries is None else entries)
    dev = torch.empty((chunk, nz, ny, nx), dtype=tdt, device="cuda")
    host = [torch.empty((chunk, nz, ny, nx), dtype=tdt, pin_memory=True) for _ in range(2)]
    free = [threading.Semaphore(1) for _ in range(2)]     # host buffer not in use by the oracle
    work = queue.Queue()
    out = [np.zeros((n, 4), dtype=np.uint32) for _ in queries]
    errors = []

    def worker():
        while True:
            item = work.get()
            if item is None:
                return
            buf, c0, cn = item
            try:
                vols = host[buf][:cn].numpy()
                if dtype == "float16":
                    vols = vols.view(np.uint16)
                for qi, (pm, t1, t2) in enumerate(queries):
                    cnt, _ = oracle.counts(vols, pm, t1, t2)
                    out[qi][c0:c0 + cn] = cnt
            except Exception as exc:  # pragma: no cover - surfaced below
                errors.append(exc)
            free[buf].release()

    th = threading.Thread(target=worker)
    th.start()
    try:
        for i, c0 in enumerate(range(0, n, chunk)):
            buf = i & 1
            cn = min(chunk, n - c0)
            gen.fill(c0, cn, dev)
            free[buf].acquire()
            host[buf][:cn].copy_(dev[:cn])
            torch.cuda.synchronize()
            work.put((buf, c0, cn))
    finally:
        work.put(None)
        th.join()
    if errors:
        raise errors[0]
    return out
