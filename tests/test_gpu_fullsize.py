"""Parity at the full workload sizes, in the launch configuration the
benchmark times.

* 1,024 entries at 64^3 (float32 surrogate volumes, t = 0.6 / 0.25, top-10):
  the oracle runs over the whole database; every count, the scores and the
  top-10 must match exactly.
* 50,000 entries at 128^3 bit-packed (top-64): the oracle counts every
  entry from the same volumes (streamed from the GPU generator through host
  memory in chunks); every count, the patient's sizes, the top-64 order and
  the hits' score bits must equal the oracle's own ranking of its own scores.
* The embedding batch at 100,000 entries of 128^3 (256 queries, 512
  candidates, top-10): the deduplicated and the per-query re-ranks give
  byte-identical hits, and for three queries the oracle counts every
  candidate from its volume and its top-10 of them equals the GPU's.
"""
import numpy as np
import pytest

import oracle
from paper_2205_04550_gb300 import DBQ_MODE_EMBED_BF16, DBQ_STORE_BITS, Database, synth
from tests._gpu_helpers import assert_hits_equal, stream_oracle_counts

pytestmark = pytest.mark.gpu

T1, T2 = np.float32(0.6), np.float32(0.25)


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_2205_04550_gb300 import build
    build.build()
    return _t


def _build_db_on_device(torch, shape, n, chunk, n_params=8, embed=False):
    db = Database(shape, n, DBQ_STORE_BITS, T1, T2, n_params, embed=embed)
    nx, ny, nz = shape
    gen = synth.DeviceGenerator(shape, synth.DB_SEED, np.arange(n))
    buf = torch.empty((chunk, nz, ny, nx), dtype=torch.float32, device="cuda")
    for c0 in range(0, n, chunk):
        cn = min(chunk, n - c0)
        gen.fill(c0, cn, buf)
        db.load(c0, buf[:cn], params=gen.theta[c0:c0 + cn])
    db.build()
    torch.cuda.synchronize()
    return db


def test_exact_query_1024_entries_64cube_full_oracle(torch):
    shape = (64, 64, 64)
    n, k = 1024, 10
    vols_dev, theta = synth.generate_device(shape, synth.DB_SEED, np.arange(n))
    vols = vols_dev.cpu().numpy()
    pat, _ = synth.patients_np(shape, [1])
    ref = oracle.query(vols, pat[0], T1, T2, k)
    with Database(shape, n, DBQ_STORE_BITS, T1, T2, 8) as db:
        db.load(0, vols_dev, params=theta)
        db.build()
        hits, params = db.query(pat[0], k)
        assert_hits_equal(hits, ref, k)
        np.testing.assert_array_equal(params, theta[ref["index"]])
        counts, pcount = db.scan_counts(pat[0])
        np.testing.assert_array_equal(counts, ref["all_counts"])
        np.testing.assert_array_equal(pcount, ref["pcount"])


def test_exact_query_50000_entries_128cube_every_entry(torch):
    shape = (128, 128, 128)
    n, k = 50_000, 64
    db = _build_db_on_device(torch, shape, n, chunk=8)
    try:
        pat, _ = synth.patients_np(shape, [1])
        patient = pat[0]
        hits, params = db.query(patient, k)
        counts, pcount = db.scan_counts(patient)
        pmask = oracle.threshold(patient, T1, T2)
        # the oracle over every entry, from the volumes themselves
        (ref_counts,) = stream_oracle_counts(shape, n, [(pmask, T1, T2)], chunk=256)
        np.testing.assert_array_equal(counts, ref_counts)
        np.testing.assert_array_equal(pcount, pmask.sum(axis=1))
        sc = oracle.scores(ref_counts, pmask.sum(axis=1).astype(np.uint32))
        idx, val = oracle.rank(sc, k)
        ref = {"index": idx, "score": val,
               "counts": np.concatenate([ref_counts[idx],
                                         np.tile(pmask.sum(axis=1), (k, 1))], axis=1)}
        assert_hits_equal(hits, ref, k)
        theta = synth.entry_params(shape, synth.DB_SEED, idx)
        np.testing.assert_array_equal(params, theta)
        # the sparse scan (patient support only) gives the identical result
        db.set_sparse(True)
        s_hits, _ = db.query(patient, k)
        s_counts, _ = db.scan_counts(patient)
        db.set_sparse(False)
        assert s_hits.tobytes() == hits.tobytes()
        np.testing.assert_array_equal(s_counts, counts)
    finally:
        db.close()


def test_embedding_batch_100000_entries_128cube(torch):
    shape = (128, 128, 128)
    nx, ny, nz = shape
    n, nq, c, k = 100_000, 256, 512, 10
    db = _build_db_on_device(torch, shape, n, chunk=8, embed=True)
    try:
        pgen = synth.DeviceGenerator(shape, synth.DB_SEED,
                                     synth.PATIENT_BASE + np.arange(1, nq + 1, dtype=np.uint64))
        pats = torch.empty((nq, nz, ny, nx), dtype=torch.float32, device="cuda")
        pgen.fill(0, nq, pats)
        plist = [pats[q] for q in range(nq)]
        _, cand = db.prefilter(plist, DBQ_MODE_EMBED_BF16, c)
        out = []
        for mode in (1, 2, 0):
            db.set_rerank(mode)
            out.append(db.query_batch(plist, k, DBQ_MODE_EMBED_BF16, c)[0])
        assert out[1].tobytes() == out[0].tobytes() and out[2].tobytes() == out[0].tobytes()
        hits = out[2]
        for q in (0, 100, 255):
            pm = oracle.threshold(pats[q].cpu().numpy(), T1, T2)
            psize = pm.sum(axis=1).astype(np.uint32)
            ents = np.sort(cand[q]).astype(np.int64)
            (ref_counts,) = stream_oracle_counts(shape, c, [(pm, T1, T2)], chunk=64, entries=ents)
            idx, val = oracle.rank(oracle.scores(ref_counts, psize), k)
            ref = {"index": ents[idx], "score": val,
                   "counts": np.concatenate([ref_counts[idx], np.tile(psize, (k, 1))], axis=1)}
            assert_hits_equal(hits[q], ref, k)
    finally:
        db.close()
