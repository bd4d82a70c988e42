"""Parity of the deduplicated re-ranking of embedding batches
(rerank_dedupe.cu) with the per-query re-ranking and with the CPU oracle.

Both passes count |P_k n E_k| exactly and rank by the same total order
(binary64 Dice sum, ties to the lower index), so their hits must agree
field by field; the oracle, scanning each query's candidate entries, pins
both.  The cases cover plane slices cut short by the plane's end, the
largest batch (256 queries x 1,024 candidates), entries picked by more
queries than a warp has lanes, and a single query.
"""
import numpy as np
import pytest

import oracle
from paper_2205_04550_gb300 import (DBQ_MODE_EMBED_BF16, DBQ_MODE_HASH, DBQ_OPT_RERANK,
                                    DBQ_STORE_BITS, Database, DbqError, db_set_option, synth)
from tests._gpu_helpers import assert_hits_equal

pytestmark = pytest.mark.gpu

T1, T2 = np.float32(0.6), np.float32(0.25)


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_2205_04550_gb300 import build
    build.build()
    return _t


def _all_modes(db, pats, k, mode, c):
    """Hits and parameters of the three DBQ_OPT_RERANK settings; all equal."""
    out = []
    for m in (1, 0, 2):
        db.set_rerank(m)
        out.append(db.query_batch(pats, k, mode, c))
    db.set_rerank(0)
    (h1, p1), (h0, p0), (h2, p2) = out
    assert h0.tobytes() == h1.tobytes() and h2.tobytes() == h1.tobytes()
    np.testing.assert_array_equal(p0, p1)
    np.testing.assert_array_equal(p2, p1)
    return h0, p0


def _oracle_on_candidates(vols, pat, cand_q, k):
    sorted_c = np.sort(cand_q)
    ref = oracle.query(vols[sorted_c], pat, T1, T2, k)
    ref["index"] = sorted_c[ref["index"]]
    return ref


def test_ragged_slices_shared_candidates(torch):
    # 30,720 voxels: 240 16-byte words per plane, 7.5 slices of 32
    shape = (32, 24, 40)
    n, nq, c, k = 700, 48, 200, 12
    vols, theta = synth.database_np(shape, n)
    pats, _ = synth.patients_np(shape, list(range(1, nq // 2 + 1)))
    rng = np.random.default_rng(5)
    copies = vols[rng.choice(n, nq - nq // 2, replace=False)]
    pats = np.concatenate([pats, copies])
    with Database(shape, n, DBQ_STORE_BITS, T1, T2, n_params=8, sketch=True) as db:
        db.load(0, vols, params=theta)
        db.build()
        _, cand = db.prefilter(list(pats), DBQ_MODE_HASH, c)
        hits, params = _all_modes(db, list(pats), k, DBQ_MODE_HASH, c)
    pairs = cand.size
    assert np.unique(cand).size < pairs        # the queries do share candidates
    for q in (0, 7, 23, 24, 30, 47):
        ref = _oracle_on_candidates(vols, pats[q], cand[q], k)
        assert_hits_equal(hits[q], ref, k)
        np.testing.assert_array_equal(params[q], theta[ref["index"]])
    for q in range(nq // 2, nq):               # a copy of an entry finds it
        assert hits[q][0]["score"] == 1.0


def test_largest_batch(torch):
    shape = (32, 32, 32)                       # 64 embedding dims
    n, nq, c, k = 1100, 256, 1024, 40
    vols, _ = synth.database_np(shape, n)
    pats, _ = synth.patients_np(shape, list(range(1, nq + 1)))
    with Database(shape, n, DBQ_STORE_BITS, T1, T2, embed=True) as db:
        db.load(0, vols)
        db.build()
        _, cand = db.prefilter(list(pats), DBQ_MODE_EMBED_BF16, c)
        hits, _ = _all_modes(db, list(pats), k, DBQ_MODE_EMBED_BF16, c)
    for q in (0, 101, 255):
        assert_hits_equal(hits[q], _oracle_on_candidates(vols, pats[q], cand[q], k), k)


def test_every_entry_picked_by_every_query(torch):
    # 40 identical queries whose candidates are all 300 entries: each entry
    # has a run of 40 pairs (more than one warp-wide window); 1.5 slices
    shape = (32, 8, 24)
    n, nq, k = 300, 40, 25
    vols, _ = synth.database_np(shape, n)
    pat, _ = synth.patients_np(shape, [3])
    pats = [pat[0]] * nq
    with Database(shape, n, DBQ_STORE_BITS, T1, T2, sketch=True) as db:
        db.load(0, vols)
        db.build()
        hits, _ = _all_modes(db, pats, k, DBQ_MODE_HASH, n)
    ref = oracle.query(vols, pat[0], T1, T2, k)
    for q in (0, 19, 39):
        assert_hits_equal(hits[q], ref, k)


def test_single_query(torch):
    shape = (32, 32, 32)
    n, c, k = 500, 300, 7
    vols, _ = synth.database_np(shape, n)
    pats, _ = synth.patients_np(shape, [9])
    with Database(shape, n, DBQ_STORE_BITS, T1, T2, embed=True) as db:
        db.load(0, vols)
        db.build()
        _, cand = db.prefilter(list(pats), DBQ_MODE_EMBED_BF16, c)
        hits, _ = _all_modes(db, list(pats), k, DBQ_MODE_EMBED_BF16, c)
    assert_hits_equal(hits[0], _oracle_on_candidates(vols, pats[0], cand[0], k), k)


def test_option_errors(torch):
    with Database((32, 8, 8), 4, DBQ_STORE_BITS, T1, T2) as db:
        for bad in (-1, 3):
            with pytest.raises(DbqError):
                db_set_option(db.handle, DBQ_OPT_RERANK, bad)
        db_set_option(db.handle, DBQ_OPT_RERANK, 1)
