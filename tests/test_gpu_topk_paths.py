"""Every path of the fused top-k (csrc/topk.cuh) against the oracle's order
(Section 2.3 query: score descending, ties to the lowest index).

The path taken depends on k, on the entries per CTA and on the grid:
  * rounds of at most 64 offers: direct counts; larger rounds: the merge
    tree (k <= 64) or the bitonic sort (k > 64);
  * the grid's lists: one level of warp tournaments (k <= 16 when all lists
    fit the shared slots; one warp, or 32 lists per warp and then warp 0),
    else groups of 16 CTAs merged by tournaments (k <= 16), merge trees
    (k <= 64) or ranks, then the groups' lists the same way.
Equal scores are the hard case for all of them (keys compare equal and the
index decides: the tournaments' reduction falls through to the index words,
the trees' searches read the index), so the databases here are made of a few
distinct volumes repeated many times, in a shuffled order, with tiny grids so
that tens of thousands of entries stay cheap for the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2205_04550_gb300 import DBQ_STORE_BITS, DBQ_STORE_F16, Database
from tests._gpu_helpers import assert_hits_equal, random_db

pytestmark = pytest.mark.gpu

T1, T2 = np.float32(0.6), np.float32(0.25)
SHAPE = (8, 8, 8)


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_2205_04550_gb300 import build
    build.build()
    return _t


def _repeated(n, distinct, seed):
    """n entries drawn from `distinct` random volumes (shuffled), plus a patient."""
    base, patient = random_db(SHAPE, distinct, seed=seed)
    rng = np.random.default_rng(seed + 1)
    pick = rng.integers(0, distinct, size=n)
    return base[pick], patient


def _load(vols, storage):
    n = vols.shape[0]
    if storage == DBQ_STORE_BITS:
        db = Database(SHAPE, n, storage, T1, T2)
        db.load(0, vols)
    else:
        db = Database(SHAPE, n, storage)
        db.load(0, vols.view(np.uint16))
    db.build()
    return db


# (n, k): 2,500 entries = 16-17 per CTA (direct-count rounds); 20,000 = 131-132
# per CTA (one round of more than 64 offers: merge tree or bitonic); k on both
# sides of 16 (tournaments), 64 (trees) and 13 (152 lists of k fit the slots)
CASES = [(2500, 1), (2500, 10), (2500, 13), (2500, 14), (2500, 16), (2500, 17), (2500, 64),
         (2500, 65), (20000, 1), (20000, 10), (20000, 16), (20000, 17), (20000, 40),
         (20000, 64), (20000, 65), (20000, 200)]


@pytest.mark.parametrize("n,k", CASES)
def test_all_equal_scores(torch, n, k):
    vols, patient = random_db(SHAPE, 1, seed=3)
    db_vols = np.repeat(vols, n, axis=0)
    with _load(db_vols, DBQ_STORE_BITS) as db:
        hits, _ = db.query(patient, k)
    np.testing.assert_array_equal(hits["index"], np.arange(k))
    assert len(set(hits["score"].tolist())) == 1


@pytest.mark.parametrize("n,k", CASES)
def test_repeated_volumes_match_oracle(torch, n, k):
    vols, patient = _repeated(n, 37, seed=n + k)
    ref = oracle.query(vols, patient, T1, T2, k)
    with _load(vols, DBQ_STORE_BITS) as db:
        hits, _ = db.query(patient, k)
        assert_hits_equal(hits, ref, k)
        db.set_sparse(True)
        hits_s, _ = db.query(patient, k)
        assert hits_s.tobytes() == hits.tobytes()


@pytest.mark.parametrize("n,k", [(2500, 10), (2500, 16), (20000, 13), (20000, 40)])
def test_repeated_volumes_binary16(torch, n, k):
    vols, patient = _repeated(n, 23, seed=7 * k)
    v16 = vols.astype(np.float16)
    p16 = patient.astype(np.float16)
    ref = oracle.query(v16, p16, T1, T2, k)
    with _load(v16, DBQ_STORE_F16) as db:
        hits, _ = db.query(p16.view(np.uint16), k, T1, T2)
    assert_hits_equal(hits, ref, k)
