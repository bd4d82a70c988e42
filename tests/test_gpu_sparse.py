"""The sparse exact scan (DBQ_OPT_SPARSE): reading only the words where the
patient's masks are non-zero must give exactly the counts, scores and order
of the full loop (Section 2.3: the Dice numerator only involves the
patient's voxels).  Bit-exact against the oracle and against the dense scan."""
import numpy as np
import pytest

import oracle
from paper_2205_04550_gb300 import (DBQ_MODE_EMBED_BF16, DBQ_STORE_BITS, Database, _dbq,
                                    synth)
from tests._gpu_helpers import assert_hits_equal, random_db

pytestmark = pytest.mark.gpu

T1, T2 = np.float32(0.6), np.float32(0.25)


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_2205_04550_gb300 import build
    build.build()
    return _t


CASES = [((1, 1, 1), 5, 5), ((9, 10, 11), 153, 10), ((17, 5, 3), 300, 300),
         ((33, 31, 30), 500, 7), ((64, 64, 64), 160, 12), ((128, 32, 32), 90, 9)]


def _sparse_patient(shape, seed, frac=0.1):
    """A patient whose masks cover a small box of the grid."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    p = np.zeros((nz, ny, nx), np.float32)
    z0, y0, x0 = (rng.integers(0, max(1, d // 2)) for d in (nz, ny, nx))
    dz, dy, dx = (max(1, int(d * frac ** (1 / 3))) for d in (nz, ny, nx))
    p[z0:z0 + dz, y0:y0 + dy, x0:x0 + dx] = rng.random((min(dz, nz - z0), min(dy, ny - y0),
                                                         min(dx, nx - x0)), dtype=np.float32)
    return p


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("shape,n,k", CASES)
def test_sparse_equals_oracle(torch, shape, n, k, mode):
    vols, _ = random_db(shape, n, seed=n)
    with Database(shape, n, DBQ_STORE_BITS, T1, T2) as db:
        db.load(0, vols)
        db.build()
        db.set_sparse(mode)
        for seed in range(3):
            patient = _sparse_patient(shape, seed)
            ref = oracle.query(vols, patient, T1, T2, k)
            counts, pcount = db.scan_counts(patient)
            np.testing.assert_array_equal(counts, ref["all_counts"])
            hits, _ = db.query(patient, k)
            assert_hits_equal(hits, ref, k)


@pytest.mark.parametrize("mode", [1, 2])
def test_sparse_empty_and_full_patients(torch, mode):
    shape = (32, 16, 8)
    vols, _ = random_db(shape, 200, seed=4)
    vols[17] = 0.0
    vols[18] = 0.0
    with Database(shape, 200, DBQ_STORE_BITS, T1, T2) as db:
        db.load(0, vols)
        db.build()
        db.set_sparse(mode)
        for patient in (np.zeros(shape[::-1], np.float32), np.ones(shape[::-1], np.float32)):
            ref = oracle.query(vols, patient, T1, T2, 20)
            hits, _ = db.query(patient, 20)
            assert_hits_equal(hits, ref, 20)
            l1, l2 = _dbq.db_last_support(db.handle)
            words = db.info()["padded_words"] // 4
            if patient.any():
                assert l1 == l2 == words
            else:
                assert l1 == l2 == 0
        # an empty patient against empty entries: Dice 1 for both, lowest index first
        hits, _ = db.query(np.zeros(shape[::-1], np.float32), 2)
        assert list(hits["index"]) == [17, 18] and hits["score"][0] == 1.0


def test_word_major_copy_follows_reloads(torch):
    """The word-major copy is rebuilt after entries are reloaded; every
    count and hit follows the new volumes (oracle), in every mode."""
    shape = (64, 32, 24)
    n = 3000                                    # 12 CTAs of counts, several slices
    vols, _ = random_db(shape, n, seed=31)
    pats = [_sparse_patient(shape, s, frac=f) for s, f in ((1, 0.05), (2, 0.3))]
    with Database(shape, n, DBQ_STORE_BITS, T1, T2) as db:
        db.load(0, vols)
        db.build()
        db.set_sparse(2)
        for p in pats:
            ref = oracle.query(vols, p, T1, T2, 40)
            hits, _ = db.query(p, 40)
            assert_hits_equal(hits, ref, 40)
        new, _ = random_db(shape, 500, seed=32)
        vols[1000:1500] = new
        vols[2999] = pats[1]                    # planted: must rank first
        db.load(1000, new)
        db.load(2999, pats[1][None])
        db.build()
        for p in pats:
            ref = oracle.query(vols, p, T1, T2, 40)
            counts, _ = db.scan_counts(p)
            np.testing.assert_array_equal(counts, ref["all_counts"])
            for mode in (2, 1, 0, 2):
                db.set_sparse(mode)
                hits, _ = db.query(p, 40)
                assert_hits_equal(hits, ref, 40)
        assert hits["index"][0] == 2999


def test_word_major_option_errors(torch):
    from paper_2205_04550_gb300 import DBQ_STORE_F16, DbqError
    with Database((8, 8, 8), 4, DBQ_STORE_F16) as db:
        with pytest.raises(DbqError, match="EINVAL"):
            _dbq.db_set_option(db.handle, _dbq.DBQ_OPT_SPARSE, 2)
    with Database((8, 8, 8), 4, DBQ_STORE_BITS, T1, T2) as db:
        for bad in (-1, 3):
            with pytest.raises(DbqError, match="EINVAL"):
                _dbq.db_set_option(db.handle, _dbq.DBQ_OPT_SPARSE, bad)


def test_sparse_toggle_and_surrogate(torch):
    shape = (64, 64, 64)
    vols, theta = synth.database_np(shape, 300)
    pats, _ = synth.patients_np(shape, [1, 2, 3])
    vols[77] = pats[2]
    with Database(shape, 300, DBQ_STORE_BITS, T1, T2, embed=True) as db:
        db.load(0, vols)
        db.build()
        for p in pats:
            dense, _ = db.query(p, 25)
            db.set_sparse(True)
            sparse, _ = db.query(p, 25)
            db.set_sparse(False)
            assert dense.tobytes() == sparse.tobytes()
            assert_hits_equal(sparse, oracle.query(vols, p, T1, T2, 25), 25)
        # re-ranking with support lists gives the same hits
        dense_b, _ = db.query_batch(list(pats), 10, DBQ_MODE_EMBED_BF16, 64)
        db.set_sparse(True)
        sparse_b, _ = db.query_batch(list(pats), 10, DBQ_MODE_EMBED_BF16, 64)
        exact_b, _ = db.query_batch(list(pats), 10)
        assert dense_b.tobytes() == sparse_b.tobytes()
        for q in range(3):
            assert_hits_equal(exact_b[q], oracle.query(vols, pats[q], T1, T2, 10), 10)
        assert sparse_b[2][0]["index"] == 77


def test_sparse_rerank_scheduling_many_queries(torch):
    """Sparse re-ranking takes its items largest support first from a device
    counter that must return to zero after every launch: many queries with
    supports from empty to the whole grid, launched repeatedly with different
    batch sizes, give the dense re-rank's hits bit for bit and the oracle's
    hits among the candidates."""
    shape = (64, 64, 32)
    n, c, k = 600, 96, 7
    vols, _ = synth.database_np(shape, n)
    pats = [_sparse_patient(shape, s, frac=f)
            for s, f in enumerate([0.002, 0.01, 0.05, 0.1, 0.3, 0.6] * 20)]
    pats[5] = np.zeros(shape[::-1], np.float32)
    pats[6] = np.ones(shape[::-1], np.float32)
    pats += list(synth.patients_np(shape, list(range(1, 31)))[0])
    vols[123] = pats[40]
    with Database(shape, n, DBQ_STORE_BITS, T1, T2, embed=True) as db:
        db.load(0, vols)
        db.build()
        dense, _ = db.query_batch(pats, k, DBQ_MODE_EMBED_BF16, c)
        _, cand = db.prefilter(pats, DBQ_MODE_EMBED_BF16, c)
        db.set_sparse(True)
        for sub in (pats, pats[:3], pats[100:], pats):
            sparse, _ = db.query_batch(sub, k, DBQ_MODE_EMBED_BF16, c)
            off = 100 if len(sub) == len(pats) - 100 else 0
            assert sparse.tobytes() == dense[off:off + len(sub)].tobytes()
    for q in (0, 5, 6, 40, 149):
        sorted_c = np.sort(cand[q])
        ref = oracle.query(vols[sorted_c], pats[q], T1, T2, k)
        ref["index"] = sorted_c[ref["index"]]
        assert_hits_equal(dense[q], ref, k)
    assert dense[40][0]["index"] == 123


def test_sparse_rerank_support_beyond_cache(torch):
    """A full patient on a 128 x 64 x 64 grid has 8,192 support positions,
    more than the shared-memory cache holds: that item falls back to the
    CTA-wide count loop while the others run one warp per entry."""
    shape = (128, 64, 64)
    n, c, k = 200, 40, 5
    vols, _ = synth.database_np(shape, n)
    pats = [np.ones(shape[::-1], np.float32)] + [_sparse_patient(shape, s) for s in range(9)]
    with Database(shape, n, DBQ_STORE_BITS, T1, T2, embed=True) as db:
        db.load(0, vols)
        db.build()
        dense, _ = db.query_batch(pats, k, DBQ_MODE_EMBED_BF16, c)
        db.set_sparse(True)
        for _ in range(2):
            sparse, _ = db.query_batch(pats, k, DBQ_MODE_EMBED_BF16, c)
            assert sparse.tobytes() == dense.tobytes()


@pytest.mark.parametrize("shape", [(128, 64, 32), (30, 17, 11)])
def test_support_lengths_follow_the_granule_definition(torch, shape):
    """The support lists hold every 16-byte word of each 64-byte granule of
    a plane where the patient's mask is non-zero (fewer words in a final
    partial granule): db_last_support against that count on the CPU."""
    nx, ny, nz = shape
    vols, _ = random_db(shape, 8, seed=1)
    with Database(shape, 8, DBQ_STORE_BITS, T1, T2) as db:
        db.load(0, vols)
        db.build()
        db.set_sparse(True)
        for seed in range(4):
            patient = _sparse_patient(shape, seed, frac=0.05 * (seed + 1))
            db.query(patient, 3)
            l1, l2 = _dbq.db_last_support(db.handle)
            v = nx * ny * nz
            wp4 = ((v + 31) // 32 + 3) // 4
            want = []
            for t in (T1, T2):
                m = np.zeros(wp4 * 128, bool)
                m[:v] = patient.reshape(-1) >= t
                word_nz = m.reshape(wp4, 128).any(axis=1)
                want.append(sum(min(4, wp4 - 4 * g) for g in range((wp4 + 3) // 4)
                                if word_nz[4 * g:4 * g + 4].any()))
            assert (l1, l2) == tuple(want), (seed, l1, l2, want)
