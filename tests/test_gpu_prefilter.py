"""Parity of the embedding prefilter (a6-a8) and of batched queries with the
CPU oracle.

* embeddings: bfloat16 bits, FP8 codes and row scales bit-exact; squared
  norms within 1e-5 relative (binary32 sums in a different order);
* tensor-core distances L = d_1 + d_2 against binary64 distances of the same
  decoded embeddings, within a tolerance from binary32 accumulation: per
  segmentation |d^2_gpu - d^2_ref| <= 2e-5 (|q|^2 + |e|^2) + 1e-6, hence
  |L_gpu - L_ref| <= sum_k sqrt(that bound);
* candidate sets: equal to the oracle's closest entries except where a
  distance lies inside the tolerance of the cut;
* re-ranked hits: bit-exact counts, scores and order among the candidates;
* batched exact queries: identical to one-at-a-time queries.
"""
import numpy as np
import pytest

import oracle
from paper_2205_04550_gb300 import (DBQ_MODE_EMBED_BF16, DBQ_MODE_EMBED_FP8, DBQ_MODE_EXACT,
                                    DBQ_STORE_BITS, DBQ_STORE_F16, Database, DbqError, _dbq,
                                    synth)
from tests._gpu_helpers import assert_hits_equal, random_db

pytestmark = pytest.mark.gpu

T1, T2 = np.float32(0.6), np.float32(0.25)
REL = 2e-5


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_2205_04550_gb300 import build
    build.build()
    return _t


def _oracle_embed(vol, shape):
    """Oracle embeddings of one volume: bf16 bits, e4m3 codes, scales for
    both segmentations, and decoded binary64 vectors."""
    nx, ny, nz = shape
    m = oracle.threshold(vol, T1, T2)
    out = {"bf16": [], "e4m3": [], "scale": [], "vb": [], "vf": []}
    for k in range(2):
        b, q, s = oracle.embed(m[k], nx, ny, nz)
        out["bf16"].append(b)
        out["e4m3"].append(q)
        out["scale"].append(s)
        out["vb"].append(oracle.bf16_to_f64(b))
        out["vf"].append(oracle.e4m3_to_f64(q) * np.float64(s))
    return {key: np.array(v) for key, v in out.items()}


def _ref_dist(qe, ee, key):
    """L = d_1 + d_2 in binary64 and the tolerance of the binary32 GPU value."""
    L, tol = 0.0, 0.0
    for k in range(2):
        a, b = qe[key][k], ee[key][k]
        L += np.sqrt(np.sum((a - b) ** 2))
        tol += np.sqrt(REL * (np.sum(a * a) + np.sum(b * b)) + 1e-6)
    return L, tol


def _surrogate(shape, n, nq, plant=()):
    vols, theta = synth.database_np(shape, n)
    pats, _ = synth.patients_np(shape, list(range(1, nq + 1)))
    for j, q in plant:
        vols[j] = pats[q]
    return vols, pats, theta


@pytest.mark.parametrize("shape", [(32, 16, 24), (64, 64, 64), (128, 64, 32)])
def test_embeddings_bit_exact(torch, shape):
    n = 40
    vols, _ = random_db(shape, n, seed=shape[1], p_zero=0.3)
    vols[:10] *= np.float32(0.7)          # some rows with few voxels above t1
    vols[10] = 0.0                         # an empty row: scale 1
    with Database(shape, n, DBQ_STORE_BITS, T1, T2, embed=True) as db:
        db.load(0, vols)
        db.build()
        got = db.embeddings(0, n)
    for e in range(n):
        ref = _oracle_embed(vols[e], shape)
        np.testing.assert_array_equal(got["bf16"][e], ref["bf16"], err_msg=str(e))
        np.testing.assert_array_equal(got["e4m3"][e], ref["e4m3"], err_msg=str(e))
        np.testing.assert_array_equal(got["scale"][e], ref["scale"].astype(np.float32))
        nb = np.sum(ref["vb"] ** 2, axis=1)
        nf = np.sum(ref["vf"] ** 2, axis=1)
        np.testing.assert_allclose(got["norm_bf16"][e], nb, rtol=1e-5, atol=1e-9)
        np.testing.assert_allclose(got["norm_fp8"][e], nf, rtol=1e-5, atol=1e-9)


@pytest.mark.parametrize("mode,key", [(DBQ_MODE_EMBED_BF16, "vb"), (DBQ_MODE_EMBED_FP8, "vf")])
def test_prefilter_distances_and_candidates(torch, mode, key):
    shape = (64, 64, 64)
    n, nq, c = 700, 7, 64
    vols, pats, _ = _surrogate(shape, n, nq, plant=((123, 0), (650, 3)))
    with Database(shape, n, DBQ_STORE_BITS, T1, T2, embed=True) as db:
        db.load(0, vols)
        db.build()
        dist, cand = db.prefilter(list(pats), mode, c)
    ents = [_oracle_embed(vols[e], shape) for e in range(n)]
    for q in range(nq):
        qe = _oracle_embed(pats[q], shape)
        ref = np.zeros(n)
        tol = np.zeros(n)
        for e in range(n):
            ref[e], tol[e] = _ref_dist(qe, ents[e], key)
        err = np.abs(dist[q].astype(np.float64) - ref)
        assert np.all(err <= tol + 1e-5 * ref), (q, float(err.max()))
        order = np.lexsort((np.arange(n), ref))
        want = set(order[:c].tolist())
        got = cand[q].tolist()
        assert len(set(got)) == c
        # ascending by the GPU distance
        assert np.all(np.diff(dist[q][got]) >= 0)
        cut = ref[order[c - 1]]
        for e in want.symmetric_difference(got):
            assert abs(ref[e] - cut) <= 2 * (tol[e] + tol[order[c - 1]]) + 1e-5 * cut, (q, e)
    # planted copies are at distance ~0 and come first
    assert cand[0][0] == 123 and cand[3][0] == 650


@pytest.mark.parametrize("mode", [DBQ_MODE_EMBED_BF16, DBQ_MODE_EMBED_FP8])
def test_embed_rerank_hits_exact_on_candidates(torch, mode):
    shape = (64, 64, 64)
    n, nq, c, k = 900, 6, 128, 10
    vols, pats, theta = _surrogate(shape, n, nq, plant=((42, 1),))
    with Database(shape, n, DBQ_STORE_BITS, T1, T2, n_params=8, embed=True) as db:
        db.load(0, vols, params=theta)
        db.build()
        _, cand = db.prefilter(list(pats), mode, c)
        hits, params = db.query_batch(list(pats), k, mode, c)
    for q in range(nq):
        ref = oracle.query(vols[np.sort(cand[q])], pats[q], T1, T2, k)
        # map the oracle's positions in the sorted candidate list back to entries
        sorted_c = np.sort(cand[q])
        ref["index"] = sorted_c[ref["index"]]
        assert_hits_equal(hits[q], ref, k)
        np.testing.assert_array_equal(params[q], theta[ref["index"]])
    assert hits[1][0]["index"] == 42 and hits[1][0]["score"] == 1.0


def test_embed_all_candidates_equals_exact_scan(torch):
    shape = (64, 32, 64)          # 256 embedding dims: both encodings tile
    n, k = 200, 15
    vols, pats, _ = _surrogate(shape, n, 3)
    with Database(shape, n, DBQ_STORE_BITS, T1, T2, embed=True) as db:
        db.load(0, vols)
        db.build()
        for mode in (DBQ_MODE_EMBED_BF16, DBQ_MODE_EMBED_FP8):
            hits, _ = db.query_batch(list(pats), k, mode, n)
            for q in range(3):
                assert_hits_equal(hits[q], oracle.query(vols, pats[q], T1, T2, k), k)


def test_batch_exact_two_databases_interleaved(torch):
    s1, s2 = (32, 32, 32), (64, 32, 16)
    v1, p1 = random_db(s1, 300, seed=1)
    v2, p2 = random_db(s2, 170, seed=2)
    v3 = v2.astype(np.float16)
    rng = np.random.default_rng(3)
    pats1 = [np.ascontiguousarray(x) for x in rng.permutation(v1)[:5]]
    pats2 = [np.ascontiguousarray(x) for x in rng.permutation(v2)[:4]]
    with Database(s1, 300, DBQ_STORE_BITS, T1, T2) as d1, \
            Database(s2, 170, DBQ_STORE_BITS, T1, T2) as d2:
        d1.load(0, v1)
        d1.build()
        d2.load(0, v2)
        d2.build()
        patients, which = [], []
        for i in range(4):
            patients += [pats1[i], pats2[i]]
            which += [0, 1]
        patients.append(pats1[4])
        which.append(0)
        hits, _ = _dbq.db_query_batch([d1.handle, d2.handle], which, patients, 12,
                                      DBQ_MODE_EXACT)
        for q, (p, w) in enumerate(zip(patients, which)):
            vols = v1 if w == 0 else v2
            assert_hits_equal(hits[q], oracle.query(vols, p, T1, T2, 12), 12)
    # a binary16 database with per-query thresholds in the same call
    with Database(s2, 170, DBQ_STORE_F16) as d3:
        d3.load(0, v3.view(np.uint16))
        d3.build()
        t1 = np.array([0.55, 0.7], np.float32)
        t2 = np.array([0.2, 0.3], np.float32)
        ps = [p2.astype(np.float16).view(np.uint16), v3[5].view(np.uint16).copy()]
        hits, _ = _dbq.db_query_batch([d3.handle], [0, 0], ps, 9, DBQ_MODE_EXACT, t1=t1, t2=t2)
        for q in range(2):
            assert_hits_equal(hits[q], oracle.query(v3, ps[q], t1[q], t2[q], 9), 9)


def test_batch_more_than_one_group_and_device_patients(torch):
    shape = (32, 32, 32)
    n, nq, k, c = 150, 300, 5, 40
    vols, _ = random_db(shape, n, seed=8)
    pats = vols[np.random.default_rng(0).integers(0, n, nq)]
    dev = torch.from_numpy(pats).cuda()
    with Database(shape, n, DBQ_STORE_BITS, T1, T2, embed=True) as db:
        db.load(0, vols)
        db.build()
        hits, _ = db.query_batch([dev[q] for q in range(nq)], k, DBQ_MODE_EMBED_BF16, c)
        ex, _ = db.query_batch([pats[q] for q in range(nq)], k, DBQ_MODE_EXACT)
    for q in range(0, nq, 37):
        assert_hits_equal(ex[q], oracle.query(vols, pats[q], T1, T2, k), k)
    # every patient is an entry: its copy (or an equal-scoring lower index) wins
    assert np.all(hits[:, 0]["score"] == 1.0) and np.all(ex[:, 0]["score"] == 1.0)


def test_prefilter_errors(torch):
    vols, pat = random_db((32, 32, 32), 20, seed=1)
    with Database((32, 32, 32), 20, DBQ_STORE_BITS, T1, T2) as db:
        db.load(0, vols)
        db.build()
        with pytest.raises(DbqError) as e:
            db.query_batch([pat], 3, DBQ_MODE_EMBED_BF16, 10)
        assert e.value.status == _dbq.DBQ_ESTATE
    with pytest.raises(DbqError):
        Database((40, 16, 16), 4, DBQ_STORE_BITS, T1, T2, embed=True)   # nx not a multiple of 32
    with pytest.raises(DbqError):
        Database((32, 32, 32), 4, DBQ_STORE_F16, embed=True)
    with Database((32, 32, 32), 20, DBQ_STORE_BITS, T1, T2, embed=True) as db:
        db.load(0, vols)
        db.build()
        for k, c in ((5, 4), (1, 21), (1, 0)):
            with pytest.raises(DbqError) as e:
                db.query_batch([pat], k, DBQ_MODE_EMBED_BF16, c)
            assert e.value.status == _dbq.DBQ_ERANGE
        with pytest.raises(DbqError) as e:           # 64 dims do not tile FP8's 128-byte K
            db.query_batch([pat], 1, DBQ_MODE_EMBED_FP8, 10)
        assert e.value.status == _dbq.DBQ_EINVAL


@pytest.mark.parametrize("dup", [0, 250])
def test_candidates_are_the_smallest_gpu_distances_with_index_ties(torch, dup):
    """Selection property on the GPU's own distances: the candidates are the
    c smallest under (distance, index), ascending -- including a cut inside a
    large group of equal distances (identical entries)."""
    shape = (64, 32, 64)
    n, c = 1200, 64
    vols, pats, _ = _surrogate(shape, n, 4)
    if dup:
        vols[300:300 + dup] = vols[299]
    with Database(shape, n, DBQ_STORE_BITS, T1, T2, embed=True) as db:
        db.load(0, vols)
        db.build()
        for mode in (DBQ_MODE_EMBED_BF16, DBQ_MODE_EMBED_FP8):
            pq = list(pats) + [vols[299].copy()]
            dist, cand = db.prefilter(pq, mode, c)
            for q in range(len(pq)):
                want = np.lexsort((np.arange(n), dist[q]))[:c]
                np.testing.assert_array_equal(cand[q], want)
    if dup:
        # the copy of entry 299 sees dup + 1 equal best distances: lowest indices first
        assert list(want[:dup + 1][:c]) == list(range(299, 299 + min(c, dup + 1)))
