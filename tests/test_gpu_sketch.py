"""Parity of the random-projection embeddings and the Hamming prefilter
(count sketch of each mask, its sign code) with the CPU oracle.

* sketch embeddings: bfloat16 bits, FP8 codes, row scales and sign codes
  bit-exact against oracle.sketch / encode_values / sign_code, on grids
  whose voxel count is and is not a multiple of 32, with an empty row;
  squared norms within 1e-5 relative (binary32 sums in another order);
* Hamming distances: exact integers, equal to oracle.hamming summed over
  both segmentations; candidates: exactly the c smallest by (distance,
  index), ascending;
* re-ranked hits of DBQ_MODE_HASH: bit-exact among the candidates;
* the L2 modes on a sketch database: distances within the binary32
  tolerance of the binary64 distances of the decoded sketches;
* flag and mode errors.
"""
import numpy as np
import pytest

import oracle
from paper_2205_04550_gb300 import (DBQ_MODE_EMBED_BF16, DBQ_MODE_EMBED_FP8, DBQ_MODE_HASH,
                                    DBQ_STORE_BITS, DBQ_STORE_F16, SKETCH_DIMS, Database,
                                    DbqError, _dbq, synth)
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


def _oracle_sketch(vol):
    """Oracle sketches of one volume, both segmentations: int32 [2][D],
    sign codes [2][D/32]."""
    m = oracle.threshold(vol, T1, T2)
    sk = np.stack([oracle.sketch(m[k], SKETCH_DIMS) for k in range(2)])
    codes = np.stack([oracle.sign_code(sk[k]) for k in range(2)])
    return sk, codes


def _surrogate(shape, n, nq, plant=()):
    vols, theta = synth.database_np(shape, n)
    pats, _ = synth.patients_np(shape, list(range(1, nq + 1)))
    for j, q in plant:
        vols[j] = pats[q]
    return vols, pats, theta


@pytest.mark.parametrize("shape", [(32, 16, 24), (30, 17, 11)])
def test_sketch_embeddings_and_codes_bit_exact(torch, shape):
    n = 12
    vols, _ = random_db(shape, n, seed=shape[2], p_zero=0.3)
    vols[:4] *= np.float32(0.7)
    vols[5] = 0.0                          # empty masks: zero sketch, scale 1
    with Database(shape, n, DBQ_STORE_BITS, T1, T2, sketch=True) as db:
        db.load(0, vols)
        db.build()
        got = db.embeddings(0, n)
        codes = db.codes(0, n)
    for e in range(n):
        sk, ref_codes = _oracle_sketch(vols[e])
        np.testing.assert_array_equal(codes[e], ref_codes, err_msg=str(e))
        for k in range(2):
            bf, q, s = oracle.encode_values(sk[k])
            np.testing.assert_array_equal(got["bf16"][e, k], bf, err_msg=f"{e},{k}")
            np.testing.assert_array_equal(got["e4m3"][e, k], q, err_msg=f"{e},{k}")
            assert got["scale"][e, k] == s, (e, k)
            vb = oracle.bf16_to_f64(bf)
            vf = oracle.e4m3_to_f64(q) * np.float64(s)
            np.testing.assert_allclose(got["norm_bf16"][e, k], np.sum(vb * vb), rtol=1e-5)
            np.testing.assert_allclose(got["norm_fp8"][e, k], np.sum(vf * vf), rtol=1e-5)
    assert not codes[5].any() and got["scale"][5].tolist() == [1.0, 1.0]


def test_hamming_distances_and_candidates_exact(torch):
    shape = (64, 64, 64)
    n, nq, c = 700, 7, 64
    vols, pats, _ = _surrogate(shape, n, nq, plant=((123, 0), (650, 3)))
    with Database(shape, n, DBQ_STORE_BITS, T1, T2, sketch=True) as db:
        db.load(0, vols)
        db.build()
        dist, cand = db.prefilter(list(pats), DBQ_MODE_HASH, c)
    ent = [_oracle_sketch(vols[e])[1] for e in range(n)]
    for q in range(nq):
        qc = _oracle_sketch(pats[q])[1]
        ref = np.array([oracle.hamming(qc, ent[e]) for e in range(n)], dtype=np.float64)
        np.testing.assert_array_equal(dist[q].astype(np.float64), ref, err_msg=str(q))
        order = np.lexsort((np.arange(n), ref))
        np.testing.assert_array_equal(cand[q], order[:c], err_msg=str(q))
    assert cand[0][0] == 123 and cand[3][0] == 650
    assert dist[0][123] == 0 and dist[3][650] == 0


@pytest.mark.parametrize("nq", [1, 37])
def test_hash_rerank_hits_exact_on_candidates(torch, nq):
    shape = (64, 48, 40)
    n, c, k = 900, 128, 10
    vols, pats, theta = _surrogate(shape, n, nq, plant=((42, 0),))
    with Database(shape, n, DBQ_STORE_BITS, T1, T2, n_params=8, sketch=True) as db:
        db.load(0, vols, params=theta)
        db.build()
        _, cand = db.prefilter(list(pats), DBQ_MODE_HASH, c)
        hits, params = db.query_batch(list(pats), k, DBQ_MODE_HASH, c)
    for q in range(nq):
        sorted_c = np.sort(cand[q])
        ref = oracle.query(vols[sorted_c], pats[q], T1, T2, k)
        ref["index"] = sorted_c[ref["index"]]
        assert_hits_equal(hits[q], ref, k)
        np.testing.assert_array_equal(params[q], theta[ref["index"]])
    assert hits[0]["index"][0] == 42 and hits[0]["score"][0] == 1.0


@pytest.mark.parametrize("mode", [DBQ_MODE_EMBED_BF16, DBQ_MODE_EMBED_FP8])
def test_sketch_l2_prefilter_distances(torch, mode):
    shape = (64, 64, 32)
    n, nq, c = 300, 3, 32
    vols, pats, _ = _surrogate(shape, n, nq, plant=((77, 2),))
    with Database(shape, n, DBQ_STORE_BITS, T1, T2, sketch=True) as db:
        db.load(0, vols)
        db.build()
        dist, cand = db.prefilter(list(pats), mode, c)

    def decoded(vol):
        sk, _ = _oracle_sketch(vol)
        rows = []
        for k in range(2):
            bf, q, s = oracle.encode_values(sk[k])
            rows.append(oracle.bf16_to_f64(bf) if mode == DBQ_MODE_EMBED_BF16
                        else oracle.e4m3_to_f64(q) * np.float64(s))
        return rows

    ents = [decoded(vols[e]) for e in range(n)]
    for q in range(nq):
        qe = decoded(pats[q])
        for e in range(n):
            L, tol = 0.0, 0.0
            for k in range(2):
                a, b = qe[k], ents[e][k]
                L += np.sqrt(np.sum((a - b) ** 2))
                tol += np.sqrt(REL * (np.sum(a * a) + np.sum(b * b)) + 1e-6)
            assert abs(float(dist[q][e]) - L) <= tol + 1e-5 * L, (q, e)
    assert cand[2][0] == 77


def test_sketch_flag_and_mode_errors(torch):
    shape = (32, 8, 8)
    with pytest.raises(DbqError, match="EINVAL"):
        _dbq.db_create(*shape, 4, DBQ_STORE_BITS, 0.6, 0.25, 0,
                       _dbq.DBQ_FLAG_EMBED | _dbq.DBQ_FLAG_SKETCH)
    with pytest.raises(DbqError, match="EINVAL"):
        _dbq.db_create(*shape, 4, DBQ_STORE_F16, 0.6, 0.25, 0, _dbq.DBQ_FLAG_SKETCH)
    vols, pat = random_db(shape, 4, seed=3)
    with Database(shape, 4, DBQ_STORE_BITS, T1, T2, embed=True) as db:
        db.load(0, vols)
        db.build()
        with pytest.raises(DbqError, match="ESTATE"):
            db.prefilter([pat], DBQ_MODE_HASH, 2)
        with pytest.raises(DbqError, match="ESTATE"):
            db.codes(0, 1)
