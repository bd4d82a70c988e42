"""Parity of the half-precision database path (thresholds chosen per query)
with the CPU oracle, which decodes binary16 with its own decoder.

Bar: bit-exact counts for every entry, score bits, arg-max and top-k order.
"""
import numpy as np
import pytest

import oracle
from paper_2205_04550_gb300 import DBQ_STORE_F16, Database, DbqError, _dbq, synth
from tests._gpu_helpers import assert_hits_equal, pack_bits_np, random_db, stream_oracle_counts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_2205_04550_gb300 import build
    build.build()
    return _t


def _f16_db(vols16, torch, device_input=False, n_params=0, params=None):
    n = vols16.shape[0]
    nz, ny, nx = vols16.shape[1:]
    db = Database((nx, ny, nz), n, DBQ_STORE_F16, n_params=n_params)
    bits = vols16.view(np.uint16)
    db.load(0, torch.from_numpy(bits.view(np.int16)).cuda() if device_input else bits,
            params=params)
    db.build()
    return db


def _thresholds(seed):
    rng = np.random.default_rng(seed)
    return np.float32(rng.uniform(0.5, 0.8)), np.float32(rng.uniform(0.15, 0.35))


CASES = [((1, 1, 1), 3, 3), ((9, 10, 11), 200, 10), ((8, 8, 8), 1500, 16),
         ((33, 31, 30), 300, 7), ((64, 64, 64), 170, 16), ((40, 40, 40), 400, 100)]


@pytest.mark.parametrize("shape,n,k", CASES)
def test_random_f16_counts_and_topk(torch, shape, n, k):
    vols, patient = random_db(shape, n, seed=7 * n + shape[0], plant=(n // 3,))
    v16 = vols.astype(np.float16)
    p16 = patient.astype(np.float16)
    t1, t2 = _thresholds(n)
    ref = oracle.query(v16, p16, t1, t2, k)
    with _f16_db(v16, torch, device_input=(n % 2 == 0)) as db:
        counts, pcount = db.scan_counts(p16.view(np.uint16), t1, t2)
        np.testing.assert_array_equal(pcount, ref["pcount"])
        np.testing.assert_array_equal(counts, ref["all_counts"])
        hits, _ = db.query(p16.view(np.uint16), k, t1, t2)
        assert_hits_equal(hits, ref, k)


def test_thresholds_on_and_between_binary16_values(torch):
    shape = (16, 16, 8)
    rng = np.random.default_rng(1)
    n = 64
    # values concentrated around the thresholds, plus specials
    base = np.float16(0.5)
    grid = (base + np.arange(-40, 40).astype(np.float16) * np.float16(2 ** -11)).astype(np.float16)
    v16 = rng.choice(grid, size=(n,) + shape[::-1]).astype(np.float16)
    flat = v16.reshape(n, -1).view(np.uint16)
    specials = np.array([0x7E00, 0xFE00, 0x8000, 0x0000, 0x7C00, 0xFC00, 0x0001, 0x3C00, 0xB800],
                        dtype=np.uint16)
    flat[:, :specials.size] = specials
    patient = rng.choice(grid, size=shape[::-1]).astype(np.float16)
    with _f16_db(v16, torch) as db:
        for t in (np.float32(0.5), np.float32(np.nextafter(np.float32(0.5), 1)),
                  np.float32(0.5 + 2 ** -11), np.float32(0.5 - 2 ** -12),
                  np.float32(0.49951172), np.float32(0.50048828), np.float32(1.0)):
            t2 = np.float32(0.25)
            ref = oracle.query(v16, patient, t, t2, 5)
            counts, _ = db.scan_counts(patient.view(np.uint16), t, t2)
            np.testing.assert_array_equal(counts, ref["all_counts"], err_msg=str(t))
            hits, _ = db.query(patient.view(np.uint16), 5, t, t2)
            assert_hits_equal(hits, ref, 5)


def test_f16_patient_kinds(torch):
    shape = (24, 20, 16)
    vols, patient = random_db(shape, 333, seed=3, plant=(100,))
    v16 = vols.astype(np.float16)
    t1, t2 = _thresholds(5)
    with _f16_db(v16, torch) as db:
        ref32 = oracle.query(v16, patient, t1, t2, 8)
        hits, _ = db.query(patient, 8, t1, t2)
        assert_hits_equal(hits, ref32, 8)
        m = oracle.threshold(patient, t1, t2)
        bits = pack_bits_np(m)
        refb = oracle.query(v16, patient, t1, t2, 8, patient_mask=m)
        hits, _ = db.query(torch.from_numpy(bits.view(np.int32)).cuda(), 8, t1, t2, kind=_dbq.DBQ_BITS)
        assert_hits_equal(hits, refb, 8)


def test_f16_surrogate_planted_best_match(torch):
    shape = (64, 64, 64)
    vols, theta = synth.database_np(shape, 300, dtype=np.float16)
    pat, _ = synth.patients_np(shape, [3], dtype=np.float16)
    vols[211] = pat[0]
    t1, t2 = np.float32(0.6), np.float32(0.25)
    ref = oracle.query(vols, pat[0], t1, t2, 16)
    assert ref["index"][0] == 211 and ref["score"][0] == 1.0
    with _f16_db(vols, torch, n_params=8, params=theta) as db:
        hits, params = db.query(pat[0].view(np.uint16), 16, t1, t2)
        assert_hits_equal(hits, ref, 16)
        np.testing.assert_array_equal(params, theta[ref["index"]])


def test_f16_errors(torch):
    v16 = np.zeros((4, 8, 8, 8), np.float16)
    with _f16_db(v16, torch) as db:
        for t1, t2 in ((0.0, 0.2), (0.6, 1.5), (float("nan"), 0.2)):
            with pytest.raises(DbqError) as e:
                db.query(v16[0].view(np.uint16), 1, t1, t2)
            assert e.value.status == _dbq.DBQ_EINVAL
        with pytest.raises(DbqError) as e:
            db.masks(0, 1)
        assert e.value.status == _dbq.DBQ_ESTATE


def test_f16_query_100000_entries_64cube_every_entry(torch):
    """Full size: 100,000 binary16 entries at 64^3 (52 GB), per-query
    thresholds t1 ~ U(0.5, 0.8), t2 ~ U(0.15, 0.35), top-16; the oracle
    counts every entry of both queries from the same binary16 values."""
    shape = (64, 64, 64)
    n, k, chunk = 100_000, 16, 64
    nx, ny, nz = shape
    gen = synth.DeviceGenerator(shape, synth.DB_SEED, np.arange(n))
    db = Database(shape, n, DBQ_STORE_F16, n_params=8)
    try:
        buf = torch.empty((chunk, nz, ny, nx), dtype=torch.float16, device="cuda")
        for c0 in range(0, n, chunk):
            cn = min(chunk, n - c0)
            gen.fill(c0, cn, buf)
            _dbq.db_load_volumes(db.handle, c0, cn, buf, kind=_dbq.DBQ_F16,
                                 params=gen.theta[c0:c0 + cn])
        db.build()
        pat, _ = synth.patients_np(shape, [2], dtype=np.float16)
        p16 = pat[0].view(np.uint16)
        queries, gpu = [], []
        for q in range(2):
            t1, t2 = _thresholds(100 + q)
            hits, params = db.query(p16, k, t1, t2)
            counts, pcount = db.scan_counts(p16, t1, t2)
            pmask = oracle.threshold(pat[0], t1, t2)
            np.testing.assert_array_equal(pcount, pmask.sum(axis=1))
            queries.append((pmask, t1, t2))
            gpu.append((hits, params, counts))
        refs = stream_oracle_counts(shape, n, queries, dtype="float16", chunk=2048)
        for (pmask, _, _), (hits, params, counts), ref_counts in zip(queries, gpu, refs):
            np.testing.assert_array_equal(counts, ref_counts)
            pc = pmask.sum(axis=1).astype(np.uint32)
            idx, val = oracle.rank(oracle.scores(ref_counts, pc), k)
            ref = {"index": idx, "score": val,
                   "counts": np.concatenate([ref_counts[idx], np.tile(pc, (k, 1))], axis=1)}
            assert_hits_equal(hits, ref, k)
            np.testing.assert_array_equal(params, gen.theta[idx])
    finally:
        db.close()
