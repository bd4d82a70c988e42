"""The downsampled loop (DS64 / DS32 of Section 2.3): nearest-neighbour
sampling of the database's masks and of the patient, then the same Dice
query.  Bit-exact against the oracle's downsampling of the thresholded
masks and its counts on them."""
import numpy as np
import pytest

import oracle
from paper_2205_04550_gb300 import DBQ_MODE_EXACT, DBQ_STORE_BITS, Database, DbqError, _dbq
from tests._gpu_helpers import assert_hits_equal, random_db

pytestmark = pytest.mark.gpu

T1, T2 = np.float32(0.6), np.float32(0.25)


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_2205_04550_gb300 import build
    build.build()
    return _t


def _ds_masks(vol, shape, f):
    nx, ny, nz = shape
    m = oracle.threshold(vol, T1, T2)
    return np.stack([oracle.downsample_nn(m[k], nx, ny, nz, f) for k in range(2)])


@pytest.mark.parametrize("shape,f", [((32, 32, 32), 2), ((32, 32, 32), 4), ((64, 32, 96), 2),
                                     ((60, 36, 24), 3)])
def test_downsampled_masks_and_query(torch, shape, f):
    n, k = 220, 12
    vols, patient = random_db(shape, n, seed=f + shape[2])
    with Database(shape, n, DBQ_STORE_BITS, T1, T2) as db:
        db.load(0, vols)
        db.build()
        ds = db.downsampled(f)
        try:
            dshape = tuple(s // f for s in shape)
            dv = int(np.prod(dshape))
            planes, sizes = ds.masks(0, n)
            dbm = np.stack([_ds_masks(vols[e], shape, f) for e in range(n)])
            for e in range(0, n, 11):
                np.testing.assert_array_equal(oracle.unpack_planes(planes[e], dv), dbm[e])
            np.testing.assert_array_equal(sizes, dbm.sum(axis=2))
            pm = _ds_masks(patient, shape, f)
            cnt, pc = oracle.counts_masks(dbm, pm)
            idx, val = oracle.rank(oracle.scores(cnt, pc), k)
            counts, pcount = ds.scan_counts(patient)
            np.testing.assert_array_equal(counts, cnt)
            np.testing.assert_array_equal(pcount, pc)
            ref = {"index": idx, "score": val,
                   "counts": np.concatenate([cnt[idx], np.tile(pc, (k, 1))], axis=1)}
            hits, _ = ds.query(patient, k)
            assert_hits_equal(hits, ref, k)
            ds.set_sparse(True)
            hits_s, _ = ds.query(torch.from_numpy(patient).cuda(), k)
            assert hits_s.tobytes() == hits.tobytes()
            ds.set_sparse(2)                    # the word-major copy of the coarse planes
            hits_t, _ = ds.query(patient, k)
            assert hits_t.tobytes() == hits.tobytes()
            counts_t, _ = ds.scan_counts(patient)
            np.testing.assert_array_equal(counts_t, cnt)
        finally:
            ds.close()


def test_downsampled_rejections(torch):
    vols, patient = random_db((32, 32, 32), 30, seed=1)
    with Database((32, 32, 32), 30, DBQ_STORE_BITS, T1, T2) as db:
        db.load(0, vols)
        db.build()
        with pytest.raises(DbqError) as e:
            db.downsampled(3)
        assert e.value.status == _dbq.DBQ_EINVAL
        ds = db.downsampled(2)
        try:
            with pytest.raises(DbqError) as e:
                _dbq.db_query_batch([ds.handle], [0], [patient], 3, DBQ_MODE_EXACT)
            assert e.value.status == _dbq.DBQ_ESTATE
            with pytest.raises(DbqError):
                ds.downsampled(2)
        finally:
            ds.close()
