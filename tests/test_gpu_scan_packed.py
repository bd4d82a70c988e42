"""Parity of the bit-packed exact query (pack + fused scan/score/top-k) with
the CPU oracle, element by element, on seeded inputs.

Bar: bit-exact on every count, on the binary64 score bits, on the arg-max
and on the whole top-k order (Section 2.3 query; ties to the lowest index).
"""
import numpy as np
import pytest

import oracle
from paper_2205_04550_gb300 import (DBQ_BITS, DBQ_F16, DBQ_F32, DBQ_STORE_BITS, Database,
                                    DbqError, _dbq, synth)
from tests._gpu_helpers import (assert_hits_equal, pack_bits_np, random_db, surrogate_db)

pytestmark = pytest.mark.gpu

T1, T2 = np.float32(0.6), np.float32(0.25)


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_2205_04550_gb300 import build
    build.build()
    _t.cuda.init()
    return _t


def _db_from(vols, t1=T1, t2=T2, n_params=0, params=None, device_input=False, torch=None):
    n = vols.shape[0]
    nz, ny, nx = vols.shape[1:]
    db = Database((nx, ny, nz), n, DBQ_STORE_BITS, t1, t2, n_params)
    src = torch.from_numpy(vols).cuda() if device_input else vols
    db.load(0, src, params=params)
    db.build()
    return db


CASES = [
    # shape, n, k: ragged volumes (not a multiple of 32 or 128 bits), N not a
    # multiple of the grid, k from 1 to N
    ((1, 1, 1), 5, 5),
    ((8, 8, 8), 1, 1),
    ((9, 10, 11), 153, 10),
    ((8, 8, 8), 1000, 64),
    ((17, 5, 3), 300, 300),
    ((32, 32, 32), 700, 16),
    ((33, 31, 30), 500, 7),
    ((64, 64, 64), 160, 12),
]


@pytest.mark.parametrize("shape,n,k", CASES)
def test_random_volumes_counts_and_topk(torch, shape, n, k):
    vols, patient = random_db(shape, n, seed=n + shape[0], plant=(n // 2, n - 1))
    ref = oracle.query(vols, patient, T1, T2, k)
    with _db_from(vols, torch=torch) as db:
        counts, pcount = db.scan_counts(patient)
        np.testing.assert_array_equal(pcount, ref["pcount"])
        np.testing.assert_array_equal(counts, ref["all_counts"])
        hits, _ = db.query(patient, k)
        assert_hits_equal(hits, ref, k)


def test_surrogate_volumes_several_tiles(torch):
    shape = (64, 64, 64)
    vols, patient, theta = surrogate_db(shape, 400, plant=(123, 321))
    ref = oracle.query(vols, patient, T1, T2, 20)
    assert ref["index"][0] == 123 and ref["index"][1] == 321 and ref["score"][0] == 1.0
    with _db_from(vols, n_params=8, params=theta, device_input=True, torch=torch) as db:
        hits, params = db.query(patient, 20)
        assert_hits_equal(hits, ref, 20)
        np.testing.assert_array_equal(params, theta[ref["index"]])
        counts, _ = db.scan_counts(torch.from_numpy(patient).cuda())
        np.testing.assert_array_equal(counts, ref["all_counts"])


def test_packer_round_trip_and_boundaries(torch):
    shape = (9, 10, 11)
    vols, _ = random_db(shape, 40, seed=3)
    flat = vols.reshape(40, -1)
    # values exactly at, just below and just above the thresholds, +0, -0, 1
    specials = np.array([T1, np.nextafter(T1, 0), np.nextafter(T1, 1), T2, np.nextafter(T2, 0),
                         np.nextafter(T2, 1), 0.0, -0.0, 1.0], dtype=np.float32)
    flat[:, :specials.size] = specials
    with _db_from(vols, torch=torch) as db:
        planes, sizes = db.masks(0, 40)
        for e in range(40):
            want = oracle.threshold(vols[e], T1, T2)
            got = oracle.unpack_planes(planes[e], flat.shape[1])
            np.testing.assert_array_equal(got, want)
            np.testing.assert_array_equal(sizes[e], want.sum(axis=1))
            # bits past the last voxel are zero
            tail = planes[e].view(np.uint32)[:, -1] >> np.uint32(flat.shape[1] % 32)
            assert not tail.any()


def test_patient_kinds_f32_f16_bits_host_and_device(torch):
    shape = (16, 12, 10)
    vols, patient = random_db(shape, 257, seed=11, plant=(200,))
    p16 = patient.astype(np.float16)
    ref32 = oracle.query(vols, patient, T1, T2, 9)
    ref16 = oracle.query(vols, p16, T1, T2, 9)
    bits = pack_bits_np(oracle.threshold(patient, T1, T2))
    refb = oracle.query(vols, patient, T1, T2, 9,
                        patient_mask=oracle.unpack_planes(bits, patient.size))
    with _db_from(vols, torch=torch) as db:
        for pat, ref in ((patient, ref32), (p16.view(np.uint16), ref16), (bits, refb)):
            hits, _ = db.query(pat, 9)
            assert_hits_equal(hits, ref, 9)
            hits, _ = db.query(torch.from_numpy(pat).cuda(), 9)
            assert_hits_equal(hits, ref, 9)


def test_pinned_host_patients_read_in_place(torch):
    """Page-locked host patients (read by the packing kernel in place) and an
    unaligned view into one (staged instead) give the oracle's hits."""
    shape = (33, 31, 30)
    vols, patient = random_db(shape, 400, seed=77, plant=(5,))
    ref = oracle.query(vols, patient, T1, T2, 12)
    with _db_from(vols, torch=torch) as db:
        pinned = torch.from_numpy(patient).pin_memory()
        hits, _ = db.query(pinned.numpy(), 12)
        assert_hits_equal(hits, ref, 12)
        counts, pcount = db.scan_counts(pinned.numpy())
        np.testing.assert_array_equal(counts, ref["all_counts"])
        np.testing.assert_array_equal(pcount, ref["pcount"])
        # f32 patient one element into a pinned buffer: 4-byte aligned only
        buf = torch.zeros(patient.size + 1, dtype=torch.float32).pin_memory()
        buf[1:] = torch.from_numpy(patient.reshape(-1))
        hits_u, _ = db.query(buf.numpy()[1:].reshape(patient.shape), 12)
        assert hits_u.tobytes() == hits.tobytes()
        # f16 and bit-plane patients from pinned memory
        p16 = torch.from_numpy(patient.astype(np.float16).view(np.int16)).pin_memory()
        ref16 = oracle.query(vols, patient.astype(np.float16).astype(np.float32), T1, T2, 12)
        hits16, _ = db.query(p16.numpy().view(np.uint16), 12, kind=DBQ_F16)
        assert_hits_equal(hits16, ref16, 12)
        bits = pack_bits_np(oracle.threshold(patient, T1, T2))
        refb = oracle.query(vols, patient, T1, T2, 12,
                            patient_mask=oracle.unpack_planes(bits, patient.size))
        pb = torch.from_numpy(bits.view(np.int32)).pin_memory()
        hitsb, _ = db.query(pb.numpy().view(np.uint32), 12)
        assert_hits_equal(hitsb, refb, 12)


def test_bits_patient_ignores_bits_past_last_voxel(torch):
    shape = (9, 10, 11)     # 990 voxels: the last word has 30 used bits
    vols, patient = random_db(shape, 50, seed=5)
    m = oracle.threshold(patient, T1, T2)
    bits = pack_bits_np(m)
    dirty = bits.copy()
    dirty[:, -1] |= np.uint32(0xC0000000)
    ref = oracle.query(vols, patient, T1, T2, 5, patient_mask=m)
    with _db_from(vols, torch=torch) as db:
        hits, _ = db.query(dirty, 5)
        assert_hits_equal(hits, ref, 5)


def test_f16_database_input_thresholds_like_oracle(torch):
    shape = (8, 8, 8)
    vols, patient = random_db(shape, 64, seed=9)
    v16 = vols.astype(np.float16)
    ref = oracle.query(v16, patient, T1, T2, 8)
    db = Database(shape, 64, DBQ_STORE_BITS, T1, T2)
    db.load(0, v16.view(np.uint16))
    db.build()
    hits, _ = db.query(patient, 8)
    assert_hits_equal(hits, ref, 8)
    db.close()


def test_all_equal_scores_tie_break_by_index(torch):
    shape = (8, 8, 8)
    vols, patient = random_db(shape, 1, seed=2)
    db_vols = np.repeat(vols, 2500, axis=0)
    with _db_from(db_vols, torch=torch) as db:
        hits, _ = db.query(patient, 100)
        np.testing.assert_array_equal(hits["index"], np.arange(100))
        assert len(set(hits["score"].tolist())) == 1


def test_determinism_repeated_queries(torch):
    vols, patient = random_db((32, 32, 32), 900, seed=21)
    with _db_from(vols, torch=torch) as db:
        first, _ = db.query(patient, 50)
        for _ in range(3):
            again, _ = db.query(patient, 50)
            assert again.tobytes() == first.tobytes()


def test_async_query_into_device_buffer(torch):
    vols, patient = random_db((16, 16, 16), 333, seed=4, plant=(7,))
    ref = oracle.query(vols, patient, T1, T2, 11)
    with _db_from(vols, torch=torch) as db:
        out = torch.zeros(11 * 40, dtype=torch.uint8, device="cuda")
        db.query_async(torch.from_numpy(patient).cuda(), 11, out)
        torch.cuda.synchronize()
        assert_hits_equal(_dbq.hits_from_device(out), ref, 11)


def test_error_paths(torch):
    vols, patient = random_db((8, 8, 8), 10, seed=1)
    db = Database((8, 8, 8), 10, DBQ_STORE_BITS, T1, T2)
    with pytest.raises(DbqError) as e:
        db.query(patient, 1)                      # not built
    assert e.value.status == _dbq.DBQ_ESTATE
    db.load(0, vols[:5])
    with pytest.raises(DbqError) as e:
        db.build()                                # entries 5..9 missing
    assert e.value.status == _dbq.DBQ_ESTATE
    db.load(5, vols[5:])
    db.build()
    for k in (0, 11, 2000):
        with pytest.raises(DbqError) as e:
            db.query(patient, k)
        assert e.value.status == _dbq.DBQ_ERANGE
    with pytest.raises(DbqError) as e:
        db.query(patient, 1, t1=0.5, t2=0.25)     # not the build thresholds
    assert e.value.status == _dbq.DBQ_EINVAL
    with pytest.raises(DbqError) as e:
        _dbq.db_load_volumes(db.handle, 8, 5, vols[:5])   # past capacity
    assert e.value.status == _dbq.DBQ_ERANGE
    hits, _ = db.query(patient, 10)               # still usable after errors
    assert_hits_equal(hits, oracle.query(vols, patient, T1, T2, 10), 10)
    db.close()
    with pytest.raises(DbqError):
        Database((8, 8, 8), 4, DBQ_STORE_BITS, 0.0, 0.25)
    with pytest.raises(DbqError):
        Database((8, 8, 8), 4, DBQ_STORE_BITS, float("nan"), 0.25)
