"""db_scan_packed_noalloc: the allocation-free variant of the bit-packed
query, for callers that cannot allocate device memory (a pool that owns the
whole GPU, a request path that must not synchronise on an allocation, a
plug-in host that forbids device allocations).

It is checked through the C ABI against the handle API's db_query and
against the CPU oracle on the same database and patients -- bit-exact, the
tolerance every parity test here uses -- on two calls in a row with different
patients, so a stale scratch array from the first call would show in the
second.  The cases cover the documented limit k = 64, fewer entries than
SMs (CTAs with no entries publish lists of sentinels into the shared array)
and k = n.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2205_04550_gb300 import DBQ_STORE_BITS, Database, _dbq
from tests._gpu_helpers import assert_hits_equal, pack_bits_np, random_db

pytestmark = pytest.mark.gpu

T1, T2 = np.float32(0.6), np.float32(0.25)


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_2205_04550_gb300 import build
    build.build()
    return _t


def _hits(t):
    return _dbq.hits_from_device(t)


@pytest.mark.parametrize("n,k", [(777, 13), (777, 64), (50, 7), (64, 64)])
def test_noalloc_matches_db_query_two_calls(torch, n, k):
    shape = (32, 32, 32)                      # 1024 words per plane, a multiple of 4
    plant = n * 2 // 3
    vols, patient_a = random_db(shape, n, seed=41 + n, plant=(plant,))
    _, patient_b = random_db(shape, 1, seed=42 + n)
    lib = _dbq.load()
    with Database(shape, n, DBQ_STORE_BITS, T1, T2) as db:
        db.load(0, vols)
        db.build()
        words = db.info()["words"]
        planes = torch.zeros((n, 2, words), dtype=torch.int32, device="cuda")
        sizes = torch.zeros((n, 2), dtype=torch.int32, device="cuda")
        _dbq.db_get_masks(db.handle, 0, n, planes, sizes)
        stream = torch.cuda.current_stream()
        best = []
        for patient in (patient_a, patient_b):
            mask = oracle.threshold(patient, T1, T2)
            pplanes = torch.from_numpy(pack_bits_np(mask).view(np.int32)).cuda()
            psizes = torch.from_numpy(mask.sum(axis=1).astype(np.int32)).cuda()
            out = torch.zeros(k * 40, dtype=torch.uint8, device="cuda")
            rc = lib.db_scan_packed_noalloc(planes.data_ptr(), sizes.data_ptr(), n, words,
                                            pplanes.data_ptr(), psizes.data_ptr(), k,
                                            out.data_ptr(), stream.cuda_stream)
            assert rc == _dbq.DBQ_OK, lib.db_last_error()
            torch.cuda.synchronize()
            want, _ = db.query(patient, k)
            got = _hits(out)
            assert got.tobytes() == want.tobytes()
            assert_hits_equal(got, oracle.query(vols, patient, T1, T2, k), k)
            best.append(int(got["index"][0]))
        # the planted copy of patient a is the best match of the first call only
        assert best[0] == plant and best[1] != plant


def test_noalloc_rejects_sizes_beyond_its_limits(torch):
    lib = _dbq.load()
    buf = torch.zeros(1 << 16, dtype=torch.int32, device="cuda")
    out = torch.zeros(65 * 40, dtype=torch.uint8, device="cuda")
    p = buf.data_ptr()
    rc = lib.db_scan_packed_noalloc(p, p, 100, 8, p, p, 65, out.data_ptr(), None)
    assert rc == _dbq.DBQ_ERANGE and b"64" in lib.db_last_error()
    rc = lib.db_scan_packed_noalloc(p, p, 100, 6, p, p, 5, out.data_ptr(), None)
    assert rc == _dbq.DBQ_EINVAL
    rc = lib.db_scan_packed_noalloc(p, p, 3, 8, p, p, 4, out.data_ptr(), None)
    assert rc == _dbq.DBQ_ERANGE
    rc = lib.db_scan_packed_noalloc(None, p, 3, 8, p, p, 1, out.data_ptr(), None)
    assert rc == _dbq.DBQ_EINVAL
    assert ctypes.sizeof(_dbq.dbq_hit) == 40
