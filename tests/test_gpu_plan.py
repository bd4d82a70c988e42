"""Query plans: many exact queries against databases of different
resolutions in one persistent launch, optionally captured in a CUDA graph.
Every hit list must equal the oracle's exact ranking (bit-exact)."""
import numpy as np
import pytest

import oracle
from paper_2205_04550_gb300 import DBQ_STORE_BITS, DBQ_STORE_F16, Database, DbqError, Plan, _dbq
from tests._gpu_helpers import assert_hits_equal, random_db

pytestmark = pytest.mark.gpu

T1, T2 = np.float32(0.6), np.float32(0.25)


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_2205_04550_gb300 import build
    build.build()
    return _t


@pytest.fixture(scope="module")
def two_dbs(torch):
    s1, s2 = (64, 64, 64), (32, 32, 32)
    v1, _ = random_db(s1, 500, seed=1)
    v2, _ = random_db(s2, 1300, seed=2)
    d1 = Database(s1, 500, DBQ_STORE_BITS, T1, T2)
    d1.load(0, v1)
    d1.build()
    d2 = Database(s2, 1300, DBQ_STORE_BITS, T1, T2)
    d2.load(0, v2)
    d2.build()
    yield (d1, v1), (d2, v2)
    d1.close()
    d2.close()


def _patients(rng, vols, count):
    out = []
    for _ in range(count):
        p = vols[rng.integers(0, len(vols))].copy()
        p[rng.random(p.shape) < 0.3] = 0.0          # a perturbed copy of an entry
        out.append(p)
    return out


@pytest.mark.parametrize("sparse", [False, True])
@pytest.mark.parametrize("items_per_sm", [1, 4, 64])
def test_plan_two_resolutions(torch, two_dbs, sparse, items_per_sm):
    (d1, v1), (d2, v2) = two_dbs
    d1.set_sparse(sparse)
    rng = np.random.default_rng(items_per_sm)
    pats = _patients(rng, v1, 5) + _patients(rng, v2, 6)
    which = [0] * 5 + [1] * 6
    perm = rng.permutation(len(pats))
    pats = [pats[i] for i in perm]
    which = [which[i] for i in perm]
    k = 16
    with Plan([d1, d2], 32, k) as plan:
        plan.set_items_per_sm(items_per_sm)
        dev = [torch.from_numpy(p).cuda() for p in pats]
        hits = torch.zeros((len(pats), k * 40), dtype=torch.uint8, device="cuda")
        plan.query(which, dev, hits)
        torch.cuda.synchronize()
        got = hits.cpu().numpy().view(_dbq.HIT_DTYPE)
        for q, (p, w) in enumerate(zip(pats, which)):
            vols = v1 if w == 0 else v2
            assert_hits_equal(got[q], oracle.query(vols, p, T1, T2, k), k)
    d1.set_sparse(False)


@pytest.mark.parametrize("sparse", [False, True])
def test_plan_captured_in_cuda_graph_and_replayed(torch, two_dbs, sparse):
    (d1, v1), (d2, v2) = two_dbs
    d1.set_sparse(sparse)
    d2.set_sparse(sparse)
    rng = np.random.default_rng(7)
    nq, k = 6, 10
    which = [0, 1, 0, 1, 1, 0]
    shapes = [v1.shape[1:] if w == 0 else v2.shape[1:] for w in which]
    slots = [torch.zeros(sh, dtype=torch.float32, device="cuda") for sh in shapes]
    hits = torch.zeros((nq, k * 40), dtype=torch.uint8, device="cuda")
    with Plan([d1, d2], nq, k) as plan:
        keep = []
        plan.query(which, slots, hits, keep=keep)     # first call outside capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                plan.query(which, slots, hits, keep=keep)
        torch.cuda.synchronize()
        for rep in range(3):
            pats = [(_patients(rng, v1, 1) if w == 0 else _patients(rng, v2, 1))[0] for w in which]
            for sl, p in zip(slots, pats):
                sl.copy_(torch.from_numpy(p))
            g.replay()
            torch.cuda.synchronize()
            got = hits.cpu().numpy().view(_dbq.HIT_DTYPE)
            for q, (p, w) in enumerate(zip(pats, which)):
                vols = v1 if w == 0 else v2
                assert_hits_equal(got[q], oracle.query(vols, p, T1, T2, k), k)
    d1.set_sparse(False)
    d2.set_sparse(False)


def _box_patient(rng, shape, frac):
    """A patient whose masks fill a random box holding about frac of the grid."""
    nx, ny, nz = shape
    p = np.zeros((nz, ny, nx), np.float32)
    d = [max(1, int(n * frac ** (1 / 3))) for n in (nz, ny, nx)]
    o = [int(rng.integers(0, n - dd + 1)) for n, dd in zip((nz, ny, nx), d)]
    p[o[0]:o[0] + d[0], o[1]:o[1] + d[1], o[2]:o[2] + d[2]] = rng.random(d, dtype=np.float32)
    return p


def test_plan_sparse_items_ordered_by_support(torch, two_dbs):
    """Sparse queries whose supports range from empty to the whole grid, with
    dense queries in the same launch: the items are re-ordered on the device
    by cost before the scan; every hit list stays the oracle's."""
    (d1, v1), (d2, v2) = two_dbs
    d1.set_sparse(True)
    rng = np.random.default_rng(11)
    fracs = [0.0, 1.0, 0.001, 0.01, 0.05, 0.2, 0.5, 0.8] * 3
    pats = [_box_patient(rng, v1.shape[1:][::-1], f) for f in fracs]
    pats[0] = np.zeros(v1.shape[1:], np.float32)
    pats[1] = np.ones(v1.shape[1:], np.float32)
    pats += _patients(rng, v2, 9)
    which = [0] * len(fracs) + [1] * 9
    perm = rng.permutation(len(pats))
    pats = [pats[i] for i in perm]
    which = [which[i] for i in perm]
    k = 12
    with Plan([d1, d2], len(pats), k) as plan:
        plan.set_tc_min_queries(0)                  # the CUDA-core loop's item ordering
        for ips in (2, 16):
            plan.set_items_per_sm(ips)
            dev = [torch.from_numpy(p).cuda() for p in pats]
            hits = torch.zeros((len(pats), k * 40), dtype=torch.uint8, device="cuda")
            plan.query(which, dev, hits)
            torch.cuda.synchronize()
            got = hits.cpu().numpy().view(_dbq.HIT_DTYPE)
            for q, (p, w) in enumerate(zip(pats, which)):
                vols = v1 if w == 0 else v2
                assert_hits_equal(got[q], oracle.query(vols, p, T1, T2, k), k)
    d1.set_sparse(False)


def test_plan_errors(torch, two_dbs):
    (d1, v1), (d2, v2) = two_dbs
    with pytest.raises(DbqError) as e:
        Plan([d1], 4, 501)
    assert e.value.status == _dbq.DBQ_ERANGE
    with Database((8, 8, 8), 4, DBQ_STORE_F16) as d3:
        d3.load(0, np.zeros((4, 8, 8, 8), np.float16).view(np.uint16))
        d3.build()
        with pytest.raises(DbqError) as e:
            Plan([d3], 4, 1)
        assert e.value.status == _dbq.DBQ_ESTATE
    with Plan([d1, d2], 2, 3) as plan:
        hits = torch.zeros((3, 3 * 40), dtype=torch.uint8, device="cuda")
        p = torch.from_numpy(v1[0]).cuda()
        with pytest.raises(DbqError):
            plan.query([0, 0, 0], [p, p, p], hits)          # more than max_queries
        with pytest.raises(DbqError):
            plan.query([2], [p], hits)                      # no such database
        with pytest.raises(DbqError):
            _dbq.db_plan_query(plan.handle, [0], [p], hits, t1=[0.5], t2=[0.25])
        with pytest.raises(DbqError):
            plan.set_tc_min_queries(-1)
        plan.status()                                       # nothing timed out


def _run_plan(torch, dbs, which, pats, k, tc_min, items_per_sm=4, tc_min_db=None):
    with Plan(dbs, len(pats), k) as plan:
        plan.set_items_per_sm(items_per_sm)
        plan.set_tc_min_queries(tc_min)
        for d, v in (tc_min_db or {}).items():
            plan.set_tc_min_queries(v, db=d)
        dev = [torch.from_numpy(p).cuda() for p in pats]
        hits = torch.zeros((len(pats), k * 40), dtype=torch.uint8, device="cuda")
        plan.query(which, dev, hits)
        plan.status()
        torch.cuda.synchronize()
        return hits.cpu().numpy().view(_dbq.HIT_DTYPE).copy()


def test_plan_tensor_core_path_matches_oracle_and_cuda_cores(torch, two_dbs):
    """Every dense query on the tensor-core contraction (threshold 1): hits
    equal to the oracle's and bit-identical to the CUDA-core loop's."""
    (d1, v1), (d2, v2) = two_dbs
    rng = np.random.default_rng(21)
    pats = _patients(rng, v1, 7) + _patients(rng, v2, 19)
    pats[0] = np.zeros_like(pats[0])                 # empty masks: Dice 1 only for empty entries
    pats[8] = np.ones_like(pats[8])
    which = [0] * 7 + [1] * 19
    perm = rng.permutation(len(pats))
    pats = [pats[i] for i in perm]
    which = [which[i] for i in perm]
    k = 20
    tc = _run_plan(torch, [d1, d2], which, pats, k, tc_min=1)
    cc = _run_plan(torch, [d1, d2], which, pats, k, tc_min=0)
    assert tc.tobytes() == cc.tobytes()
    for q, (p, w) in enumerate(zip(pats, which)):
        vols = v1 if w == 0 else v2
        assert_hits_equal(tc[q], oracle.query(vols, p, T1, T2, k), k)


@pytest.mark.parametrize("shape,n", [((30, 17, 11), 300), ((128, 16, 8), 129)])
def test_plan_tensor_core_ragged_sizes(torch, shape, n):
    """Grids whose voxel count is not a multiple of the 256-voxel K-slice,
    entry counts one past a 128-entry tile, more than 128 queries (two
    passes of the contraction over the database), and a sparse database
    next to the dense one in the same call."""
    vols, _ = random_db(shape, n, seed=n)
    rng = np.random.default_rng(n)
    pats = _patients(rng, vols, 131)
    v3, _ = random_db((16, 16, 16), 200, seed=5)
    with Database(shape, n, DBQ_STORE_BITS, T1, T2) as db, \
            Database((16, 16, 16), 200, DBQ_STORE_BITS, T1, T2) as ds:
        db.load(0, vols)
        db.build()
        ds.load(0, v3)
        ds.build()
        ds.set_sparse(True)
        sp = _patients(rng, v3, 20)
        allp = pats + sp
        which = [0] * len(pats) + [1] * len(sp)
        k = 9
        # the sparse database stays on the CUDA-core loop (its own threshold 0)
        tc = _run_plan(torch, [db, ds], which, allp, k, tc_min=16, tc_min_db={1: 0})
        cc = _run_plan(torch, [db, ds], which, allp, k, tc_min=0)
    assert tc.tobytes() == cc.tobytes()
    for q in list(range(0, 131, 13)) + [130]:
        assert_hits_equal(tc[q], oracle.query(vols, pats[q], T1, T2, k), k)
    for q in (0, 19):
        assert_hits_equal(tc[131 + q], oracle.query(v3, sp[q], T1, T2, k), k)


def test_plan_tensor_core_graph_replay(torch, two_dbs):
    (d1, v1), (d2, v2) = two_dbs
    rng = np.random.default_rng(3)
    nq, k = 24, 6
    which = [1] * 20 + [0] * 4
    shapes = [v1.shape[1:] if w == 0 else v2.shape[1:] for w in which]
    slots = [torch.zeros(sh, dtype=torch.float32, device="cuda") for sh in shapes]
    hits = torch.zeros((nq, k * 40), dtype=torch.uint8, device="cuda")
    with Plan([d1, d2], nq, k) as plan:
        plan.set_tc_min_queries(16)                 # database 1 on the tensor cores
        keep = []
        plan.query(which, slots, hits, keep=keep)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                plan.query(which, slots, hits, keep=keep)
        torch.cuda.synchronize()
        for rep in range(2):
            pats = [(_patients(rng, v1, 1) if w == 0 else _patients(rng, v2, 1))[0] for w in which]
            for sl, p in zip(slots, pats):
                sl.copy_(torch.from_numpy(p))
            g.replay()
            torch.cuda.synchronize()
            plan.status()
            got = hits.cpu().numpy().view(_dbq.HIT_DTYPE)
            for q, (p, w) in enumerate(zip(pats, which)):
                vols = v1 if w == 0 else v2
                assert_hits_equal(got[q], oracle.query(vols, p, T1, T2, k), k)


@pytest.mark.parametrize("k", [300, 500])
def test_plan_tensor_core_large_k(torch, two_dbs, k):
    """The selection after the contraction with k close to its shared-memory
    capacity (flushes after every round of offers): the oracle's full
    ranking down to position k, bit-identical to the CUDA-core loop."""
    (d1, v1), _ = two_dbs
    rng = np.random.default_rng(k)
    pats = _patients(rng, v1, 17)
    which = [0] * len(pats)
    tc = _run_plan(torch, [d1], which, pats, k, tc_min=16)
    cc = _run_plan(torch, [d1], which, pats, k, tc_min=0)
    assert tc.tobytes() == cc.tobytes()
    for q in (0, 8, 16):
        assert_hits_equal(tc[q], oracle.query(v1, pats[q], T1, T2, k), k)


@pytest.mark.parametrize("shape,n", [((128, 128, 128), 64), ((256, 256, 256), 8)])
def test_plan_tensor_core_counts_near_the_binary32_limit(torch, shape, n):
    """The contraction's counts where they are largest: full and nearly full
    masks at 128^3 (counts up to 2^21) and 256^3 (up to 2^24, the largest
    grid the tensor-core path takes).  The binary32 accumulators must still
    hold the exact integers: hits bit-identical to the CUDA-core loop's and
    equal to the oracle's."""
    nx, ny, nz = shape
    rng = np.random.default_rng(n)
    vols = np.empty((n, nz, ny, nx), np.float32)
    for e in range(n):
        if e % 4 == 0:
            vols[e] = 1.0                                    # E_1 = E_2 = V
        else:
            vols[e] = rng.random((nz, ny, nx), dtype=np.float32)
            vols[e][rng.random((nz, ny, nx)) < 0.02 * e / n] = 0.0
    pats = [np.ones((nz, ny, nx), np.float32), vols[1].copy(), vols[n - 1].copy()]
    for _ in range(3):
        p = rng.random((nz, ny, nx), dtype=np.float32)
        p[rng.random(p.shape) < 0.01] = 0.0
        pats.append(p)
    which = [0] * len(pats)
    k = min(n, 8)
    with Database(shape, n, DBQ_STORE_BITS, T1, T2) as db:
        db.load(0, vols)
        db.build()
        tc = _run_plan(torch, [db], which, pats, k, tc_min=1)
        cc = _run_plan(torch, [db], which, pats, k, tc_min=0)
    assert tc.tobytes() == cc.tobytes()
    for q, p in enumerate(pats):
        ref = oracle.query(vols, p, T1, T2, k)
        assert_hits_equal(tc[q], ref, k)
    # the full patient against a full entry: I = E = P = V exactly
    assert int(tc[0]["i2"][0]) == nx * ny * nz and tc[0]["score"][0] == 1.0


def test_plan_tensor_core_timeout_path_reports_and_recovers(torch, two_dbs):
    """The bounded-wait path of the tensor-core kernel: with the test stall
    on, the kernel's first wait is on a barrier nothing arrives at; it gives
    up after 1 ms, records the timeout, drains and frees its tensor memory,
    and db_plan_status reports DBQ_ETIMEOUT.  The next call, with the stall
    off, returns the oracle's hits on the same plan."""
    (d1, v1), _ = two_dbs
    rng = np.random.default_rng(99)
    pats = _patients(rng, v1, 4)
    which = [0] * len(pats)
    k = 5
    with Plan([d1], len(pats), k) as plan:
        plan.set_tc_min_queries(1)
        dev = [torch.from_numpy(p).cuda() for p in pats]
        hits = torch.zeros((len(pats), k * 40), dtype=torch.uint8, device="cuda")
        _dbq.db_plan_set(plan.handle, _dbq.DBQ_PLAN_TEST_STALL_NS, 1_000_000)
        plan.query(which, dev, hits)
        with pytest.raises(DbqError) as e:
            plan.status()
        assert e.value.status == _dbq.DBQ_ETIMEOUT
        plan.status()                                    # the condition was cleared
        _dbq.db_plan_set(plan.handle, _dbq.DBQ_PLAN_TEST_STALL_NS, 0)
        plan.query(which, dev, hits)
        plan.status()
        torch.cuda.synchronize()
        got = hits.cpu().numpy().view(_dbq.HIT_DTYPE)
        for q, p in enumerate(pats):
            assert_hits_equal(got[q], oracle.query(v1, p, T1, T2, k), k)


def test_plan_sparse_database_on_the_tensor_cores(torch, two_dbs):
    """A database with the sparse option and many queries in one call is
    scanned as a contraction (which reads every word) when it passes its
    threshold: the hits equal the sparse CUDA-core loop's and the oracle's.
    Per-database thresholds: database 0 on the contraction, database 1 kept
    on the loop."""
    (d1, v1), (d2, v2) = two_dbs
    d1.set_sparse(True)
    d2.set_sparse(True)
    try:
        rng = np.random.default_rng(31)
        pats = _patients(rng, v1, 20) + _patients(rng, v2, 20)
        which = [0] * 20 + [1] * 20
        k = 7
        tc = _run_plan(torch, [d1, d2], which, pats, k, tc_min=1, tc_min_db={1: 0})
        cc = _run_plan(torch, [d1, d2], which, pats, k, tc_min=0)
    finally:
        d1.set_sparse(False)
        d2.set_sparse(False)
    assert tc.tobytes() == cc.tobytes()
    for q in (0, 7, 19, 20, 39):
        vols = v1 if which[q] == 0 else v2
        assert_hits_equal(tc[q], oracle.query(vols, pats[q], T1, T2, k), k)


def test_plan_per_database_threshold_errors(torch, two_dbs):
    (d1, _), (d2, _) = two_dbs
    with Plan([d1, d2], 4, 3) as plan:
        with pytest.raises(DbqError) as e:
            plan.set_tc_min_queries(5, db=2)
        assert e.value.status == _dbq.DBQ_ERANGE
        with pytest.raises(DbqError):
            plan.set_tc_min_queries(-2, db=0)
        plan.set_tc_min_queries(-1, db=0)             # back to the plan-wide value


@pytest.mark.parametrize("nq", [1, 63, 64, 65, 128])
def test_plan_tensor_core_query_counts(torch, two_dbs, nq):
    """One query to a full pass of 128 on the contraction (M = 128 rows, the
    rows past the last query zero): hits bit-identical to the CUDA-core loop
    and equal to the oracle."""
    (d1, v1), _ = two_dbs
    rng = np.random.default_rng(400 + nq)
    pats = _patients(rng, v1, nq)
    which = [0] * nq
    k = 6
    tc = _run_plan(torch, [d1], which, pats, k, tc_min=1)
    cc = _run_plan(torch, [d1], which, pats, k, tc_min=0)
    assert tc.tobytes() == cc.tobytes()
    for q in sorted({0, nq // 2, nq - 1}):
        assert_hits_equal(tc[q], oracle.query(v1, pats[q], T1, T2, k), k)


def test_plan_word_major_sparse_counts(torch, two_dbs):
    """Queries of databases with a word-major copy (DBQ_OPT_SPARSE 2) that stay
    off the contraction: the counts of all of them over the copy, then the
    per-query selection -- the oracle's hits, bit-identical to the CUDA-core
    loop; 140 queries of one database (two passes of 128), and graph replay."""
    (d1, v1), (d2, v2) = two_dbs
    rng = np.random.default_rng(41)
    p1 = _patients(rng, v1, 5) + [_box_patient(rng, (64, 64, 64), f) for f in (0.01, 0.05, 0.2, 0.5)]
    p2 = _patients(rng, v2, 60) + [_box_patient(rng, (32, 32, 32), 0.002 * (1 + i)) for i in range(78)]
    p2 += [np.zeros_like(p2[0]), np.ones_like(p2[0])]
    pats = p1 + p2
    which = [0] * len(p1) + [1] * len(p2)
    perm = rng.permutation(len(pats))
    pats = [pats[i] for i in perm]
    which = [which[i] for i in perm]
    k = 12
    cc = _run_plan(torch, [d1, d2], which, pats, k, tc_min=0)
    d1.set_sparse(2)
    d2.set_sparse(2)
    try:
        wm = _run_plan(torch, [d1, d2], which, pats, k, tc_min=0)
        assert wm.tobytes() == cc.tobytes()
        for q, (p, w) in enumerate(zip(pats, which)):
            vols = v1 if w == 0 else v2
            assert_hits_equal(wm[q], oracle.query(vols, p, T1, T2, k), k)
        # captured once, replayed with new patients in the same device slots
        dev = [torch.from_numpy(p).cuda() for p in pats]
        hits = torch.zeros((len(pats), k * 40), dtype=torch.uint8, device="cuda")
        with Plan([d1, d2], len(pats), k) as plan:
            plan.set_tc_min_queries(0)
            keep = []
            plan.query(which, dev, hits, keep=keep)     # first call outside capture
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                with torch.cuda.graph(g, stream=s):
                    plan.query(which, dev, hits, keep=keep)
            torch.cuda.synchronize()
            new = [_box_patient(rng, (64, 64, 64) if w == 0 else (32, 32, 32), 0.05) for w in which]
            for sl, p in zip(dev, new):
                sl.copy_(torch.from_numpy(p))
            g.replay()
            torch.cuda.synchronize()
            got = hits.cpu().numpy().view(_dbq.HIT_DTYPE)
            for q in range(0, len(new), 7):
                vols = v1 if which[q] == 0 else v2
                assert_hits_equal(got[q], oracle.query(vols, new[q], T1, T2, k), k)
    finally:
        d1.set_sparse(False)
        d2.set_sparse(False)
