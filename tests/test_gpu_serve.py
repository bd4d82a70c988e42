"""The continuous-batching server: requests that arrive while others are on
the GPU are batched, admitted by memory and run on concurrent lanes; every
request's hits must be identical to the same query run alone."""
import numpy as np
import pytest

from paper_2205_04550_gb300 import DBQ_MODE_EMBED_BF16, DBQ_STORE_BITS, Database, serve, synth
from tests._gpu_helpers import random_db

pytestmark = pytest.mark.gpu

T1, T2 = np.float32(0.6), np.float32(0.25)


@pytest.fixture(scope="module")
def dbs():
    import torch  # noqa: F401
    from paper_2205_04550_gb300 import build
    build.build()
    s1, s2 = (64, 64, 64), (32, 32, 32)
    v1, _ = synth.database_np(s1, 400)
    v2, _ = random_db(s2, 700, seed=3)
    d1 = Database(s1, 400, DBQ_STORE_BITS, T1, T2, embed=True)
    d1.load(0, v1)
    d1.build()
    d2 = Database(s2, 700, DBQ_STORE_BITS, T1, T2, embed=True)
    d2.load(0, v2)
    d2.build()
    yield (d1, v1), (d2, v2)
    d1.close()
    d2.close()


def _requests(v1, v2, count, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for _ in range(count):
        if rng.random() < 0.7:
            p = v1[rng.integers(0, len(v1))].copy()
            db = 0
        else:
            p = v2[rng.integers(0, len(v2))].copy()
            db = 1
        p[rng.random(p.shape) < 0.2] = 0.0
        reqs.append((p, db))
    return reqs


@pytest.mark.parametrize("mode", ["exact", "embed_bf16"])
def test_results_in_the_mix_equal_results_alone(dbs, mode):
    (d1, v1), (d2, v2) = dbs
    reqs = _requests(v1, v2, 240, seed=11)
    arrivals = serve.poisson_arrivals(3000.0, len(reqs), seed=7)
    srv = serve.Server([d1, d2], mode=mode, k=10, n_candidates=64, max_batch=32, lanes=2)
    try:
        results = serve.run_open_loop(srv, reqs, arrivals)
        st = srv.stats()
    finally:
        srv.close()
    assert st["completed"] == len(reqs) and st["p99_ms"] >= st["p50_ms"] > 0
    databases = [d1, d2]
    for i in range(len(reqs)):
        p, db = reqs[i]
        if mode == "exact":
            alone, _ = databases[db].query(p, 10)
        else:
            alone, _ = databases[db].query_batch([p], 10, DBQ_MODE_EMBED_BF16, 64)
            alone = alone[0]
        assert results[i].tobytes() == alone.tobytes(), i


def test_admission_by_memory_budget(dbs):
    (d1, v1), (d2, v2) = dbs
    one = v1[0].nbytes + 10 * 40
    srv = serve.Server([d1, d2], mode="exact", k=10, max_batch=16, lanes=2, budget=3 * one)
    try:
        reqs = _requests(v1, v2, 40, seed=5)
        reqs = [(p, 0) if db == 0 else (v1[3], 0) for p, db in reqs]
        results = serve.run_open_loop(srv, reqs, np.zeros(len(reqs)))
        for (p, db), r in zip(reqs[:5], results[:5]):
            alone, _ = d1.query(p, 10)
            assert r.tobytes() == alone.tobytes()
    finally:
        srv.close()
    tiny = serve.Server([d1], mode="exact", k=10, max_batch=4, lanes=1, budget=1000)
    try:
        with pytest.raises(serve.AdmissionError):
            tiny.submit(v1[0], 0)
    finally:
        tiny.close()


def test_hash_mode_in_the_mix_equals_alone():
    """Serving over sketch databases with the Hamming prefilter: each
    request's hits equal the same query run alone."""
    import torch  # noqa: F401
    from paper_2205_04550_gb300 import DBQ_MODE_HASH, build
    build.build()
    s1, s2 = (48, 40, 32), (32, 32, 32)
    v1, _ = synth.database_np(s1, 300)
    v2, _ = random_db(s2, 500, seed=5)
    d1 = Database(s1, 300, DBQ_STORE_BITS, T1, T2, sketch=True)
    d2 = Database(s2, 500, DBQ_STORE_BITS, T1, T2, sketch=True)
    try:
        d1.load(0, v1)
        d1.build()
        d2.load(0, v2)
        d2.build()
        reqs = _requests(v1, v2, 120, seed=13)
        arrivals = serve.poisson_arrivals(3000.0, len(reqs), seed=9)
        srv = serve.Server([d1, d2], mode="hash", k=10, n_candidates=64, max_batch=32, lanes=2)
        try:
            results = serve.run_open_loop(srv, reqs, arrivals)
        finally:
            srv.close()
        databases = [d1, d2]
        for i in range(len(reqs)):
            p, db = reqs[i]
            alone, _ = databases[db].query_batch([p], 10, DBQ_MODE_HASH, 64)
            assert results[i].tobytes() == alone[0].tobytes(), i
    finally:
        d1.close()
        d2.close()


def test_batches_of_different_lanes_overlap_on_the_device(dbs):
    """Requests that arrive while earlier ones are on the GPU run on the
    other lane at the same time: a burst of small batches leaves at least one
    pair of batches from different lanes whose device spans overlap, and
    every result still equals the query alone."""
    (d1, v1), (d2, v2) = dbs
    reqs = _requests(v1, v2, 96, seed=21)
    srv = serve.Server([d1, d2], mode="exact", k=10, max_batch=4, lanes=2, max_wait_s=0.0)
    try:
        results = serve.run_open_loop(srv, reqs, np.zeros(len(reqs)))
        overlaps = srv.device_overlaps()
        spans = srv.device_spans()
    finally:
        srv.close()
    assert len({lane for lane, _, _ in spans}) == 2
    assert overlaps > 0, spans[:8]
    databases = [d1, d2]
    for i, (p, db) in enumerate(reqs):
        alone, _ = databases[db].query(p, 10)
        assert results[i].tobytes() == alone.tobytes(), i
