"""Host-side logic without a GPU: the plan autotuner's searches and cache
(tune.py) against a fake plan with a known cost model and fake CUDA events,
and the server's batching, memory admission and overlap counting (serve.py)
on a server object whose device parts are left out.
"""
import queue
import threading
import types

import numpy as np
import pytest
import torch

from paper_2205_04550_gb300 import serve, tune


class _Clock:
    t = 0.0


class _FakeEvent:
    """torch.cuda.Event stand-in reading a fake clock advanced by the plan."""

    def __init__(self, clock, enable_timing=True):
        self.clock = clock
        self.t = None

    def record(self, stream=None):
        self.t = self.clock.t

    def elapsed_time(self, end):
        return end.t - self.t


class _FakePlan:
    """Plan stand-in: query() advances the clock by cost(which, tc_min, items)."""

    def __init__(self, databases, max_queries, cost, clock):
        self.databases = databases
        self.max_queries = max_queries
        self.k = 10
        self.tc = {}
        self.items = 4
        self.cost = cost
        self.clock = clock
        self.queries = 0

    def set_tc_min_queries(self, value, db):
        self.tc[db] = value

    def set_items_per_sm(self, value):
        self.items = value

    def query(self, which, patients, hits, stream=None):
        self.queries += 1
        self.clock.t += self.cost(which, dict(self.tc), self.items)


@pytest.fixture
def fake_cuda(monkeypatch, tmp_path):
    clock = _Clock()
    monkeypatch.setattr(tune, "CACHE", str(tmp_path / "autotune.json"))
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "get_device_properties",
                        lambda d: types.SimpleNamespace(name="fake", multi_processor_count=152))
    monkeypatch.setattr(torch.cuda, "Event", lambda enable_timing=True: _FakeEvent(clock))
    return clock


def _db(shape=(64, 64, 64), n=1000, sparse_mode=0):
    return types.SimpleNamespace(shape=shape, capacity=n, sparse_mode=sparse_mode)


def _crossover_cost(tc_ms, loop_ms_per_query):
    """Contraction: a flat cost (threshold 1 sends every query to it); loop:
    a cost per query (threshold 0 keeps every query on it)."""
    def cost(which, tc, items):
        d = which[0]
        return tc_ms if tc.get(d) == 1 else loop_ms_per_query * len(which)
    return cost


def test_crossover_is_the_smallest_batch_where_the_contraction_is_no_slower(fake_cuda):
    plan = _FakePlan([_db()], 128, _crossover_cost(10.0, 1.5), fake_cuda)
    res = tune.tune_crossover(plan, 0, ["p"], None, reps=2)
    # loop 3, 6, 9 ms at 2, 4, 6 queries beats 10 ms; 12 ms at 8 does not
    assert res["tc_min"] == 8 and not res["cached"]
    assert plan.tc[0] == 8
    assert sorted(res["ms"], key=int) == ["2", "4", "6", "8"]
    assert res["ms"]["8"] == [10.0, 12.0]


def test_crossover_when_the_loop_always_wins(fake_cuda):
    plan = _FakePlan([_db()], 128, _crossover_cost(1000.0, 1.0), fake_cuda)
    res = tune.tune_crossover(plan, 0, ["p"], None, reps=1)
    assert res["tc_min"] == 2 * max(tune.TC_BATCHES)
    assert plan.tc[0] == 2 * max(tune.TC_BATCHES)


def test_crossover_cache_is_keyed_by_grid_size_and_sparse_mode(fake_cuda):
    plan = _FakePlan([_db()], 128, _crossover_cost(10.0, 1.5), fake_cuda)
    tune.tune_crossover(plan, 0, ["p"], None)
    timed = plan.queries
    again = tune.tune_crossover(plan, 0, ["p"], None)
    assert again["cached"] and again["tc_min"] == 8 and plan.queries == timed
    # another entry count, and the sparse loop, are tuned apart
    other = _FakePlan([_db(n=2000)], 128, _crossover_cost(10.0, 3.0), fake_cuda)
    assert tune.tune_crossover(other, 0, ["p"], None)["tc_min"] == 4
    sparse = tune.tune_crossover(plan, 0, ["p"], None, sparse=2)
    assert not sparse["cached"]


def test_crossover_stops_at_the_plans_capacity(fake_cuda):
    plan = _FakePlan([_db()], 6, _crossover_cost(1000.0, 1.0), fake_cuda)
    res = tune.tune_crossover(plan, 0, ["p"], None, reps=1)
    assert sorted(res["ms"], key=int) == ["2", "4", "6"]


def test_items_per_sm_is_the_fastest_candidate_and_cached(fake_cuda):
    best = 8

    def cost(which, tc, items):
        return 5.0 + abs(np.log2(items) - np.log2(best))
    plan = _FakePlan([_db(), _db((128, 128, 128), 500)], 128, cost, fake_cuda)
    which = [0, 1, 1, 0]
    res = tune.tune_plan(plan, which, ["a", "b", "c", "d"], None, crossover=False)
    assert res["items_per_sm"] == best and plan.items == best and not res["cached"]
    assert set(res["ms"]) == {str(c) for c in tune.CANDIDATES}
    plan.items = 1
    again = tune.tune_plan(plan, which, ["a", "b", "c", "d"], None, crossover=False)
    assert again["cached"] and plan.items == best
    # a different mix of queries is another workload
    assert tune.workload_key(plan, [0, 0, 1]) != tune.workload_key(plan, which)


def _bare_server(budget, max_batch=4, max_wait_s=0.01):
    srv = object.__new__(serve.Server)
    srv._pending = queue.Queue()
    srv._lock = threading.Lock()
    srv._lane_free = threading.Condition(srv._lock)
    srv.max_batch = max_batch
    srv.max_wait_s = max_wait_s
    srv.budget = budget
    srv.reserved = 0
    return srv


def _req(nbytes, tag):
    r = types.SimpleNamespace(nbytes=nbytes, tag=tag)
    return r


def test_batches_take_waiting_requests_in_order_up_to_max_batch():
    srv = _bare_server(budget=1 << 30, max_batch=3)
    for i in range(5):
        srv._pending.put(_req(10, i))
    assert [r.tag for r in srv._take_batch()] == [0, 1, 2]
    assert [r.tag for r in srv._take_batch()] == [3, 4]
    srv._pending.put(_req(10, 5))
    srv._pending.put(None)                    # shutdown after the waiting request
    assert [r.tag for r in srv._take_batch()] == [5]
    assert srv._take_batch() is None          # the sentinel was put back


def test_admission_keeps_the_budget_and_requeues_the_rest():
    srv = _bare_server(budget=100)
    batch = [_req(40, i) for i in range(4)]
    take, used = srv._admit(batch)
    assert [r.tag for r in take] == [0, 1] and used == 80 and srv.reserved == 80
    assert [srv._pending.get_nowait().tag for _ in range(2)] == [2, 3]
    # a request that does not fit waits until a batch releases its memory
    out = {}
    t = threading.Thread(target=lambda: out.update(res=srv._admit([_req(40, 9)])))
    t.start()
    t.join(timeout=0.2)
    assert t.is_alive()
    with srv._lock:
        srv.reserved -= 80
        srv._lane_free.notify_all()
    t.join(timeout=5)
    assert not t.is_alive() and [r.tag for r in out["res"][0]] == [9]


def test_overlaps_count_pairs_of_batches_from_different_lanes():
    srv = object.__new__(serve.Server)
    spans = [(0, 0.0, 10.0), (1, 5.0, 15.0), (0, 12.0, 20.0), (1, 21.0, 22.0), (0, 21.5, 23.0)]
    srv.device_spans = lambda: spans
    # (0:0-10, 1:5-15), (1:5-15, 0:12-20), (1:21-22, 0:21.5-23)
    assert srv.device_overlaps() == 3


def test_poisson_arrivals_are_seeded_and_have_the_rate():
    a = serve.poisson_arrivals(1000.0, 20000, seed=3)
    assert np.array_equal(a, serve.poisson_arrivals(1000.0, 20000, seed=3))
    assert np.all(np.diff(a) > 0)
    assert abs(len(a) / a[-1] - 1000.0) < 30.0
