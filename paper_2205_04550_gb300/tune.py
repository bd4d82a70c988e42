"""Autotuner for query plans.

Two choices are tuned, both timed with CUDA events on the real inputs and
cached in a JSON file so later runs reuse them without timing; every setting
returns identical hits, only the speed differs.

* Per database, the batch size from which its queries are scanned all at
  once as a tensor-core contraction instead of one CUDA-core loop per query
  (DBQ_PLAN_TC_MIN_QUERIES for that database; the loop's cost, and so the
  crossover, differs between the dense and the sparse loop).  The loop's cost grows
  with the batch (one AND + POPC per word per query) while the contraction's
  barely does, and where they cross depends on the GPU and on the database's
  resolution and size: ``tune_crossover`` times both paths at batch sizes
  TC_BATCHES and keeps the smallest at which the contraction is no slower
  (cached per GPU, grid and entry count).
* The number of work items per SM of the persistent CUDA-core launch, which
  balances the grid differently for each mix of databases, batch size and
  sparse setting (``tune_plan``, cached per workload).
"""
from __future__ import annotations

import json
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(_HERE, "_build", "autotune.json")
CANDIDATES = (1, 2, 4, 8, 16, 32, 64)
TC_BATCHES = (2, 4, 6, 8, 12, 16, 24, 32)
_lock = threading.Lock()


def _load_cache() -> dict:
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(key: str, value: dict):
    with _lock:
        cache = _load_cache()
        cache[key] = value
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, CACHE)


def workload_key(plan, which, sparse_flags=None) -> str:
    import torch
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    dbs = [(d.shape, d.capacity) for d in plan.databases]
    counts = [which.count(i) for i in range(len(plan.databases))]
    return json.dumps({"gpu": props.name, "sms": props.multi_processor_count, "dbs": dbs,
                       "queries": counts, "k": plan.k, "sparse": sparse_flags},
                      sort_keys=True)


def _time_plan(plan, which, patients, hits_dev, reps: int, stream) -> float:
    import torch
    plan.query(which, patients, hits_dev, stream=stream)             # warm-up
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(reps):
        plan.query(which, patients, hits_dev, stream=stream)
    end.record(stream)
    torch.cuda.synchronize()
    return start.elapsed_time(end) / reps


def crossover_key(db, sparse=False) -> str:
    import torch
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    return json.dumps({"gpu": props.name, "sms": props.multi_processor_count,
                       "crossover": [list(db.shape), db.capacity], "sparse": int(sparse)},
                      sort_keys=True)


def tune_crossover(plan, d: int, patients_dev, hits_dev, batches=TC_BATCHES, reps: int = 2,
                   use_cache: bool = True, sparse: bool = False) -> dict:
    """The smallest batch of TC_BATCHES at which database ``d`` of the plan
    is scanned no slower as a tensor-core contraction than by the CUDA-core
    loop; sets it as that database's threshold and returns {"tc_min": B,
    "ms": {B: [contraction, loop]}}.  ``patients_dev`` are patients of
    database d (cycled to fill a batch); ``hits_dev`` holds k hits for up to
    max(batches) queries.  If the loop wins at every size, the threshold is
    twice the largest size tried.  ``sparse`` names the database's
    DBQ_OPT_SPARSE setting, which changes the loop's cost (cached apart)."""
    import torch
    db = plan.databases[d]
    key = crossover_key(db, sparse)
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            plan.set_tc_min_queries(int(hit["tc_min"]), db=d)
            return dict(hit, cached=True)
    stream = torch.cuda.current_stream()
    timings, best = {}, None
    for b in batches:
        if b > plan.max_queries:
            break
        pats = [patients_dev[i % len(patients_dev)] for i in range(b)]
        which = [d] * b
        plan.set_tc_min_queries(1, db=d)
        t_tc = _time_plan(plan, which, pats, hits_dev, reps, stream)
        plan.set_tc_min_queries(0, db=d)
        t_cc = _time_plan(plan, which, pats, hits_dev, reps, stream)
        timings[str(b)] = [t_tc, t_cc]
        if t_tc <= t_cc:
            best = b
            break
    if best is None:
        best = 2 * max(batches)
    plan.set_tc_min_queries(best, db=d)
    out = {"tc_min": best, "ms": timings}
    _store(key, out)
    return dict(out, cached=False)


def tune_plan(plan, which, patients_dev, hits_dev, candidates=CANDIDATES, reps: int = 3,
              use_cache: bool = True, sparse_flags=None, crossover: bool = True) -> dict:
    """Choose the plan's settings for this workload: first, per database with
    queries, the tensor-core crossover (``tune_crossover``), then
    DBQ_PLAN_ITEMS_PER_SM; sets them on the plan and returns
    {"items_per_sm": best, "ms": {candidate: ms}, "tc_min": {db: B}}."""
    import torch
    which = list(which)
    tc_min = {}
    if crossover:
        for d, db in enumerate(plan.databases):
            mine = [patients_dev[q] for q in range(len(which)) if which[q] == d]
            if mine:
                mode = getattr(db, "sparse_mode", 1 if sparse_flags else 0)
                tc_min[str(d)] = tune_crossover(plan, d, mine, hits_dev, use_cache=use_cache,
                                                sparse=mode)["tc_min"]
    key = workload_key(plan, which, sparse_flags)
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            plan.set_items_per_sm(int(hit["items_per_sm"]))
            return dict(hit, cached=True, tc_min=tc_min)
    stream = torch.cuda.current_stream()
    timings = {}
    for c in candidates:
        plan.set_items_per_sm(c)
        plan.query(which, patients_dev, hits_dev, stream=stream)       # warm-up
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for _ in range(reps):
            plan.query(which, patients_dev, hits_dev, stream=stream)
        end.record(stream)
        torch.cuda.synchronize()
        timings[c] = start.elapsed_time(end) / reps
    best = min(timings, key=timings.get)
    plan.set_items_per_sm(best)
    out = {"items_per_sm": best, "ms": {str(c): t for c, t in timings.items()}}
    _store(key, out)
    return dict(out, cached=False, tc_min=tc_min)
