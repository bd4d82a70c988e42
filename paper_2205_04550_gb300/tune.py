"""Autotuner for query plans.

The persistent plan launch splits every query into work items (slices of
its database entries); how many items per SM balance the grid best depends
on the GPU, the databases' sizes and resolutions, the batch size and whether
the scans are sparse.  ``tune_plan`` times the candidate settings with CUDA
events on the real inputs, keeps the fastest, and caches it per
(GPU, workload key) in a JSON file so later runs reuse it without timing.
Every setting returns identical hits; only the speed differs.
"""
from __future__ import annotations

import json
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(_HERE, "_build", "autotune.json")
CANDIDATES = (1, 2, 4, 8, 16, 32, 64)
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


def tune_plan(plan, which, patients_dev, hits_dev, candidates=CANDIDATES, reps: int = 3,
              use_cache: bool = True, sparse_flags=None) -> dict:
    """Choose DBQ_PLAN_ITEMS_PER_SM for this plan and workload; sets it on the
    plan and returns {"items_per_sm": best, "ms": {candidate: ms}}."""
    import torch
    key = workload_key(plan, list(which), sparse_flags)
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            plan.set_items_per_sm(int(hit["items_per_sm"]))
            return dict(hit, cached=True)
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
    return dict(out, cached=False)
