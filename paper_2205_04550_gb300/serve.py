"""Continuous-batching query server over resident databases.

Single-patient requests arrive at any time.  A scheduler thread gathers the
waiting requests into batches of up to ``max_batch`` queries -- admitting a
request only while the device-memory budget has room for its patient slot
and its share of the batch workspace -- and hands each batch to a free
*lane*: a CUDA stream with its own pinned staging, device patient slots,
device hit buffer and query plan.  Lanes run concurrently, so a batch that
is admitted while others are on the GPU overlaps with them on the device.

Two query paths, matching the library's modes:

* ``exact``: one persistent launch (``db_plan_query``) per batch over all of
  its queries, whatever database each query names;
* ``embed_bf16`` / ``embed_fp8`` / ``hash``: per database in the batch, the
  tensor-core embedding prefilter (or the Hamming prefilter on sign codes of
  a sketch database) plus exact re-ranking (``db_query_batch``); a database
  handle serialises its own batches (its prefilter workspace is shared), so
  embedding batches overlap across databases.

Results are per request (the ranked hits), latency is completion minus
arrival, and ``stats()`` reports p50/p99 latency and completed queries/s.
Batch composition never changes a request's result: every query is computed
independently (tested).  Each batch's span on its lane's stream (from its
first copy to its last kernel) is recorded with CUDA events, so
``device_overlaps()`` can show that batches of different lanes overlapped on
the device.
"""
from __future__ import annotations

import queue
import threading
import time
from concurrent.futures import Future, ThreadPoolExecutor

import numpy as np

from . import _dbq
from ._dbq import (DBQ_MODE_EMBED_BF16, DBQ_MODE_EMBED_FP8, DBQ_MODE_EXACT, DBQ_MODE_HASH,
                   HIT_DTYPE)

MODES = {"exact": DBQ_MODE_EXACT, "embed_bf16": DBQ_MODE_EMBED_BF16,
         "embed_fp8": DBQ_MODE_EMBED_FP8, "hash": DBQ_MODE_HASH}


class AdmissionError(RuntimeError):
    pass


class _Request:
    __slots__ = ("patient", "db", "future", "t_arrive", "t_done", "nbytes")

    def __init__(self, patient, db, nbytes):
        self.patient = patient
        self.db = db
        self.future = Future()
        self.t_arrive = time.perf_counter()
        self.t_done = None
        self.nbytes = nbytes


class _Lane:
    """One stream with its own staging, device slots and plan."""

    def __init__(self, torch, databases, max_batch, k, max_voxels):
        from . import Plan
        self.torch = torch
        self.stream = torch.cuda.Stream()
        self.max_batch = max_batch
        self.k = k
        self.pinned = torch.empty((max_batch, max_voxels), dtype=torch.float32).pin_memory()
        self.slots = torch.empty((max_batch, max_voxels), dtype=torch.float32, device="cuda")
        self.hits = torch.zeros((max_batch, k * 40), dtype=torch.uint8, device="cuda")
        self.hits_host = torch.zeros((max_batch, k * 40), dtype=torch.uint8).pin_memory()
        self.plan = Plan(databases, max_batch, k)
        self.busy = False

    def close(self):
        self.plan.close()


class Server:
    """Continuous-batching server (see module docstring).

    databases   list of ``Database`` (bit-packed; built with ``embed=True`` for
                the embedding modes), resident for the server's lifetime.
    mode        "exact", "embed_bf16", "embed_fp8" or "hash".
    budget      device bytes the server may hold for requests in flight
                (patient slots and hit buffers); None = 90 % of the free
                memory at start.
    tune        exact mode: time, once per database (cached by ``tune``),
                the batch size from which a batch's queries of that database
                are scanned together on the tensor cores, and use it on every
                lane; otherwise the plans' default threshold applies.
    copy_threads host threads copying a batch's patients into pinned staging.
    """

    def __init__(self, databases, mode: str = "exact", k: int = 10, n_candidates: int = 512,
                 max_batch: int = 128, lanes: int = 2, budget: int | None = None,
                 max_wait_s: float = 0.002, tune: bool = True, copy_threads: int = 8):
        import torch
        self.torch = torch
        self.databases = list(databases)
        if mode not in MODES:
            raise ValueError(f"mode must be one of {sorted(MODES)}")
        self.mode = MODES[mode]
        self.k = k
        self.n_candidates = n_candidates
        self.max_batch = max_batch
        self.max_wait_s = max_wait_s
        self.voxels = [int(np.prod(d.shape)) for d in self.databases]
        max_vox = max(self.voxels)
        free, _ = torch.cuda.mem_get_info()
        self.budget = int(0.9 * free) if budget is None else int(budget)
        self.reserved = 0
        self._lanes = [_Lane(torch, self.databases, max_batch, k, max_vox) for _ in range(lanes)]
        # host copies of the patients into the lanes' pinned staging run on a
        # pool (numpy releases the GIL while copying): a batch of 128 patients
        # is hundreds of MB, more than one thread copies in a plan's time
        self._copy_pool = ThreadPoolExecutor(max_workers=copy_threads)
        self.tc_min = {}
        if tune and self.mode == DBQ_MODE_EXACT:
            self._tune_crossovers()
        self._pending: "queue.Queue[_Request]" = queue.Queue()
        self._lock = threading.Lock()
        self._lane_free = threading.Condition(self._lock)
        self._done: list[_Request] = []
        self._spans: list = []          # (lane, start event, end event) per batch
        self._ref = torch.cuda.Event(enable_timing=True)
        self._ref.record()
        torch.cuda.synchronize()
        self._stop = False
        self._t0 = time.perf_counter()
        self._sched = threading.Thread(target=self._schedule, daemon=True)
        self._sched.start()

    # ------------------------------------------------------------ public
    def submit(self, patient: np.ndarray, db: int) -> Future:
        """Queue one patient volume (float32, the database's grid) against
        database ``db``; the future resolves to its hits (HIT_DTYPE [k])."""
        if not 0 <= db < len(self.databases):
            raise ValueError("no such database")
        vol = np.ascontiguousarray(patient, dtype=np.float32).reshape(-1)
        if vol.size != self.voxels[db]:
            raise ValueError("patient grid does not match the database")
        need = vol.nbytes + self.k * 40
        if need > self.budget:
            raise AdmissionError(f"request needs {need} bytes, budget is {self.budget}")
        req = _Request(vol, db, need)
        self._pending.put(req)
        return req.future

    def stats(self) -> dict:
        with self._lock:
            done = list(self._done)
        if not done:
            return {"completed": 0}
        lat = np.array([r.t_done - r.t_arrive for r in done])
        t_first = min(r.t_arrive for r in done)
        t_last = max(r.t_done for r in done)
        return {"completed": len(done), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_ms": float(lat.mean() * 1e3),
                "queries_per_s": len(done) / max(t_last - t_first, 1e-9)}

    def reset_stats(self):
        with self._lock:
            self._done = []
            self._spans = []

    def device_spans(self) -> list:
        """[(lane, start_ms, end_ms)] of the recorded batches on the device,
        relative to the server's start (synchronises the device)."""
        self.torch.cuda.synchronize()
        with self._lock:
            spans = list(self._spans)
        return [(lane, self._ref.elapsed_time(a), self._ref.elapsed_time(b))
                for lane, a, b in spans]

    def device_overlaps(self) -> int:
        """Pairs of batches from different lanes whose device spans overlap."""
        spans = sorted(self.device_spans(), key=lambda t: t[1])
        pairs = 0
        for i, (li, a0, a1) in enumerate(spans):
            for lj, b0, b1 in spans[i + 1:]:
                if b0 >= a1:
                    break
                if lj != li:
                    pairs += 1
        return pairs

    def close(self):
        self._stop = True
        self._pending.put(None)
        self._sched.join(timeout=30)
        self.torch.cuda.synchronize()
        for lane in self._lanes:
            lane.close()
        self._copy_pool.shutdown(wait=True)

    # ------------------------------------------------------------ internals
    def _tune_crossovers(self):
        """Per database, the tuned tensor-core crossover (zero patients: the
        cost of either dense path does not depend on the patient; a sparse
        database's loop is timed on them as well), set on every lane's plan."""
        from . import tune as _tune
        torch = self.torch
        plan = self._lanes[0].plan
        if plan.max_queries < max(_tune.TC_BATCHES):
            return
        for d, db in enumerate(self.databases):
            pats = [torch.zeros(self.voxels[d], dtype=torch.float32, device="cuda")]
            res = _tune.tune_crossover(plan, d, pats, self._lanes[0].hits,
                                       sparse=getattr(db, "sparse_mode", 0))
            self.tc_min[d] = int(res["tc_min"])
            for lane in self._lanes:
                lane.plan.set_tc_min_queries(self.tc_min[d], db=d)
        torch.cuda.synchronize()

    def _take_batch(self):
        """Block for the first request, then gather more for up to
        max_wait_s while the batch and the memory budget have room."""
        first = self._pending.get()
        if first is None:
            return None
        batch = [first]
        deadline = time.perf_counter() + self.max_wait_s
        while len(batch) < self.max_batch:
            timeout = deadline - time.perf_counter()
            try:
                nxt = self._pending.get(timeout=max(timeout, 0)) if timeout > 0 else \
                    self._pending.get_nowait()
            except queue.Empty:
                break
            if nxt is None:
                self._pending.put(None)
                break
            batch.append(nxt)
        return batch

    def _admit(self, batch):
        """Reserve memory for the batch, waiting for in-flight batches to
        release theirs; requests beyond the budget go back to the queue."""
        with self._lock:
            while True:
                room = self.budget - self.reserved
                take, used = [], 0
                for r in batch:
                    if used + r.nbytes <= room:
                        take.append(r)
                        used += r.nbytes
                if take:
                    self.reserved += used
                    for r in batch[len(take):]:
                        self._pending.put(r)
                    return take, used
                self._lane_free.wait(timeout=0.05)

    def _schedule(self):
        # A lane is claimed before the batch is gathered: while every lane is
        # busy, arriving requests wait in the queue and all of them (up to
        # max_batch) form the next batch, so batches grow with the load and
        # each scan of a database serves as many queries as are waiting.
        while not self._stop:
            with self._lock:
                while True:
                    lane = next((l for l in self._lanes if not l.busy), None)
                    if lane is not None:
                        lane.busy = True
                        break
                    self._lane_free.wait(timeout=0.05)
            batch = self._take_batch()
            if batch is None:
                with self._lock:
                    lane.busy = False
                    self._lane_free.notify_all()
                return
            batch, used = self._admit(batch)
            threading.Thread(target=self._run, args=(lane, batch, used), daemon=True).start()

    def _run(self, lane: _Lane, batch, used: int):
        torch = self.torch
        try:
            n = len(batch)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(lane.stream):
                ev0.record(lane.stream)
                rows = lane.pinned.numpy()

                def stage(i):
                    rows[i, :batch[i].patient.size] = batch[i].patient

                list(self._copy_pool.map(stage, range(n)))
                for i, r in enumerate(batch):
                    lane.slots[i, :r.patient.size].copy_(lane.pinned[i, :r.patient.size],
                                                         non_blocking=True)
                which = [r.db for r in batch]
                if self.mode == DBQ_MODE_EXACT:
                    lane.plan.query(which, [lane.slots[i] for i in range(n)], lane.hits[:n],
                                    kind=_dbq.DBQ_F32, stream=lane.stream)
                    ev1.record(lane.stream)
                    lane.hits_host[:n].copy_(lane.hits[:n], non_blocking=True)
                    lane.stream.synchronize()
                    hits = lane.hits_host[:n].numpy().view(HIT_DTYPE).reshape(n, self.k)
                else:
                    hits = np.zeros((n, self.k), dtype=HIT_DTYPE)
                    for d in sorted(set(which)):
                        idx = [i for i in range(n) if which[i] == d]
                        h, _ = _dbq.db_query_batch(
                            [self.databases[d].handle], [0] * len(idx),
                            [lane.slots[i] for i in idx], self.k, self.mode,
                            self.n_candidates, kind=_dbq.DBQ_F32, stream=lane.stream)
                        hits[idx] = h
                    ev1.record(lane.stream)
            now = time.perf_counter()
            for i, r in enumerate(batch):
                r.t_done = now
                r.future.set_result(hits[i].copy())
            with self._lock:
                self._done.extend(batch)
                if len(self._spans) < 100_000:
                    self._spans.append((self._lanes.index(lane), ev0, ev1))
        except Exception as exc:  # deliver the failure to every request of the batch
            for r in batch:
                if not r.future.done():
                    r.future.set_exception(exc)
        finally:
            with self._lock:
                self.reserved -= used
                lane.busy = False
                self._lane_free.notify_all()


def poisson_arrivals(rate_per_s: float, count: int, seed: int = 7) -> np.ndarray:
    """Arrival times (s) of a Poisson process, seeded."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, count))


def run_open_loop(server: Server, requests, arrivals) -> list:
    """Submit ``requests`` [(patient, db)] at the given arrival times (s from
    now) and wait for all; returns the futures' results in request order."""
    t0 = time.perf_counter()
    futs = []
    for (patient, db), t in zip(requests, arrivals):
        delay = t0 + t - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        futs.append(server.submit(patient, db))
    return [f.result(timeout=600) for f in futs]
