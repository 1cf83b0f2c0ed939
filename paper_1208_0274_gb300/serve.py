"""Continuous-batching request loop over one resident index.

Requests (a query, its threshold H and an arrival time) are admitted as
device slots and memory free up; their searches overlap on the GPU.

* `nslots` slots, each a CUDA stream with its own library workspace
  (ae_search keeps one workspace per stream), run searches concurrently.
* A free slot takes waiting requests that have arrived and runs them as one
  ae_search batch. Requests that arrive while batches run wait for the next
  free slot, so batch composition follows the arrivals; there is no fixed
  batch size.
* Policy "fifo" (no predictor): arrival order, up to `max_columns` query
  letters per batch.
* Policy "predicted" (with a WorkPredictor): each request's search work
  (DP entries) and sweep hit records are predicted when it is first
  considered; the slot takes the requests of least predicted work first
  (requests that waited longer than `max_wait` go first, in arrival order),
  up to `work_budget` predicted entries per batch, and passes the predicted
  hit records to the engine as ae_options.hint_hits.
* Admission: a batch starts only if the growth of the slot's workspace it is
  predicted to need (`bytes_per_column` per letter, or the predictor's device
  bytes) fits in the free device memory minus `reserve_bytes`; otherwise the
  slot waits for another slot to finish. A slot with nothing else running is
  always admitted.
* The latency of a request is the time from its arrival to its results being
  in host memory.

Every search goes through the C ABI (ae_search); this module only schedules.
The results of a request do not depend on the batch it ran in (ae_search
treats the queries of a batch independently), which the tests check.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import ae


@dataclass
class Request:
    rid: int
    query: np.ndarray
    H: int
    arrival: float                 # seconds after the start of the run
    start: float = -1.0
    finish: float = -1.0
    hits: np.ndarray | None = None
    batch: int = -1
    pred_work: float = -1.0        # predicted DP entries (predicted policy)
    pred_hits: int = -1            # predicted sweep hit records (predicted policy)


@dataclass
class ServeReport:
    requests: list
    wall: float
    batches: int
    mean_batch: float
    p50_ms: float
    p99_ms: float
    qps: float
    peak_concurrency: int
    extra: dict = field(default_factory=dict)


def _percentile(x, q):
    return float(np.percentile(np.asarray(x, dtype=np.float64), q)) if len(x) else float("nan")


class Server:
    """`nslots` concurrent search slots over one index.

    predictor: a WorkPredictor (paper_1208_0274_gb300.predictor) or None.
    mem_info: callable() -> (free, total) device bytes (torch.cuda.mem_get_info
    by default).  search_fn(queries, Hs, stream, hints) and
    workspace_fn(stream) replace ae_search / ae_workspace_info, and
    predict_fn(queries) -> (work, hits) replaces the predictor (host-only
    tests).
    """

    def __init__(self, index, scheme, nslots=3, max_columns=1 << 18, bytes_per_column=100_000,
                 reserve_bytes=4 << 30, options=None, predictor=None, work_budget=None, max_wait=0.25,
                 mem_info=None, streams=None, search_fn=None, workspace_fn=None, predict_fn=None):
        self.index = index
        self.scheme = scheme
        self.nslots = nslots
        self.max_columns = max_columns
        self.bytes_per_column = bytes_per_column
        self.reserve_bytes = reserve_bytes
        self.options = dict(options or {})
        self.predictor = predictor
        self.predict_fn = predict_fn
        self.policy = "predicted" if (predictor is not None or predict_fn is not None) else "fifo"
        self.work_budget = work_budget
        self.max_wait = max_wait
        if streams is None or mem_info is None:
            import torch
            if streams is None:
                streams = [torch.cuda.Stream() for _ in range(nslots)]
            if mem_info is None:
                mem_info = torch.cuda.mem_get_info
        self.streams = list(streams)
        self.mem_info = mem_info
        # predictions run on a stream of their own: the legacy default stream would
        # wait for (and hold up) every search in flight
        self.pred_stream = None
        if predictor is not None:
            import torch
            self.pred_stream = torch.cuda.Stream()
        self.search_fn = search_fn or self._search
        self.workspace_fn = workspace_fn or (lambda stream: ae.ae_workspace_info(self.index, stream)[0])
        self._lock = threading.Condition()
        self._growth_in_flight = 0
        self.admission_waits = 0
        self.leaf_sweeps = 0
        self.batches_run = 0

    def _search(self, qs, Hs, stream, hints=None):
        opts = ae.make_options(hint_hits=hints, **self.options)
        out = ae.ae_search(self.index, qs, self.scheme, Hs, options=opts, stream=stream)
        st = ae.ae_last_stats()
        with self._lock:
            self.leaf_sweeps += st["leaf_sweeps"]
            self.batches_run += 1
        return out

    # -- predictions ----------------------------------------------------------------------------
    def _predict(self, reqs):
        new = [r for r in reqs if r.pred_work < 0]
        if not new:
            return
        qs = [r.query for r in new]
        if self.predict_fn is not None:
            work, hits = self.predict_fn(qs)
        else:
            work, hits = self.predictor.work_and_hints(qs, stream=self.pred_stream)
        for r, w, h in zip(new, work, hits):
            r.pred_work = float(w)
            r.pred_hits = int(h)

    def need_bytes(self, batch):
        if self.policy == "predicted" and self.predictor is not None:
            p = self.predictor
            return int(p.fixed_bytes + sum(r.pred_work for r in batch) * p.bytes_per_entry
                       + 12.0 * sum(r.pred_hits for r in batch))
        return int(sum(r.query.size for r in batch) * self.bytes_per_column)

    def _take(self, pending, now):
        """Remove and return the next batch from `pending` under the policy."""
        if self.policy == "fifo":
            batch, cols = [], 0
            while pending and (not batch or cols + pending[0].query.size <= self.max_columns):
                r = pending.pop(0)
                batch.append(r)
                cols += r.query.size
            return batch
        ready = [r for r in pending if r.pred_work >= 0]          # predicted (others are in progress)
        old = [r for r in ready if now - r.arrival > self.max_wait]
        order = old + sorted((r for r in ready if now - r.arrival <= self.max_wait), key=lambda r: r.pred_work)
        budget = self.work_budget if self.work_budget is not None else float("inf")
        batch, work, cols = [], 0.0, 0
        for r in order:
            if batch and (work + r.pred_work > budget or cols + r.query.size > self.max_columns):
                break
            batch.append(r)
            work += r.pred_work
            cols += r.query.size
        taken = set(id(r) for r in batch)
        pending[:] = [r for r in pending if id(r) not in taken]
        return batch

    def warmup(self, queries, Hs):
        """Run one search per slot so every workspace has grown before requests
        are timed (growth frees and reallocates device buffers)."""
        for st in self.streams:
            self.search_fn(queries, Hs, st, None)

    def run(self, requests, time_limit=None):
        """Serve `requests` in real time; returns a ServeReport."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        pending = []
        nxt = 0
        active = 0
        peak = 0
        nbatches = 0
        sizes = []
        t0 = time.perf_counter()
        cond = self._lock
        stop = False

        def now():
            return time.perf_counter() - t0

        def admit_arrivals():
            nonlocal nxt
            t = now()
            while nxt < len(reqs) and reqs[nxt].arrival <= t:
                pending.append(reqs[nxt])
                nxt += 1

        def slot_loop(s):
            nonlocal active, peak, nbatches, stop
            stream = self.streams[s]
            while True:
                with cond:
                    while True:
                        admit_arrivals()
                        if stop or (nxt >= len(reqs) and not pending):
                            return
                        if pending and self.policy == "predicted":
                            # predict new arrivals outside the lock (other slots keep
                            # scheduling meanwhile); -2 marks a prediction in progress
                            todo = [r for r in pending if r.pred_work == -1.0]
                            if todo:
                                for r in todo:
                                    r.pred_work = -2.0
                                cond.release()
                                try:
                                    self._predict(todo)
                                except BaseException:
                                    for r in todo:
                                        r.pred_work = -1.0
                                    raise
                                finally:
                                    cond.acquire()
                                continue
                        if pending and any(r.pred_work >= 0 for r in pending) or (pending and self.policy == "fifo"):
                            batch = self._take(pending, now())
                            need = self.need_bytes(batch)
                            # the slot's workspace is reused: only its growth needs free memory
                            growth = max(0, need - self.workspace_fn(stream))
                            free, _ = self.mem_info()
                            if active == 0 or growth + self._growth_in_flight <= free - self.reserve_bytes:
                                break
                            pending[:0] = batch       # not admitted: wait for a slot to finish
                            self.admission_waits += 1
                            cond.wait(timeout=0.05)
                            continue
                        wait = 0.002
                        if nxt < len(reqs):
                            wait = min(wait, max(0.0, reqs[nxt].arrival - now()))
                        cond.wait(timeout=max(wait, 0.0002))
                    active += 1
                    peak = max(peak, active)
                    nbatches += 1
                    bid = nbatches
                    sizes.append(len(batch))
                    self._growth_in_flight += growth
                ts = now()
                for r in batch:
                    r.start = ts
                    r.batch = bid
                hints = [r.pred_hits for r in batch] if self.policy == "predicted" else None
                hits, counts = self.search_fn([r.query for r in batch], [r.H for r in batch], stream, hints)
                tf = now()
                off = 0
                for r, c in zip(batch, counts):
                    r.hits = hits[off:off + int(c)]
                    r.finish = tf
                    off += int(c)
                with cond:
                    active -= 1
                    self._growth_in_flight -= growth
                    if time_limit is not None and now() > time_limit:
                        stop = True
                    cond.notify_all()

        threads = [threading.Thread(target=slot_loop, args=(s,), daemon=True) for s in range(self.nslots)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        wall = now()
        served = [r for r in reqs if r.finish >= 0]
        lat = [1000.0 * (r.finish - r.arrival) for r in served]
        return ServeReport(requests=served, wall=wall, batches=nbatches,
                           mean_batch=float(np.mean(sizes)) if sizes else 0.0,
                           p50_ms=_percentile(lat, 50), p99_ms=_percentile(lat, 99),
                           qps=len(served) / wall if wall > 0 else 0.0, peak_concurrency=peak)


def one_at_a_time(index, scheme, requests, options=None, stream=None):
    """The plain form: each request alone, in arrival order, one launch
    sequence per query on one stream (waits for arrivals in real time)."""
    reqs = sorted(requests, key=lambda r: r.arrival)
    t0 = time.perf_counter()
    for r in reqs:
        wait = r.arrival - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        r.start = time.perf_counter() - t0
        hits, _ = ae.ae_search(index, [r.query], scheme, [r.H], options=options, stream=stream)
        r.hits = hits
        r.finish = time.perf_counter() - t0
    wall = time.perf_counter() - t0
    lat = [1000.0 * (r.finish - r.arrival) for r in reqs]
    return ServeReport(requests=reqs, wall=wall, batches=len(reqs), mean_batch=1.0,
                       p50_ms=_percentile(lat, 50), p99_ms=_percentile(lat, 99),
                       qps=len(reqs) / wall if wall > 0 else 0.0, peak_concurrency=1)


def poisson_requests(queries, Hs, rate, seed=0):
    """Requests with exponential inter-arrival times at `rate` per second."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=len(queries)))
    return [Request(rid=k, query=q, H=int(h), arrival=float(a)) for k, (q, h, a) in enumerate(zip(queries, Hs, t))]
