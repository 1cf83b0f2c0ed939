"""Host logic of the request loop (paper_1208_0274_gb300.serve) with a fake
search: arrivals are admitted while other batches run, batches follow the
arrivals, admission keeps the predicted workspace growth within the free
device memory, and every request gets the results of its own query."""
import threading
import time

import numpy as np

from paper_1208_0274_gb300 import serve


def _fake_hits(q):
    # a deterministic per-query result that depends on the query only
    v = int(q.astype(np.int64).sum())
    n = 1 + v % 5
    out = np.zeros(n, dtype=[("text_end", "<i8"), ("query_end", "<i4"), ("score", "<i4")])
    out["text_end"] = v + np.arange(n)
    out["query_end"] = q.size - 1
    out["score"] = 30 + n
    return out


class FakeDevice:
    def __init__(self, total):
        self.total = total
        self.used = 0
        self.ws = {}
        self.peak_used = 0
        self.lock = threading.Lock()
        self.concurrent = 0
        self.peak_concurrent = 0

    def mem_info(self):
        with self.lock:
            return self.total - self.used, self.total

    def workspace(self, stream):
        with self.lock:
            return self.ws.get(stream, 0)

    def search(self, qs, Hs, stream, bytes_per_col):
        need = sum(q.size for q in qs) * bytes_per_col
        with self.lock:
            grow = max(0, need - self.ws.get(stream, 0))
            self.used += grow
            self.ws[stream] = self.ws.get(stream, 0) + grow
            assert self.used <= self.total, "admitted beyond the device memory"
            self.peak_used = max(self.peak_used, self.used)
            self.concurrent += 1
            self.peak_concurrent = max(self.peak_concurrent, self.concurrent)
        time.sleep(0.002 + 1e-6 * sum(q.size for q in qs))
        hits = [_fake_hits(q) for q in qs]
        with self.lock:
            self.concurrent -= 1
        return np.concatenate(hits), np.array([h.size for h in hits], dtype=np.int64)


def _requests(k, rate, seed):
    rng = np.random.default_rng(seed)
    qs = [rng.integers(0, 4, size=int(rng.integers(200, 5000))).astype(np.uint8) for _ in range(k)]
    return serve.poisson_requests(qs, [25] * k, rate, seed=seed)


def test_requests_are_admitted_while_others_run_and_get_their_own_results():
    dev = FakeDevice(total=1 << 40)
    reqs = _requests(120, rate=2000.0, seed=1)
    srv = serve.Server(None, None, nslots=3, bytes_per_column=1000, reserve_bytes=0, mem_info=dev.mem_info,
                       streams=["s0", "s1", "s2"], workspace_fn=dev.workspace,
                       search_fn=lambda qs, Hs, st, hints: dev.search(qs, Hs, st, 1000))
    rep = srv.run(reqs)
    assert len(rep.requests) == 120
    for r in rep.requests:
        assert np.array_equal(r.hits, _fake_hits(r.query))
        assert r.finish >= r.start >= r.arrival - 1e-9
    assert rep.peak_concurrency >= 2 and dev.peak_concurrent >= 2
    assert rep.mean_batch > 1.0            # arrivals during a batch join the next one
    assert rep.batches < 120
    assert rep.p99_ms >= rep.p50_ms > 0


def test_admission_keeps_workspace_growth_within_free_memory():
    bpc = 1000
    total = 3 * 5000 * bpc + 2000 * bpc     # room for about three large batches at once
    dev = FakeDevice(total=total)
    reqs = _requests(60, rate=5000.0, seed=2)
    srv = serve.Server(None, None, nslots=4, max_columns=5000, bytes_per_column=bpc, reserve_bytes=0,
                       mem_info=dev.mem_info, streams=[0, 1, 2, 3], workspace_fn=dev.workspace,
                       search_fn=lambda qs, Hs, st, hints: dev.search(qs, Hs, st, bpc))
    rep = srv.run(reqs)                     # FakeDevice.search asserts used <= total
    assert len(rep.requests) == 60
    assert dev.peak_used <= total
    for r in rep.requests:
        assert np.array_equal(r.hits, _fake_hits(r.query))


def test_a_lone_slot_is_always_admitted():
    # with nothing running, a batch larger than the free memory still runs (the
    # search itself then reports AE_ENOMEM or succeeds); the loop never stalls
    dev = FakeDevice(total=10)
    reqs = _requests(5, rate=1000.0, seed=3)
    srv = serve.Server(None, None, nslots=2, bytes_per_column=0, reserve_bytes=100, mem_info=dev.mem_info,
                       streams=[0, 1], workspace_fn=dev.workspace,
                       search_fn=lambda qs, Hs, st, hints: dev.search(qs, Hs, st, 0))
    rep = srv.run(reqs)
    assert len(rep.requests) == 5


def test_poisson_arrivals_have_the_requested_rate():
    reqs = serve.poisson_requests([np.zeros(1, np.uint8)] * 20_000, [1] * 20_000, rate=200.0, seed=4)
    t = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(t) >= 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 200.0) < 0.05 / 200.0
    assert abs(gaps.std() - 1 / 200.0) < 0.05 / 200.0     # exponential: sd = mean


def test_predicted_policy_takes_least_work_first_within_a_budget_and_passes_hints():
    dev = FakeDevice(total=1 << 40)
    seen = []

    def search(qs, Hs, st, hints):
        seen.append(([q.size for q in qs], list(hints)))
        return dev.search(qs, Hs, st, 1)

    # all requests are waiting when the single slot first looks: it must take
    # them in order of predicted work (= length here), budget-limited
    reqs = _requests(40, rate=1e9, seed=5)
    srv = serve.Server(None, None, nslots=1, bytes_per_column=0, reserve_bytes=0, mem_info=dev.mem_info,
                       streams=[0], workspace_fn=dev.workspace, search_fn=search, work_budget=6000,
                       max_wait=1e9, predict_fn=lambda qs: ([float(q.size) for q in qs], [7 * q.size for q in qs]))
    rep = srv.run(reqs)
    assert len(rep.requests) == 40
    for r in rep.requests:
        assert np.array_equal(r.hits, _fake_hits(r.query))
    sizes0, hints0 = seen[0]
    assert hints0 == [7 * m for m in sizes0]
    assert sizes0 == sorted(sizes0) and (sum(sizes0) <= 6000 or len(sizes0) == 1)
    smallest = min(q.query.size for q in reqs)
    assert sizes0[0] == smallest


def test_requests_waiting_longer_than_max_wait_go_first():
    dev = FakeDevice(total=1 << 40)
    order = []

    def search(qs, Hs, st, hints):
        order.extend(q.size for q in qs)
        return dev.search(qs, Hs, st, 1)

    big = np.zeros(50_000, np.uint8)
    small = [np.zeros(100 + k, np.uint8) for k in range(30)]
    reqs = [serve.Request(rid=0, query=big, H=1, arrival=0.0)]
    reqs += [serve.Request(rid=k + 1, query=q, H=1, arrival=0.0) for k, q in enumerate(small)]
    srv = serve.Server(None, None, nslots=1, bytes_per_column=0, reserve_bytes=0, mem_info=dev.mem_info,
                       streams=[0], workspace_fn=dev.workspace, search_fn=search, work_budget=500,
                       max_wait=0.0, predict_fn=lambda qs: ([float(q.size) for q in qs], [0] * len(qs)))
    time.sleep(0.01)
    srv.run(reqs)
    assert order[0] == 50_000          # waited past max_wait: goes first despite its size
