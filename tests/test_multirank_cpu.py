"""The N > 1 host paths on CPU ranks (gloo, real work, no GPU).

* Query sharding (bench.py under torchrun): each rank runs the oracle on its
  shard of the queries; the shards partition the queries, the job time is the
  maximum and the work the sum over ranks, and the ranks' results together are
  the results of all queries.
* One search split over ranks (multirank.split_search): each rank searches
  its part of the forks -- here the oracle restricted to the start columns
  y with y % R == rank, the share of the forks a part owns -- the results are
  exchanged keyed on text end and merged by the per-cell maximum, and rank 0
  must hold exactly the unrestricted oracle's results.
* A rank that leaves before the exchange makes the others raise SplitError
  (no partial results) within their process group's timeout.
"""
import datetime
import os
import socket
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
import oracle  # noqa: E402
from workloads import Scheme, random_pair  # noqa: E402

SCHEME = Scheme(1, -3, -5, -2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port, timeout_s=60):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=timeout_s))


def _problem(seed=3, n=6_000, nq=5):
    rng = np.random.default_rng(seed)
    T, _ = random_pair(n, 1, seed=seed)
    qs = []
    for k in range(nq):
        _, P = random_pair(1, int(rng.integers(80, 400)), seed=seed * 100 + k)
        L = min(P.size - 6, 60 + 20 * k)
        x = int(rng.integers(0, n - L))
        P[5:5 + L] = T[x:x + L]
        qs.append(P)
    return T, qs, [14 + k for k in range(nq)]


def _collect(q, procs, n, timeout=300):
    """n results from the ranks' queue; fails at once if a rank crashed."""
    import queue as _queue
    out, t0 = [], time.time()
    while len(out) < n:
        try:
            out.append(q.get(timeout=2))
        except _queue.Empty:
            dead = [p.exitcode for p in procs if p.exitcode not in (None, 0)]
            assert not dead, f"a rank crashed: exit codes {dead}"
            assert time.time() - t0 < timeout, "ranks timed out"
    return out


def _hits(oi, oj, os_):
    from paper_1208_0274_gb300 import ae
    w = np.zeros(oi.size, dtype=ae.HIT_DTYPE)
    w["text_end"], w["query_end"], w["score"] = oi, oj, os_
    return w


def _numpy_merge(records, nq):
    """Per-cell maximum of (query, text end, query end, score) records, grouped
    by query and sorted -- the contract of ae_hits_merge, on the host."""
    from paper_1208_0274_gb300 import ae
    if records.shape[0] == 0:
        return np.zeros(0, dtype=ae.HIT_DTYPE), np.zeros(nq, dtype=np.int64)
    r = records[np.lexsort((records[:, 2], records[:, 1], records[:, 0]))]
    new = np.r_[True, np.any(r[1:, :3] != r[:-1, :3], axis=1)]
    grp = np.cumsum(new) - 1
    best = np.full(int(grp[-1]) + 1, np.iinfo(np.int64).min)
    np.maximum.at(best, grp, r[:, 3])
    u = r[new]
    h = np.zeros(u.shape[0], dtype=ae.HIT_DTYPE)
    h["text_end"], h["query_end"], h["score"] = u[:, 1], u[:, 2], best
    return h, np.bincount(u[:, 0], minlength=nq).astype(np.int64)


def _shard_rank(rank, world, port, out):
    _init(rank, world, port)
    T, qs, Hs = _problem()
    mine = bench.shard(len(qs), rank, world)
    t0 = time.perf_counter()
    res = {k: oracle.sw_hits(T, qs[k], SCHEME, Hs[k]) for k in mine}
    ms = 1000 * (time.perf_counter() - t0)
    units = sum(qs[k].size * T.size for k in mine)
    tot_ms, tot_units = bench.job_totals(ms, units, dist, device="cpu")
    out.put((rank, mine, ms, tot_ms, tot_units, res))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_queries_and_aggregate():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(_collect(q, procs, world), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    T, qs, Hs = _problem()
    shards = [r[1] for r in res]
    assert sorted(k for sh in shards for k in sh) == list(range(len(qs)))     # a partition
    assert all(set(a).isdisjoint(b) for a in shards for b in shards if a is not b)
    want_units = sum(p.size for p in qs) * T.size
    for _, _, _, tot_ms, tot_units, _ in res:
        assert tot_ms == pytest.approx(max(r[2] for r in res)) and tot_units == want_units
    got = {}
    for r in res:
        got.update(r[5])
    for k in range(len(qs)):
        want = oracle.sw_hits(T, qs[k], SCHEME, Hs[k])
        assert all(np.array_equal(a, b) for a, b in zip(got[k], want))


def _split_rank(rank, world, port, out, leave=False):
    from paper_1208_0274_gb300 import multirank
    _init(rank, world, port, timeout_s=15)
    T, qs, Hs = _problem(seed=7, nq=4)

    def search(part, parts):
        if leave and part == 1:
            os._exit(0)          # this rank leaves between steps, with nothing in flight
        hs, cs = [], []
        for P, H in zip(qs, Hs):
            allowed = (np.arange(P.size) % parts) == part
            h = _hits(*oracle.sw_hits_starts(T, P, SCHEME, H, allowed))
            hs.append(h)
            cs.append(h.size)
        return np.concatenate(hs), np.array(cs, dtype=np.int64)

    try:
        r = multirank.split_search(None, qs, SCHEME, Hs, dist, search=search, merge=_numpy_merge,
                                   n_text=T.size, max_query_len=max(q.size for q in qs))
        out.put((rank, "ok", r))
    except multirank.SplitError as e:
        out.put((rank, "split_error", str(e)))
    try:
        dist.destroy_process_group()
    except Exception:
        pass


@pytest.mark.parametrize("world", [2, 3])
def test_split_search_exchange_equals_unsplit_oracle(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(_collect(q, procs, world), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
    assert all(r[1] == "ok" for r in res), res
    hits, counts = res[0][2]
    assert all(r[2] is None for r in res[1:])
    T, qs, Hs = _problem(seed=7, nq=4)
    parts = np.split(hits, np.cumsum(counts)[:-1])
    for k, (P, H) in enumerate(zip(qs, Hs)):
        want = _hits(*oracle.sw_hits(T, P, SCHEME, H))
        assert want.size > 0 and np.array_equal(parts[k], want), k
    # the maxima come from more than one part: the exchange is needed
    suppliers = set()
    for P, H in zip(qs, Hs):
        full = {(int(a), int(b)): int(c) for a, b, c in _hits(*oracle.sw_hits(T, P, SCHEME, H))}
        for r in range(world):
            part = _hits(*oracle.sw_hits_starts(T, P, SCHEME, H, (np.arange(P.size) % world) == r))
            if any(full.get((int(a), int(b))) == int(c) for a, b, c in part):
                suppliers.add(r)
    assert len(suppliers) > 1


def test_split_search_rank_that_leaves_gives_error_not_partial_results():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_rank, args=(r, world, port, q, True)) for r in range(world)]
    for p in procs:
        p.start()
    res = _collect(q, procs, 1, timeout=120)[0]
    for p in procs:
        p.join(timeout=60)
    assert res[0] == 0 and res[1] == "split_error"


def test_single_rank_totals_are_local():
    assert bench.job_totals(12.5, 7) == (12.5, 7.0)
    assert bench.shard(5, 0, 1) == [0, 1, 2, 3, 4]


def test_owner_ranges_partition_the_text():
    from paper_1208_0274_gb300 import multirank
    te = np.arange(0, 1001)
    for world in (1, 2, 3, 8):
        own = multirank.owner_of(te, 1001, world)
        assert own.min() == 0 and own.max() == world - 1
        assert np.all(np.diff(own) >= 0)          # contiguous, increasing ranges
