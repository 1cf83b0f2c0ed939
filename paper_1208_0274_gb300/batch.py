"""Many queries against one resident index, spread over concurrent streams.

search_many(index, queries, Hs, ...) splits the queries into `nstreams`
groups, searches each group with one ae_search_device call on its own CUDA
stream (each stream has its own library workspace, and the engine processes
a group in batches of `batch_columns` query letters), and returns the results
in input order.  Groups run concurrently, so one group's host synchronisation
and text-position-sweep tail overlap the others' kernels.

Packing of queries onto streams:
  * "round_robin": query k goes to stream k mod nstreams, and each stream
    takes its queries in input order (static);
  * "lpt": queries in decreasing order of predicted work (DP entries, from a
    WorkPredictor) each go to the stream with the least predicted work so far
    (longest processing time first), so the streams finish together; each
    stream then takes its queries in decreasing order of predicted work, so
    the engine's consecutive batches hold queries of similar work and the
    heavy ones share batches (their sweep tails overlap instead of each
    lengthening a different batch).
The packing never changes a result: every query is searched independently.
"""
from __future__ import annotations

import threading

import numpy as np

from . import ae


def pack_round_robin(n, nstreams):
    return [list(range(s, n, nstreams)) for s in range(nstreams)]


def pack_lpt(work, nstreams):
    """Longest-processing-time-first assignment of items with `work` to
    `nstreams` bins; each bin keeps its items in input order."""
    load = np.zeros(nstreams)
    bins = [[] for _ in range(nstreams)]
    for k in np.argsort(-np.asarray(work, dtype=np.float64), kind="stable"):
        s = int(np.argmin(load))
        bins[s].append(int(k))
        load[s] += float(work[k])
    return [sorted(b) for b in bins]


def search_many(index, queries, Hs, scheme, nstreams=2, policy="round_robin", predictor=None, options=None,
                streams=None, hint_hits=None):
    """Returns (hits per query as a list of HIT_DTYPE arrays, info dict).
    `options` is a dict of ae_options fields; `hint_hits` (per query) or a
    predictor's hit hints size each group's sweep buffers.  Streams made here
    (streams=None) have their library workspaces released before returning;
    the workspaces of caller streams are kept for the next call."""
    import torch
    n = len(queries)
    if policy == "lpt":
        if predictor is None:
            raise ValueError("lpt packing needs a predictor")
        work = predictor.work(queries)
        groups = [sorted(g, key=lambda k: -work[k]) for g in pack_lpt(work, nstreams)]
        if hint_hits is None:
            hint_hits = predictor.hint_hits(queries)
    elif policy == "round_robin":
        groups = pack_round_robin(n, nstreams)
    else:
        raise ValueError(policy)
    own = streams is None
    if own:
        streams = [torch.cuda.Stream() for _ in range(nstreams)]
    out = [None] * n
    errors = []
    launches = [0] * nstreams
    sweeps = [0] * nstreams

    def run(s):
        try:
            idx = groups[s]
            if not idx:
                return
            qs = [ae._u8(queries[k]) for k in idx]
            seq = np.concatenate(qs)
            offsets = np.concatenate([[0], np.cumsum([q.size for q in qs])]).astype(np.int64)
            st = streams[s]
            with torch.cuda.stream(st):
                d_seq = torch.from_numpy(seq).to("cuda", non_blocking=False)
            hints = None if hint_hits is None else [int(hint_hits[k]) for k in idx]
            opts = ae.make_options(hint_hits=hints, **(options or {}))
            cap = max(1 << 16, sum(q.size for q in qs))
            while True:
                with torch.cuda.stream(st):
                    d_hits = torch.empty(cap * 16, dtype=torch.uint8, device="cuda")
                status, counts = ae.ae_search_device(index, d_seq.data_ptr(), offsets, scheme, [Hs[k] for k in idx],
                                                     d_hits.data_ptr(), cap, options=opts, stream=st)
                stats = ae.ae_last_stats()
                launches[s] += stats["launches"]
                sweeps[s] += stats["leaf_sweeps"]
                if status == ae.AE_OK:
                    break
                if status != ae.AE_EOVERFLOW:
                    raise ae.AEError(status, "ae_search_device")
                cap = int(counts.sum()) + 1024
            total = int(counts.sum())
            with torch.cuda.stream(st):
                h = d_hits[: total * 16].cpu().numpy().view(ae.HIT_DTYPE)
            starts = np.concatenate([[0], np.cumsum(counts)])
            for j, k in enumerate(idx):
                out[k] = h[starts[j]:starts[j + 1]]
        except BaseException as e:   # surfaced to the caller below
            errors.append(e)

    threads = [threading.Thread(target=run, args=(s,)) for s in range(nstreams)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if own:      # workspaces are kept per stream: free those of streams made here
        for st in streams:
            ae.ae_workspace_release(index, st)
    if errors:
        raise errors[0]
    return out, {"groups": [len(g) for g in groups], "launches": int(sum(launches)), "leaf_sweeps": int(sum(sweeps))}
