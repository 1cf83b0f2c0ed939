"""One search split over ranks (one process per GPU), with its result exchange.

The forks of a search are partitioned over the ranks (ae_options.fork_parts /
fork_part: seed subtrees by gram, or start columns for walks from the root).
A cell's largest similarity can come from forks of different ranks, so the
ranks exchange their results keyed on text end -- rank r owns the text ends
[r n / R, (r + 1) n / R) -- with one all-to-all of counts and one of records,
and each owner keeps the per-cell maximum (ae_hits_merge on its device).
Rank 0 then gathers the owners' parts.  Queries are independent, so the same
exchange serves any number of queries at once; the records carry their query.

A rank that fails or leaves makes the collectives of the others raise (their
process group has a finite timeout); split_search then raises SplitError on
every surviving rank instead of returning partial results.
"""
from __future__ import annotations

import numpy as np

from . import ae

RECORD_FIELDS = 4   # query, text end, query end, score (int64 each)


class SplitError(RuntimeError):
    """A rank of a split search failed or left; no result is returned."""


def owner_of(text_end, n_text, world):
    """Rank owning each text end: contiguous ranges of the text."""
    te = np.asarray(text_end, dtype=np.int64)
    return np.minimum((te * world) // max(int(n_text), 1), world - 1)


def to_records(hits, counts):
    """ae_search results (grouped by query) -> int64 records (query, text end,
    query end, score)."""
    q = np.repeat(np.arange(len(counts), dtype=np.int64), np.asarray(counts, dtype=np.int64))
    rec = np.empty((hits.size, RECORD_FIELDS), dtype=np.int64)
    rec[:, 0] = q
    rec[:, 1] = hits["text_end"]
    rec[:, 2] = hits["query_end"]
    rec[:, 3] = hits["score"]
    return rec


def exchange(records, n_text, dist, group=None):
    """Send every record to the rank that owns its text end; return the
    records this rank owns (from every rank, itself included)."""
    import torch
    world = dist.get_world_size(group)
    own = owner_of(records[:, 1], n_text, world) if records.size else np.zeros(0, np.int64)
    order = np.argsort(own, kind="stable")
    send = np.ascontiguousarray(records[order]) if records.size else np.zeros((0, RECORD_FIELDS), np.int64)
    counts = np.bincount(own, minlength=world).astype(np.int64)
    r_counts = torch.empty(world, dtype=torch.int64)
    dist.all_to_all_single(r_counts, torch.from_numpy(counts), group=group)
    recv = torch.empty((int(r_counts.sum()), RECORD_FIELDS), dtype=torch.int64)
    dist.all_to_all_single(recv, torch.from_numpy(send), output_split_sizes=r_counts.tolist(),
                           input_split_sizes=counts.tolist(), group=group)
    return recv.numpy()


def merge_on_device(records, nq, n_text, max_query_len, device="cuda"):
    """Per-cell maximum of records with the library's kernels (ae_hits_merge).
    Returns (hits grouped by query and sorted like ae_search, counts)."""
    import torch
    n = records.shape[0]
    if n == 0:
        return np.zeros(0, dtype=ae.HIT_DTYPE), np.zeros(nq, dtype=np.int64)
    h = np.zeros(n, dtype=ae.HIT_DTYPE)
    h["text_end"], h["query_end"], h["score"] = records[:, 1], records[:, 2], records[:, 3]
    d_in = torch.from_numpy(h.view(np.uint8)).to(device)
    d_q = torch.from_numpy(np.ascontiguousarray(records[:, 0].astype(np.int32))).to(device)
    d_out = torch.empty(n * 16, dtype=torch.uint8, device=device)
    counts, total = ae.ae_hits_merge(d_in.data_ptr(), d_q.data_ptr(), n, nq, n_text, max_query_len,
                                     d_out.data_ptr())
    return d_out[: total * 16].cpu().numpy().view(ae.HIT_DTYPE).copy(), counts


def gather_parts(hits, counts, dist, group=None):
    """Rank 0: the owners' parts in rank order, regrouped by query (each part
    is sorted and the parts cover increasing text ranges, so the result keeps
    the (text end, query end) order).  Other ranks: None."""
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    parts = [None] * world if rank == 0 else None
    dist.gather_object((hits, counts), parts, dst=0, group=group)
    if rank != 0:
        return None
    nq = len(counts)
    per_query = [[] for _ in range(nq)]
    for h, c in parts:
        starts = np.concatenate([[0], np.cumsum(c)])
        for q in range(nq):
            per_query[q].append(h[starts[q]:starts[q + 1]])
    out = [np.concatenate(p) if p else np.zeros(0, dtype=ae.HIT_DTYPE) for p in per_query]
    return np.concatenate(out) if out else np.zeros(0, dtype=ae.HIT_DTYPE), np.array([x.size for x in out],
                                                                                     dtype=np.int64)


def split_search(index, queries, scheme, H, dist, group=None, options=None, search=None, merge=None,
                 n_text=None, max_query_len=None):
    """The search of `queries` split over the ranks of `dist`: this rank
    searches its part of the forks, the results are exchanged and merged, and
    rank 0 returns (hits, counts) of the whole search (others: None).

    search(part, parts) -> (hits, counts) and merge(records, nq) -> (hits,
    counts) default to the library (ae_search with fork_parts/fork_part, and
    ae_hits_merge); tests may pass other implementations of the same
    contracts.  Raises SplitError if any rank fails or leaves."""
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    nq = len(queries)
    if n_text is None:
        n_text = ae.ae_index_info(index)["n"]
    if max_query_len is None:
        max_query_len = max([len(q) for q in queries] + [1])
    if search is None:
        def search(part, parts):
            kw = {}
            if options:
                kw.update(options)
            kw.update(fork_parts=parts, fork_part=part)
            return ae.ae_search(index, queries, scheme, H, options=ae.make_options(**kw))
    if merge is None:
        def merge(records, nq_):
            return merge_on_device(records, nq_, n_text, max_query_len)
    try:
        hits, counts = search(rank, world)
        mine = exchange(to_records(hits, counts), n_text, dist, group)
        mh, mc = merge(mine, nq)
        return gather_parts(mh, mc, dist, group)
    except SplitError:
        raise
    except Exception as e:   # a peer that failed or left: no partial results
        raise SplitError(f"rank {rank}: split search failed: {e}") from e
