"""Autotuner for the batched search: picks the engine's chunk shapes and the
number of concurrent streams for a workload by timing them on a sample.

Knobs (none changes a result):
  * batch_columns — query letters per engine batch (the frontier chunk: a
    larger chunk amortises per-level launches and host synchronisation over
    more nodes, a smaller one keeps the level arenas small);
  * leaf_delay — levels a single-occurrence trie node keeps expanding in the
    trie walk before its row moves to the text-position sweep (trades trie
    rows, processed in wide level-synchronous launches, against sweep tasks);
  * nstreams — concurrent groups in search_many.

The search is coordinate descent: starting from the defaults, each knob in
turn is set to its fastest value with the others held, over `rounds` passes.
A configuration's time is the minimum of `repeats` runs of the sample; one
that runs out of device memory costs infinity.
Results are cached in a JSON file keyed by the device, the text, the scheme
and the sample's size class, so a later call with the same key returns the
cached choice without timing anything.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

DEFAULT_SPACE = {
    "batch_columns": [1 << 17, 1 << 18, 1 << 19, 1 << 20],
    "leaf_delay": [4, 8, 12],
    "nstreams": [1, 2, 3],
}
DEFAULT_CONFIG = {"batch_columns": 1 << 18, "leaf_delay": 8, "nstreams": 2}
CACHE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune_cache.json")


def workload_key(device, n, alphabet, scheme, lengths):
    """Cache key: device name, text size, alphabet, scheme, and the sample's
    query count and total length rounded to powers of two."""
    lengths = np.asarray(lengths, dtype=np.int64)
    tot = int(lengths.sum()) if lengths.size else 0
    cls = (int(math.log2(max(len(lengths), 1))), int(math.log2(max(tot, 1))))
    sc = (scheme.match, scheme.mismatch, scheme.gap_open, scheme.gap_extend, scheme.matrix is not None)
    return f"{device}|n={n}|a={alphabet}|s={sc}|q={cls[0]}|m={cls[1]}"


def load_cache(path=CACHE_PATH):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache, path=CACHE_PATH):
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def coordinate_descent(time_fn, space=None, start=None, rounds=2, repeats=2):
    """Minimise time_fn(config) over the product space by coordinate descent.
    Returns (best config, best time, list of (config, time) evaluated)."""
    space = space or DEFAULT_SPACE
    best = dict(start or DEFAULT_CONFIG)
    seen = {}
    trail = []

    def cost(cfg):
        key = tuple(sorted(cfg.items()))
        if key not in seen:
            seen[key] = min(time_fn(dict(cfg)) for _ in range(repeats))
            trail.append((dict(cfg), seen[key]))
        return seen[key]

    best_t = cost(best)
    for _ in range(rounds):
        changed = False
        for knob, values in space.items():
            for v in values:
                cand = dict(best)
                cand[knob] = v
                t = cost(cand)
                if t < best_t:
                    best, best_t, changed = cand, t, True
        if not changed:
            break
    return best, best_t, trail


def tune(index, queries, Hs, scheme, sample=512, space=None, cache_path=CACHE_PATH, device_name=None,
         time_fn=None, seed=0, rounds=2, repeats=2):
    """The tuned configuration (dict with batch_columns, leaf_delay, nstreams)
    for searching `queries` against `index`; times a random sample of
    `sample` queries unless the cache holds the answer."""
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name()
    rng = np.random.default_rng(seed)
    pick = rng.choice(len(queries), size=min(sample, len(queries)), replace=False)
    sq = [queries[k] for k in pick]
    sh = [Hs[k] for k in pick]
    n = getattr(index, "n", None)
    if n is None:
        from . import ae
        n = ae.ae_index_info(index)["n"]
    key = workload_key(device_name, n, index.alphabet, scheme, [len(q) for q in sq])
    cache = load_cache(cache_path)
    if key in cache:
        return dict(cache[key]["config"]), True
    if time_fn is None:
        from .batch import search_many

        def time_fn(cfg):
            import torch
            from . import ae
            opts = {"batch_columns": cfg["batch_columns"], "leaf_delay": cfg["leaf_delay"]}
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                search_many(index, sq, sh, scheme, nstreams=cfg["nstreams"], options=opts)
            except ae.AEError as e:          # a configuration that does not fit is never chosen
                if e.status != ae.AE_ENOMEM:
                    raise
                return float("inf")
            torch.cuda.synchronize()
            return time.perf_counter() - t0

    best, best_t, trail = coordinate_descent(time_fn, space, rounds=rounds, repeats=repeats)
    cache[key] = {"config": best, "seconds": best_t, "evaluated": len(trail)}
    save_cache(cache, cache_path)
    return best, False
