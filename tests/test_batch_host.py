"""Host logic of the batched search: packing queries onto streams (static
round-robin and predicted longest-processing-time first) and the autotuner's
coordinate descent and cache, with fake timings."""
import numpy as np

from paper_1208_0274_gb300 import autotune, batch
from workloads import Scheme


def test_round_robin_covers_every_query_once():
    g = batch.pack_round_robin(10, 3)
    assert g == [[0, 3, 6, 9], [1, 4, 7], [2, 5, 8]]


def test_lpt_balances_predicted_work_within_the_classic_bound():
    rng = np.random.default_rng(0)
    work = np.exp(rng.uniform(np.log(100), np.log(20_000), size=4096))
    for s in (2, 3, 8):
        bins = batch.pack_lpt(work, s)
        assert sorted(k for b in bins for k in b) == list(range(work.size))
        loads = np.array([work[b].sum() for b in bins])
        # Graham's bound: LPT makespan <= (4/3 - 1/(3s)) OPT, and OPT >= max(mean load, max item)
        opt_lb = max(work.sum() / s, work.max())
        assert loads.max() <= (4 / 3 - 1 / (3 * s)) * opt_lb + 1e-9
        rr = np.array([work[g].sum() for g in batch.pack_round_robin(work.size, s)])
        assert loads.max() <= rr.max() + 1e-9
    # a tiny case by hand: 7, 5, 4, 3, 3 on two streams -> {7, 3, ...}
    bins = batch.pack_lpt([3, 7, 4, 5, 3], 2)
    loads = sorted(sum([3, 7, 4, 5, 3][k] for k in b) for b in bins)
    assert loads == [10, 12] and all(b == sorted(b) for b in bins)


def test_coordinate_descent_finds_the_minimum_of_a_separable_cost():
    target = {"batch_columns": 1 << 19, "leaf_delay": 12, "nstreams": 3}

    def cost(cfg):
        return sum(abs(np.log2(cfg[k]) - np.log2(target[k])) for k in target) + 1.0

    best, t, trail = autotune.coordinate_descent(cost, rounds=3, repeats=1)
    assert best == target and t == 1.0
    assert len(trail) <= 1 + 2 * sum(len(v) for v in autotune.DEFAULT_SPACE.values())


def test_tune_uses_and_fills_the_cache(tmp_path):
    class FakeIndex:
        alphabet = 0
        n = 1_000_000

    calls = []

    def time_fn(cfg):
        calls.append(cfg)
        return 1.0 / cfg["nstreams"] + cfg["batch_columns"] * 1e-9

    qs = [np.zeros(1000, np.uint8)] * 100
    path = str(tmp_path / "cache.json")
    best, cached = autotune.tune(FakeIndex(), qs, [20] * 100, Scheme(), sample=50, cache_path=path,
                                 device_name="dev", time_fn=time_fn)
    assert not cached and best["nstreams"] == 3
    assert best["batch_columns"] == min(autotune.DEFAULT_SPACE["batch_columns"])
    n_calls = len(calls)
    best2, cached2 = autotune.tune(FakeIndex(), qs, [20] * 100, Scheme(), sample=50, cache_path=path,
                                   device_name="dev", time_fn=time_fn)
    assert cached2 and best2 == best and len(calls) == n_calls
    # another device or text size is another key
    _, cached3 = autotune.tune(FakeIndex(), qs, [20] * 100, Scheme(), sample=50, cache_path=path,
                               device_name="other", time_fn=time_fn)
    assert not cached3
