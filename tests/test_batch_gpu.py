"""The batched search over concurrent streams (paper_1208_0274_gb300.batch)
and its autotuner on the GPU: every packing gives each query exactly the
results of one ae_search over all queries."""
import numpy as np
import pytest

from workloads import Scheme, dna_scale_text, dna_scale_query, log_uniform_lengths

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1208_0274_gb300 import ae, autotune  # noqa: E402
from paper_1208_0274_gb300.batch import search_many  # noqa: E402
from paper_1208_0274_gb300.predictor import WorkPredictor  # noqa: E402

SCHEME = Scheme(1, -3, -5, -2)


@pytest.fixture(scope="module")
def problem():
    text = dna_scale_text(seed=51, n=2_000_000)
    rng = np.random.default_rng(52)
    lens = log_uniform_lengths(200, 100, 5_000, rng)
    qs = [dna_scale_query(text, int(m), rng, frac=0.05)[0] for m in lens]
    Hs = [20] * len(qs)
    idx = ae.ae_index_build(text, ae.AE_DNA)
    hits, counts = ae.ae_search(idx, qs, SCHEME, Hs)
    starts = np.concatenate([[0], np.cumsum(counts)])
    want = [hits[starts[k]:starts[k + 1]] for k in range(len(qs))]
    yield text, qs, Hs, idx, want
    idx.close()


def test_round_robin_and_lpt_packings_give_the_same_results(problem):
    text, qs, Hs, idx, want = problem
    out, info = search_many(idx, qs, Hs, SCHEME, nstreams=3, policy="round_robin",
                            options={"batch_columns": 50_000})
    assert info["groups"] == [67, 67, 66]
    assert all(np.array_equal(a, b) for a, b in zip(out, want))
    rng = np.random.default_rng(53)
    train = [dna_scale_query(text, int(m), rng, frac=0.05)[0] for m in log_uniform_lengths(64, 100, 5_000, rng)]
    pred = WorkPredictor(idx, SCHEME, seed=2)
    T = pred.log_searches(train, [20] * len(train))
    pred.fit(pred.features(train), T, epochs=100)
    out2, info2 = search_many(idx, qs, Hs, SCHEME, nstreams=2, policy="lpt", predictor=pred,
                              options={"batch_columns": 100_000, "leaf_delay": 4})
    assert sum(info2["groups"]) == len(qs)
    assert all(np.array_equal(a, b) for a, b in zip(out2, want))
    assert sum(h.size for h in want) > 0


def test_autotuner_picks_from_its_space_and_caches(problem, tmp_path):
    text, qs, Hs, idx, want = problem
    space = {"batch_columns": [1 << 16, 1 << 18], "leaf_delay": [4, 8], "nstreams": [1, 2]}
    path = str(tmp_path / "tune.json")
    cfg, cached = autotune.tune(idx, qs, Hs, SCHEME, sample=64, space=space, cache_path=path, rounds=1, repeats=1)
    assert not cached
    for k, v in cfg.items():
        assert v in space[k] or v == autotune.DEFAULT_CONFIG[k]
    cfg2, cached2 = autotune.tune(idx, qs, Hs, SCHEME, sample=64, space=space, cache_path=path)
    assert cached2 and cfg2 == cfg
    out, _ = search_many(idx, qs, Hs, SCHEME, nstreams=cfg["nstreams"],
                         options={"batch_columns": cfg["batch_columns"], "leaf_delay": cfg["leaf_delay"]})
    assert all(np.array_equal(a, b) for a, b in zip(out, want))
