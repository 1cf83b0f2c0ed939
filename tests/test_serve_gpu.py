"""The request loop on the GPU: requests arriving while others run are
admitted into concurrent slots (their own CUDA streams and workspaces), and
every request's results are identical to those of the same query searched
alone, and to the oracle's for a sample."""
import numpy as np
import pytest

import oracle
from workloads import Scheme, dna_scale_text, dna_scale_query, log_uniform_lengths

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1208_0274_gb300 import ae, serve  # noqa: E402

SCHEME = Scheme(1, -3, -5, -2)


@pytest.fixture(scope="module")
def setup():
    text = dna_scale_text(n=2_000_000)
    rng = np.random.default_rng(11)
    k = 64
    lens = log_uniform_lengths(k, 200, 8_000, rng)
    qs = [dna_scale_query(text, int(m), rng, frac=0.05)[0] for m in lens]
    Hs = [22 if m < 2000 else 24 for m in lens]
    idx = ae.ae_index_build(text, ae.AE_DNA)
    yield text, qs, Hs, idx
    idx.close()


def test_results_are_the_same_alone_and_in_the_mix(setup):
    text, qs, Hs, idx = setup
    k = len(qs)
    srv = serve.Server(idx, SCHEME, nslots=3, max_columns=1 << 16, bytes_per_column=20_000)
    srv.warmup(qs[:8], Hs[:8])
    reqs = serve.poisson_requests(qs, Hs, rate=2_000.0, seed=12)
    rep = srv.run(reqs)
    assert len(rep.requests) == k
    assert rep.peak_concurrency >= 2, "no two searches overlapped"
    assert rep.mean_batch > 1.0, "no request joined a batch in flight"
    total = 0
    for r in rep.requests:
        alone, counts = ae.ae_search(idx, [r.query], SCHEME, [r.H])
        assert counts[0] == r.hits.size and np.array_equal(alone, r.hits), f"request {r.rid}"
        total += alone.size
    assert total > 0
    # two short requests against the oracle
    oracle.build()
    short = sorted(rep.requests, key=lambda r: r.query.size)[:2]
    for r in short:
        oi, oj, os_ = oracle.sw_hits(text, r.query, SCHEME, r.H)
        want = np.zeros(oi.size, dtype=ae.HIT_DTYPE)
        want["text_end"], want["query_end"], want["score"] = oi, oj, os_
        assert np.array_equal(r.hits, want)
    for st in srv.streams:
        b, _ = ae.ae_workspace_info(idx, st)
        assert b > 0
        ae.ae_workspace_release(idx, st)
        assert ae.ae_workspace_info(idx, st)[0] == 0


def test_learned_policy_gives_the_same_results(setup):
    from paper_1208_0274_gb300.predictor import WorkPredictor
    text, qs, Hs, idx = setup
    rng = np.random.default_rng(13)
    train = [dna_scale_query(text, int(m), rng, frac=0.05)[0] for m in log_uniform_lengths(48, 200, 8_000, rng)]
    pred = WorkPredictor(idx, SCHEME, seed=1)
    T = pred.log_searches(train, [22] * len(train))
    pred.fit(pred.features(train), T, epochs=200, batch=16)
    srv = serve.Server(idx, SCHEME, nslots=3, max_columns=1 << 16, predictor=pred, work_budget=2e7)
    srv.warmup(qs[:8], Hs[:8])
    rep = srv.run(serve.poisson_requests(qs, Hs, rate=2_000.0, seed=14))
    assert len(rep.requests) == len(qs)
    assert rep.peak_concurrency >= 2
    assert all(r.pred_work > 0 for r in rep.requests)
    for r in rep.requests:
        alone, _ = ae.ae_search(idx, [r.query], SCHEME, [r.H])
        assert np.array_equal(alone, r.hits), f"request {r.rid}"
    for st in srv.streams:
        ae.ae_workspace_release(idx, st)
