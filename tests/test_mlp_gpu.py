"""The work predictor's kernels against its oracle (oracle/mlp_oracle.py):
features, forward pass, gradients and the Adam step, then training on counts
logged by the engine and the gain of its hit hints over the engine without
them (results identical either way)."""
import numpy as np
import pytest

from oracle import mlp_oracle as mo
from workloads import Scheme, dna_scale_text, dna_scale_query, log_uniform_lengths

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1208_0274_gb300 import ae  # noqa: E402
from paper_1208_0274_gb300.predictor import WorkPredictor  # noqa: E402

SCHEME = Scheme(1, -3, -5, -2)


@pytest.fixture(scope="module")
def small_index():
    text = dna_scale_text(seed=31, n=300_000)
    idx = ae.ae_index_build(text, ae.AE_DNA)
    yield text, idx
    idx.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_features_match_oracle(small_index):
    text, idx = small_index
    rng = np.random.default_rng(1)
    qs = [np.frombuffer(b"A", np.uint8), np.frombuffer(b"AC", np.uint8), np.frombuffer(b"ACG", np.uint8)]
    qs += [dna_scale_query(text, int(m), rng)[0] for m in (50, 777, 5_000)]
    pred = WorkPredictor(idx, SCHEME)
    got = pred.features(qs)
    want = mo.features(text, qs)
    assert got.shape == (len(qs), 66)
    assert np.allclose(got[:, :65], want[:, :65], rtol=1e-6, atol=1e-7)
    assert np.allclose(got[:, 65], want[:, 65], rtol=1e-5, atol=1e-6)
    # a letter outside ACGT is an error
    bad = np.frombuffer(b"ACGN", np.uint8)
    with pytest.raises(RuntimeError):
        pred.features([bad])


def _random_problem(B, seed):
    rng = np.random.default_rng(seed)
    p = mo.init_params(seed=seed).astype(np.float32)
    p[mo.n_params() - 2:] = [0.25, -0.5]
    X = rng.normal(size=(B, 66)).astype(np.float32)
    T = rng.normal(size=(B, 2)).astype(np.float32)
    return p, X, T


def _identity_norm(m):
    m.set_norm(np.zeros(66), np.ones(66), np.zeros(2), np.ones(2))


@pytest.mark.parametrize("B", [1, 37, 300, 2053])
def test_forward_and_gradients_match_oracle(B):
    p, X, T = _random_problem(B, seed=B)
    m = ae.Mlp(0)
    _identity_norm(m)
    m.set_params(p)
    dx, dt = _dev(X), _dev(T)
    dy = torch.empty((B, 2), dtype=torch.float32, device="cuda")
    m.forward(dx.data_ptr(), B, dy.data_ptr())
    y_gpu = dy.cpu().numpy()
    y_or, _ = mo.forward(p.astype(np.float64), X, bf16=True)
    assert np.allclose(y_gpu, y_or, rtol=2e-3, atol=2e-3 * np.abs(y_or).max())
    loss, g = m.loss_grad(dx.data_ptr(), dt.data_ptr(), B)
    L_or, g_or = mo.loss_and_grads(p.astype(np.float64), X, T, bf16=True)
    assert abs(loss - L_or) <= 1e-3 * abs(L_or) + 1e-6
    scale = np.abs(g_or).max()
    assert np.abs(g - g_or).max() <= 3e-3 * scale
    assert np.linalg.norm(g - g_or) <= 2e-3 * np.linalg.norm(g_or)
    # and close to the exact-arithmetic gradient (bf16 operands are the only approximation)
    _, g_exact = mo.loss_and_grads(p.astype(np.float64), X, T, bf16=False)
    assert np.linalg.norm(g - g_exact) <= 3e-2 * np.linalg.norm(g_exact)
    m.close()


def test_normalisation_is_applied_inside_the_model():
    B = 64
    p, X, T = _random_problem(B, seed=5)
    rng = np.random.default_rng(6)
    x_mu, x_sd = rng.normal(size=66), rng.uniform(0.5, 2.0, size=66)
    y_mu, y_sd = np.array([3.0, -1.0]), np.array([2.0, 0.5])
    m = ae.Mlp(0)
    m.set_norm(x_mu, x_sd, y_mu, y_sd)
    m.set_params(p)
    Xr = (X * x_sd + x_mu).astype(np.float32)
    dy = torch.empty((B, 2), dtype=torch.float32, device="cuda")
    dxr = _dev(Xr)
    m.forward(dxr.data_ptr(), B, dy.data_ptr())
    Xn = ((Xr.astype(np.float64) - x_mu) / x_sd)
    y_or, _ = mo.forward(p.astype(np.float64), Xn, bf16=True)
    assert np.allclose(dy.cpu().numpy(), y_or * y_sd + y_mu, rtol=5e-3, atol=5e-3 * np.abs(y_or * y_sd).max())
    # the loss is taken against normalised targets
    Tr = (T * y_sd + y_mu).astype(np.float32)
    dtr = _dev(Tr)
    loss, _ = m.loss_grad(dxr.data_ptr(), dtr.data_ptr(), B, want_grads=False)
    L_or, _ = mo.loss_and_grads(p.astype(np.float64), Xn, T, bf16=True)
    assert abs(loss - L_or) <= 5e-3 * abs(L_or)
    m.close()


def test_one_adam_step_matches_oracle():
    B = 128
    p, X, T = _random_problem(B, seed=9)
    m = ae.Mlp(0)
    _identity_norm(m)
    m.set_params(p)
    lr = 1e-2
    wd = 0.3
    dx, dt = _dev(X), _dev(T)  # held: a freed temporary's memory would be handed to the next tensor
    m.train(dx.data_ptr(), dt.data_ptr(), B, epochs=1, batch=B, lr=lr, weight_decay=wd, seed=3)
    p1 = m.get_params()
    _, g_or = mo.loss_and_grads(p.astype(np.float64), X, T, bf16=True)
    z = np.zeros_like(g_or)
    want, _, _ = mo.adam(p.astype(np.float64), g_or, z, z, t=1, lr=lr, wd=wd)
    # the first step moves every parameter by lr * g / (|g| + eps): where |g| is
    # small the sign may differ between bf16 and exact products, so compare the
    # rest exactly and bound the step everywhere
    sure = np.abs(g_or) > 1e-2 * np.abs(g_or).max()
    assert np.allclose(p1[sure], want[sure], atol=1e-3 * lr + 1e-6)
    assert sure.sum() > 0.2 * p.size
    assert np.abs(p1.astype(np.float64) - p).max() <= lr * (1 + wd * np.abs(p).max() + 1e-3)
    m.close()


@pytest.mark.parametrize("B", [1, 31, 64])
def test_small_and_ragged_training_step_matches_oracle(B):
    # mini-batches ragged against the 16-row mma tile and the 16-deep K chunks of the
    # weight gradients (1, 31), and whole tiles (64)
    p, X, T = _random_problem(B, seed=100 + B)
    m = ae.Mlp(0)
    _identity_norm(m)
    m.set_params(p)
    lr, wd = 1e-2, 0.3
    dx, dt = _dev(X), _dev(T)  # held: a freed temporary's memory would be handed to the next tensor
    m.train(dx.data_ptr(), dt.data_ptr(), B, epochs=1, batch=B, lr=lr, weight_decay=wd, seed=3)
    p1 = m.get_params()
    _, g_or = mo.loss_and_grads(p.astype(np.float64), X, T, bf16=True)
    z = np.zeros_like(g_or)
    want, _, _ = mo.adam(p.astype(np.float64), g_or, z, z, t=1, lr=lr, wd=wd)
    # as in the 128-row step: parameters with small gradients are only bounded
    sure = np.abs(g_or) > 1e-2 * np.abs(g_or).max()
    assert np.allclose(p1[sure], want[sure], atol=1e-3 * lr + 1e-6)
    assert sure.sum() > 0.2 * p.size
    assert np.abs(p1.astype(np.float64) - p).max() <= lr * (1 + wd * np.abs(p).max() + 1e-3)
    m.close()


def test_training_over_epochs_reduces_the_loss_and_keeps_the_step_count():
    rng = np.random.default_rng(12)
    n = 1000
    X = rng.normal(size=(n, 66)).astype(np.float32)
    w = rng.normal(size=(66, 2))
    T = (np.tanh(X @ w / 8.0) * 3.0 + 1.0).astype(np.float32)
    m = ae.Mlp(2)
    _identity_norm(m)
    dx, dt = _dev(X), _dev(T)
    l0, _ = m.loss_grad(dx.data_ptr(), dt.data_ptr(), n, want_grads=False)
    l1 = m.train(dx.data_ptr(), dt.data_ptr(), n, epochs=20, batch=32, lr=3e-3, seed=1)
    l2, _ = m.loss_grad(dx.data_ptr(), dt.data_ptr(), n, want_grads=False)
    assert l2 < 0.1 * l0 and l1 < 0.2 * l0
    # Adam's step count carries over between calls: with one mini-batch per epoch
    # (whose gradient no row order changes beyond rounding), two calls of one epoch
    # equal one call of two; a restarted count would take a first step twice
    a, b = ae.Mlp(2), ae.Mlp(2)
    for mm in (a, b):
        _identity_norm(mm)
    dxs, dts = _dev(X[:32]), _dev(T[:32])
    a.train(dxs.data_ptr(), dts.data_ptr(), 32, epochs=2, batch=32, lr=3e-3, seed=1)
    for _ in range(2):
        b.train(dxs.data_ptr(), dts.data_ptr(), 32, epochs=1, batch=32, lr=3e-3, seed=1)
    assert np.allclose(a.get_params(), b.get_params(), rtol=1e-4, atol=1e-6)
    for mm in (m, a, b):
        mm.close()


def test_training_reduces_the_loss_on_a_learnable_target():
    rng = np.random.default_rng(11)
    n = 2048
    X = rng.normal(size=(n, 66)).astype(np.float32)
    w = rng.normal(size=(66, 2))
    T = (np.tanh(X @ w / 8.0) * 3.0 + 1.0).astype(np.float32)
    m = ae.Mlp(1)
    _identity_norm(m)
    dx, dt = _dev(X), _dev(T)
    l0, _ = m.loss_grad(dx.data_ptr(), dt.data_ptr(), n, want_grads=False)
    l1 = m.train(dx.data_ptr(), dt.data_ptr(), n, epochs=60, batch=128, lr=3e-3, seed=1)
    l2, _ = m.loss_grad(dx.data_ptr(), dt.data_ptr(), n, want_grads=False)
    assert l2 < 0.05 * l0 and l1 < 0.1 * l0
    m.close()


@pytest.fixture(scope="module")
def logged():
    """Queries searched alone by the engine against a 4 Mbp text; their
    entries and sweep hit records are the training targets."""
    text = dna_scale_text(seed=41, n=4_000_000)
    idx = ae.ae_index_build(text, ae.AE_DNA)
    rng = np.random.default_rng(42)
    k = 320
    lens = log_uniform_lengths(k, 100, 20_000, rng)
    fracs = rng.choice([0.0, 0.01, 0.05, 0.2], size=k)
    qs = [dna_scale_query(text, int(m), rng, frac=float(f))[0] for m, f in zip(lens, fracs)]
    Hs = [18] * k
    pred = WorkPredictor(idx, SCHEME, seed=3)
    T = pred.log_searches(qs, Hs)
    X = pred.features(qs)
    yield text, idx, pred, qs, Hs, X, T
    idx.close()


def test_trained_predictor_estimates_search_work(logged):
    text, idx, pred, qs, Hs, X, T = logged
    tr, te = np.arange(0, 240), np.arange(240, 320)
    pred.fit(X[tr], T[tr], seed=7)
    P = pred.predict_features(X[te])
    err_e = np.abs(P[:, 0] - T[te, 0])
    # entries within ~15% for the median held-out query
    assert np.median(err_e) < 0.15, np.median(err_e)
    # better than predicting the training mean
    base = np.abs(T[tr, 0].mean() - T[te, 0])
    assert err_e.mean() < 0.5 * base.mean()
    # hit records: rank correlation with the truth
    from scipy.stats import spearmanr
    rho = spearmanr(P[:, 1], T[te, 1]).correlation
    assert rho > 0.5, rho
    print(f"median |log err| entries {np.median(err_e):.3f}, hits rho {rho:.3f}")


def test_hit_hints_avoid_sweep_reruns_and_change_no_result(logged):
    text, idx, pred, qs, Hs, X, T = logged
    if not pred.trained:
        pred.fit(X[:240], T[:240], seed=7)
    # a batch whose sweep writes more hit records than the engine's default
    # first-search buffer holds: the queries with the most hit records
    order = np.argsort(-T[:, 1])
    batch, tot = [], 0.0
    for k in order:
        batch.append(int(k))
        tot += np.expm1(T[k, 1])
        if tot > 3.0e6:
            break
    bq = [qs[k] for k in batch]
    bh = [Hs[k] for k in batch]
    st = torch.cuda.Stream()
    ae.ae_workspace_release(idx, st)
    h0, c0 = ae.ae_search(idx, bq, SCHEME, bh, stream=st)
    s0 = ae.ae_last_stats()
    ae.ae_workspace_release(idx, st)
    hints = pred.hint_hits(bq)
    h1, c1 = ae.ae_search(idx, bq, SCHEME, bh, options=ae.make_options(hint_hits=hints), stream=st)
    s1 = ae.ae_last_stats()
    ae.ae_workspace_release(idx, st)
    assert np.array_equal(c0, c1) and np.array_equal(h0, h1)
    assert s0["leaf_raw_hits"] > (1 << 20), "the batch does not overflow the default buffer"
    assert s0["leaf_sweeps"] > s1["leaf_sweeps"], (s0["leaf_sweeps"], s1["leaf_sweeps"])
    print(f"sweeps without hints {s0['leaf_sweeps']} ({s0['ms_total']:.1f} ms), with {s1['leaf_sweeps']} "
          f"({s1['ms_total']:.1f} ms); hinted {int(hints.sum()):,} vs written {s1['leaf_raw_hits']:,}")
