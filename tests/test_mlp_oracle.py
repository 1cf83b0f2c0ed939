"""Pins of the work-predictor oracle (oracle/mlp_oracle.py) against facts that
do not come from the oracle itself: finite differences of the loss, hand
counts of 3-mers, a brute-force substring count, bfloat16 bit patterns, and
the closed form of Adam's first step."""
import numpy as np

from oracle import mlp_oracle as mo


def test_gradients_match_central_finite_differences():
    rng = np.random.default_rng(0)
    p = mo.init_params(seed=1) * 0.5
    # keep ReLUs away from their kink so the loss is smooth within +-h
    p[-2:] = [0.3, -0.2]
    X = rng.normal(size=(7, 66))
    T = rng.normal(size=(7, 2))
    L, g = mo.loss_and_grads(p, X, T)
    h = 1e-6
    idx = np.concatenate([rng.choice(p.size, 60, replace=False),
                          np.arange(p.size - 260, p.size)])          # includes all of W3, b3
    for k in idx:
        e = np.zeros_like(p)
        e[k] = h
        fd = (mo.loss_and_grads(p + e, X, T)[0] - mo.loss_and_grads(p - e, X, T)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 + 1e-5 * abs(fd), (k, fd, g[k])
    assert L > 0


def test_loss_is_half_mean_squared_error_and_zero_at_the_target():
    p = mo.init_params(seed=2)
    X = np.random.default_rng(3).normal(size=(5, 66))
    Y, _ = mo.forward(p, X)
    L, g = mo.loss_and_grads(p, X, Y)
    assert L == 0.0 and np.all(g == 0.0)
    L2, _ = mo.loss_and_grads(p, X, Y + 2.0)        # every residual is -2
    assert abs(L2 - (5 * 2 * 4.0) / (2 * 5)) < 1e-12


def test_bias_only_network_is_linear_regression_of_the_mean():
    # with all weights zero the output is b3, and dL/db3 = mean(b3 - t)
    P = mo.unpack(np.zeros(mo.n_params()))
    P["b3"] = np.array([1.0, -1.0])
    T = np.array([[3.0, 0.0], [5.0, 2.0]])
    L, g = mo.loss_and_grads(mo.pack(P), np.ones((2, 66)), T)
    G = mo.unpack(g)
    assert np.allclose(G["b3"], [1.0 - 4.0, -1.0 - 1.0])
    assert np.all(G["W1"] == 0) and np.all(G["W2"] == 0) and np.all(G["W3"] == 0)


def test_bf16_rounding_on_bit_patterns():
    f = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 1.0 + 3 * 2 ** -8, -2.5, 0.0, 3.0e38], dtype=np.float32)
    r = mo.bf16_round(f)
    # bfloat16 keeps 7 fraction bits (ulp 2^-7 at 1): 1 + 2^-8 is a tie -> even (1.0);
    # 1 + 1.5 * 2^-8 is above the tie -> 1 + 2^-7; 1 + 2^-7 + 2^-8 is a tie between an
    # odd (1 + 2^-7) and an even (1 + 2^-6) neighbour -> 1 + 2^-6
    assert list(r[:4]) == [1.0, 1.0, 1.0 + 2 ** -7, 1.0 + 2 ** -6]
    assert r[4] == -2.5 and r[5] == 0.0
    assert abs(r[6] - 3.0e38) / 3.0e38 < 2 ** -8
    x = np.random.default_rng(4).normal(size=10_000).astype(np.float32)
    rel = np.abs(mo.bf16_round(x) - x) / np.abs(x)
    assert rel.max() <= 2 ** -8 + 1e-12


def test_features_on_hand_counted_strings():
    # text of 8 letters: K = ceil(log4 9) + 4 = 6
    text = b"ACGTACGT"
    assert mo.interval_window(8) == 6
    F = mo.features(text, [b"AAAA", b"ACG", b"AC", b"ACGTAC", b"CGTACGT"])
    # AAAA: windows AAA, AAA -> spectrum[0] = 1
    assert F[0, 0] == 1.0 and F[0, 1:64].sum() == 0.0
    # ACG is 3-mer index 16*0 + 4*1 + 2 = 6
    assert F[1, 6] == 1.0 and F[1, :64].sum() == 1.0
    # AC has no 3-mer
    assert F[2, :64].sum() == 0.0
    # ACGTAC: ACG, CGT, GTA, TAC -> indices 6, 27, 44, 49, a quarter each
    assert set(np.nonzero(F[3, :64])[0]) == {6, 27, 44, 49} and np.allclose(F[3, [6, 27, 44, 49]], 0.25)
    assert np.allclose(F[:, 64], np.log1p([4, 3, 2, 6, 7]))
    # windows of 6: shorter queries have none; ACGTAC occurs once in the text;
    # CGTACGT has windows CGTACG (once) and GTACGT (once)
    assert list(F[:3, 65]) == [0.0, 0.0, 0.0]
    assert np.isclose(F[3, 65], np.log1p(1)) and np.isclose(F[4, 65], np.log1p(1))
    F2 = mo.features(b"ACGTACGTAAAAAAAAAA", [b"AAAAAAA", b"CCCCCCCC"])   # n = 18: K = 7
    # AAAAAAA occurs at 4 positions of the run of ten A; CCCCCCC nowhere
    assert np.isclose(F2[0, 65], np.log1p(4)) and F2[1, 65] == 0.0


def test_interval_feature_against_brute_force_substring_count():
    rng = np.random.default_rng(5)
    letters = np.frombuffer(b"ACGT", dtype=np.uint8)
    text = rng.choice(letters, size=3000).tobytes()
    q = bytes(text[1000:1030]) + rng.choice(letters, size=20).tobytes()
    K = mo.interval_window(len(text))
    assert K == 10
    F = mo.features(text, [q])
    want = 0.0
    for k in range(len(q) - K + 1):
        w = q[k:k + K]
        occ = sum(1 for s in range(len(text) - K + 1) if text[s:s + K] == w)
        want += np.log1p(occ) / (len(q) - K + 1)
    assert np.isclose(F[0, 65], want) and want > 0


def test_adam_first_step_moves_each_parameter_by_lr_times_the_gradient_sign():
    p = np.array([0.5, -1.0, 2.0, 0.0])
    g = np.array([3.0, -0.01, 1e-3, -7.0])
    z = np.zeros(4)
    p1, m, v = mo.adam(p, g, z, z, t=1, lr=0.01, eps=0.0)
    assert np.allclose(p1, p - 0.01 * np.sign(g))
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    # with a zero gradient, decoupled weight decay alone scales the parameter by (1 - lr * wd)
    p2, _, _ = mo.adam(p, z, z, z, t=1, lr=0.01, wd=0.5)
    assert np.allclose(p2, p * (1 - 0.005))
