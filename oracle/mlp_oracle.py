"""CPU oracle of the work predictor — TEST INFRASTRUCTURE ONLY.

Only ``tests/`` may import this module; the GPU predictor (ae_mlp_*) neither
imports nor links it.

The predictor is not part of the paper's method: it estimates, for a DNA
query, the work of its search (log1p of the DP entries computed, log1p of the
raw hits written by the text-position sweep) so that buffers and batches can
be sized before the search. It never changes a result. What it computes is
written out here from the definitions:

* ``features`` — 66 numbers per query: the 3-mer spectrum (64 relative
  frequencies over the m-2 windows, index 16*a + 4*b + c for letters a b c
  in ACGT order), log1p(m), and the mean over the query's windows of K
  letters, K = ceil(log4(n+1)) + 4, of log1p(size of the suffix-array
  interval of the window), the interval size being the number of
  occurrences of the window in the text (Section 2.3: the range of a string
  in the suffix array holds one row per occurrence). Counted here directly
  on the text, without an index.
* ``forward`` / ``loss_and_grads`` — the 66-128-128-2 perceptron
  y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 with the loss
  L = sum((y - t)^2) / (2 B) over a batch of B, and its exact gradients by the
  chain rule, in fp64. ``bf16=True`` first rounds every matrix-product operand
  (inputs, weights, activations, upstream gradients) to bfloat16 with
  round-to-nearest-even, the precision the GPU kernels multiply in; products
  are then summed in fp64.
* ``adam`` — one Adam step (Kingma and Ba, 2015, Algorithm 1) with decoupled
  weight decay (Loshchilov and Hutter, 2019).

Pins (tests/test_mlp_oracle.py): central finite differences of the loss
against ``loss_and_grads``; features on hand-counted strings; the
interval-size feature against a brute-force substring count; bf16 rounding on
hand-picked bit patterns; Adam's first step equals lr * sign(g), and weight
decay alone shrinks a parameter by the factor (1 - lr * wd).
"""
from __future__ import annotations

import numpy as np

DNA = b"ACGT"
SIZES = (66, 128, 128, 2)


def param_shapes():
    """(name, shape) in the packed parameter order W1, b1, W2, b2, W3, b3."""
    d0, d1, d2, d3 = SIZES
    return [("W1", (d1, d0)), ("b1", (d1,)), ("W2", (d2, d1)), ("b2", (d2,)), ("W3", (d3, d2)), ("b3", (d3,))]


def n_params():
    return sum(int(np.prod(s)) for _, s in param_shapes())


def unpack(flat):
    out, k = {}, 0
    for name, shape in param_shapes():
        size = int(np.prod(shape))
        out[name] = np.asarray(flat[k:k + size], dtype=np.float64).reshape(shape)
        k += size
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in param_shapes()])


def bf16_round(x):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as
    float64. bfloat16 keeps the top 16 bits of the float32 pattern."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(a)
    if nan.any():
        out[nan] = np.nan
    return out


def _q(x, bf16):
    return bf16_round(x) if bf16 else np.asarray(x, dtype=np.float64)


def forward(params, X, bf16=False):
    """Returns (y, cache) for inputs X (B x 66)."""
    p = unpack(params) if not isinstance(params, dict) else params
    X = np.asarray(X, dtype=np.float64)
    Z1 = _q(X, bf16) @ _q(p["W1"], bf16).T + p["b1"]
    A1 = np.maximum(Z1, 0.0)
    Z2 = _q(A1, bf16) @ _q(p["W2"], bf16).T + p["b2"]
    A2 = np.maximum(Z2, 0.0)
    Y = _q(A2, bf16) @ _q(p["W3"], bf16).T + p["b3"]
    return Y, (X, Z1, A1, Z2, A2)


def loss_and_grads(params, X, T, bf16=False):
    """L = sum((y - t)^2) / (2B) and dL/dparams (packed like params)."""
    p = unpack(params) if not isinstance(params, dict) else params
    Y, (X, Z1, A1, Z2, A2) = forward(p, X, bf16)
    B = X.shape[0]
    R = Y - np.asarray(T, dtype=np.float64)
    L = float((R * R).sum() / (2.0 * B))
    dY = R / B
    g = {}
    g["W3"] = _q(dY, bf16).T @ _q(A2, bf16)
    g["b3"] = dY.sum(axis=0)
    dA2 = _q(dY, bf16) @ _q(p["W3"], bf16)
    dZ2 = dA2 * (Z2 > 0)
    g["W2"] = _q(dZ2, bf16).T @ _q(A1, bf16)
    g["b2"] = dZ2.sum(axis=0)
    dA1 = _q(dZ2, bf16) @ _q(p["W2"], bf16)
    dZ1 = dA1 * (Z1 > 0)
    g["W1"] = _q(dZ1, bf16).T @ _q(X, bf16)
    g["b1"] = dZ1.sum(axis=0)
    return L, pack(g)


def adam(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """One Adam step at step number t >= 1 with decoupled weight decay wd;
    returns new (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grads
    v = beta2 * v + (1.0 - beta2) * grads * grads
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return params - lr * (mh / (np.sqrt(vh) + eps) + wd * params), m, v


def kmer3_counts(codes):
    """Occurrences of each of the 64 3-mers in a code string (0..3)."""
    c = np.asarray(codes, dtype=np.int64)
    out = np.zeros(64, dtype=np.int64)
    if c.size >= 3:
        w = 16 * c[:-2] + 4 * c[1:-1] + c[2:]
        out += np.bincount(w, minlength=64)
    return out


def encode(seq):
    lut = np.full(256, 255, dtype=np.uint8)
    for k, ch in enumerate(DNA):
        lut[ch] = k
        lut[ord(chr(ch).lower())] = k
    c = lut[np.frombuffer(bytes(seq), dtype=np.uint8) if not isinstance(seq, np.ndarray) else seq]
    if (c == 255).any():
        raise ValueError("not a DNA letter")
    return c


def interval_window(n):
    """Window length K = ceil(log4(n + 1)) + 4 (at most 32)."""
    k = 0
    while 4 ** k < n + 1:
        k += 1
    return min(k + 4, 32)


def _window_codes(c, K):
    c = np.asarray(c, dtype=np.int64)
    if c.size < K:
        return np.zeros(0, dtype=np.int64)
    v = np.zeros(c.size - K + 1, dtype=np.int64)
    for i in range(K):
        v = v * 4 + c[i:c.size - K + 1 + i]
    return v


def features(text, queries):
    """66 features per query (rows), from the definitions above."""
    t = encode(text)
    K = interval_window(t.size)
    words, occ = np.unique(_window_codes(t, K), return_counts=True)
    F = np.zeros((len(queries), 66), dtype=np.float64)
    for r, q in enumerate(queries):
        c = encode(q)
        cnt = kmer3_counts(c)
        w = max(c.size - 2, 0)
        if w > 0:
            F[r, :64] = cnt / w
        F[r, 64] = np.log1p(c.size)
        qw = _window_codes(c, K)
        if qw.size:
            pos = np.searchsorted(words, qw)
            pos = np.minimum(pos, max(words.size - 1, 0))
            found = (words.size > 0) & (words[pos] == qw) if words.size else np.zeros(qw.size, bool)
            F[r, 65] = float(np.log1p(np.where(found, occ[pos], 0)).mean())
    return F


def init_params(seed=0):
    """He-uniform weights, zero biases (a deterministic starting point)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in param_shapes():
        if name.startswith("W"):
            bound = np.sqrt(6.0 / shape[1])
            p[name] = rng.uniform(-bound, bound, size=shape)
        else:
            p[name] = np.zeros(shape)
    return pack(p)
