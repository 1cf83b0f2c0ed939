"""Learned work predictor for DNA searches (the ae_mlp_* entry points).

For a query it estimates log1p(DP entries) and log1p(sweep hit records) of
its search from 66 features (3-mer spectrum, length, mean FM-interval size of
its windows; see include/ae_mlp.h).  The network runs in libae's kernels: the
features, the forward pass, the backward pass and Adam.  This module computes
on the host only the training set's normalisation (per-feature mean and spread
handed to ae_mlp_set_norm) and the hit-hint margin (a quantile of held-out
residuals), and moves arrays.

Uses (none changes a result):
  * hint_hits(queries): per-query expected sweep hit records for
    ae_options.hint_hits, which sizes each batch's hit buffer;
  * work(queries) / device_bytes(queries): expected work and working memory,
    used by the request loop to order requests and to admit them.
Training data are logged by the plain engine: each query is searched alone
and the counters of ae_last_stats (entries, leaf_raw_hits) are its targets.
"""
from __future__ import annotations

import numpy as np

from . import ae


def _torch():
    import torch
    return torch


class _on:
    """Run torch copies and libae calls on one stream (torch's current stream
    when none is given), so that they are ordered."""

    def __init__(self, stream):
        torch = _torch()
        self.s = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = torch.cuda.stream(self.s)

    def __enter__(self):
        self.ctx.__enter__()
        return self.s

    def __exit__(self, *a):
        return self.ctx.__exit__(*a)


class WorkPredictor:
    def __init__(self, index, scheme, seed=0, device="cuda"):
        if index.alphabet != ae.AE_DNA:
            raise ValueError("the work predictor handles DNA indexes")
        self.index = index
        self.scheme = scheme
        self.device = device
        self.mlp = ae.Mlp(seed)
        self.trained = False
        self.hit_margin = 1.0        # multiplicative margin on hit hints (from held-in residuals)
        self.bytes_per_entry = 16.0  # device bytes per predicted entry (calibrated in log_searches)
        self.fixed_bytes = 0.0       # device bytes of the smallest search (calibrated in log_searches)

    # -- features -------------------------------------------------------------------------------
    def features_device(self, queries, stream=None):
        """(torch float32 tensor nq x 66 on the device) features of host queries."""
        torch = _torch()
        qs = [ae._u8(q) for q in queries]
        off = np.concatenate([[0], np.cumsum([q.size for q in qs])]).astype(np.int64)
        seq = np.concatenate(qs) if qs else np.zeros(0, np.uint8)
        with _on(stream) as st:
            d_seq = torch.from_numpy(seq if seq.size else np.zeros(1, np.uint8)).to(self.device)
            feat = torch.empty((max(len(qs), 1), ae.MLP_IN), dtype=torch.float32, device=self.device)
            if qs:
                ae.ae_mlp_features(self.index, d_seq.data_ptr(), off, feat.data_ptr(), stream=st)
        return feat[: len(qs)]

    def features(self, queries, stream=None):
        with _on(stream) as st:
            return self.features_device(queries, st).cpu().numpy()

    # -- training data --------------------------------------------------------------------------
    def log_searches(self, queries, Hs, stream=None):
        """Search each query alone; returns targets (n x 2: log1p entries,
        log1p sweep hit records) and calibrates device bytes per entry from a
        fresh workspace per query."""
        T = np.zeros((len(queries), 2), dtype=np.float32)
        obs = []
        for k, (q, h) in enumerate(zip(queries, Hs)):
            ae.ae_workspace_release(self.index, stream)
            ae.ae_search(self.index, [q], self.scheme, [int(h)], stream=stream)
            s = ae.ae_last_stats()
            T[k, 0] = np.log1p(s["entries"])
            T[k, 1] = np.log1p(s["leaf_raw_hits"])
            wb, _ = ae.ae_workspace_info(self.index, stream)
            obs.append((s["entries"], wb))
        ae.ae_workspace_release(self.index, stream)
        if obs:
            # device bytes of a search = a fixed part (sweep scratch, minimum buffers) + a part
            # proportional to the entries; the proportional rate covers 90% of the searches
            e = np.array([o[0] for o in obs], dtype=np.float64)
            b = np.array([o[1] for o in obs], dtype=np.float64)
            self.fixed_bytes = float(b.min())
            rate = (b - self.fixed_bytes)[e > 0] / e[e > 0]
            self.bytes_per_entry = float(np.quantile(rate, 0.9)) if rate.size else self.bytes_per_entry
        return T

    # -- training -------------------------------------------------------------------------------
    def fit(self, X, T, epochs=300, batch=32, lr=1e-3, weight_decay=0.05, spectrum_scale=32.0, seed=0,
            holdout=0.2, stream=None):
        """Train on features X (n x 66) and targets T (n x 2).  Inputs are
        standardised per feature, the 64 spectrum features with a standard
        deviation `spectrum_scale` times their own, so that the network starts
        from the length and interval features and takes composition into
        account only where the data support it (the spectrum of an i.i.d.
        query is mostly sampling noise).  A `holdout` fraction of the rows is
        kept out of training and calibrates the hit-hint margin (the 90th
        percentile of its log residuals); returns the last epoch's loss."""
        torch = _torch()
        X = np.ascontiguousarray(X, dtype=np.float32)
        T = np.ascontiguousarray(T, dtype=np.float32)
        n = X.shape[0]
        order = np.random.default_rng(seed).permutation(n)
        nh = int(round(holdout * n)) if n >= 10 else 0
        cal, tr = order[:nh], order[nh:]
        Xt, Tt = np.ascontiguousarray(X[tr]), np.ascontiguousarray(T[tr])
        x_mu, x_sd = Xt.mean(0), Xt.std(0)
        x_sd = np.where(x_sd > 1e-6, x_sd, 1.0).astype(np.float32)
        x_sd[:64] *= spectrum_scale
        y_mu, y_sd = Tt.mean(0), Tt.std(0)
        y_sd = np.where(y_sd > 1e-6, y_sd, 1.0).astype(np.float32)
        self.mlp.set_norm(x_mu, x_sd, y_mu, y_sd)
        with _on(stream) as st:
            dx = torch.from_numpy(Xt).to(self.device)
            dt = torch.from_numpy(Tt).to(self.device)
            loss = self.mlp.train(dx.data_ptr(), dt.data_ptr(), Xt.shape[0], epochs, batch, lr,
                                  weight_decay=weight_decay, seed=seed, stream=st)
        self.trained = True
        rows = cal if nh else tr
        P = self.predict_features(X[rows], stream)
        res = T[rows, 1] - P[:, 1]
        self.hit_margin = float(np.exp(max(0.0, np.quantile(res, 0.9))))
        return loss

    # -- prediction -----------------------------------------------------------------------------
    def predict_features(self, X, stream=None):
        torch = _torch()
        X = np.ascontiguousarray(X, dtype=np.float32)
        if X.shape[0] == 0:
            return np.zeros((0, 2), dtype=np.float32)
        with _on(stream) as st:
            dx = torch.from_numpy(X).to(self.device)
            dy = torch.empty((X.shape[0], 2), dtype=torch.float32, device=self.device)
            self.mlp.forward(dx.data_ptr(), X.shape[0], dy.data_ptr(), stream=st)
            return dy.cpu().numpy()

    def predict(self, queries, stream=None):
        """(n x 2) predicted log1p(entries), log1p(sweep hit records)."""
        torch = _torch()
        if not queries:
            return np.zeros((0, 2), dtype=np.float32)
        with _on(stream) as st:
            feat = self.features_device(queries, st)
            dy = torch.empty((len(queries), 2), dtype=torch.float32, device=self.device)
            self.mlp.forward(feat.data_ptr(), len(queries), dy.data_ptr(), stream=st)
            return dy.cpu().numpy()

    def hint_hits(self, queries, stream=None):
        P = self.predict(queries, stream)
        return np.ceil(np.expm1(np.maximum(P[:, 1], 0.0)) * self.hit_margin).astype(np.int64)

    def work(self, queries, stream=None):
        """Expected DP entries per query."""
        P = self.predict(queries, stream)
        return np.expm1(np.maximum(P[:, 0], 0.0))

    def work_and_hints(self, queries, stream=None):
        """(expected DP entries, hit hints) per query from one forward pass."""
        P = self.predict(queries, stream)
        work = np.expm1(np.maximum(P[:, 0], 0.0))
        hints = np.ceil(np.expm1(np.maximum(P[:, 1], 0.0)) * self.hit_margin).astype(np.int64)
        return work, hints

    def device_bytes(self, queries, stream=None):
        """Expected device bytes of one search over `queries` together."""
        P = self.predict(queries, stream)
        ent = np.expm1(np.maximum(P[:, 0], 0.0)).sum()
        hits = (np.expm1(np.maximum(P[:, 1], 0.0)) * self.hit_margin).sum()
        return float(self.fixed_bytes + ent * self.bytes_per_entry + 12.0 * hits)
