"""Thresholds H from an E-value (Section 7) for the scaled DNA workload.

Section 7 sets H = ceil((ln(K m n) - ln E) / lambda) with K and lambda taken
from BLAST's tables, which are not available here. This script estimates them
for the gapped scheme <1,-3,-5,-2> at the workload's composition (41% GC) by
fitting an extreme-value (Gumbel) law to the oracle's best local score over
random sequence pairs:  P(S_max < x) = exp(-K m n e^{-lambda x}), so that
lambda = pi / (sd * sqrt 6) and K = exp(lambda * mean - gamma) / (m n)
(method of moments; edge effects ignored). It calls only the oracle and the
input generators, and prints the thresholds the workload module freezes.

    python -m oracle.evalue_fit [pairs] [length]
    python -m oracle.evalue_fit sweep      # the scheme and E-value sweeps' thresholds
"""
import math
import sys

import numpy as np

import oracle
from workloads import DNA, Scheme, gc_probs, iid_text

EULER_GAMMA = 0.5772156649015329


def fit(pairs=200, length=1000, gc=0.41, seed=99, scheme=None):
    scheme = scheme or Scheme(1, -3, -5, -2)
    rng = np.random.default_rng(seed)
    best = []
    for _ in range(pairs):
        a = iid_text(length, DNA, gc_probs(gc), rng)
        b = iid_text(length, DNA, gc_probs(gc), rng)
        best.append(int(oracle.sw_matrix(a, b, scheme).max()))
    s = np.asarray(best, dtype=np.float64)
    lam = math.pi / (s.std(ddof=1) * math.sqrt(6.0))
    K = math.exp(lam * s.mean() - EULER_GAMMA) / (length * length)
    return lam, K, s


def thresholds(lam, K, n=100_000_000, lengths=(10_000, 100_000, 1_000_000), E=10.0):
    return {m: oracle.threshold_from_evalue(K, lam, m, n, E) for m in lengths}


# The paper's scheme sweep (Section 7.4, Fig. 9: m = 100,000, E = 10) and E-value
# sweep (Section 7.3, Fig. 8: E from 1e-15 to 10 under <1,-3,-5,-2>), at the
# scaled text length n = 10^8.
SWEEP_SCHEMES = [(1, -3, -5, -2), (1, -4, -5, -2), (1, -1, -5, -2), (1, -3, -2, -2)]
SWEEP_E = [1e-15, 1e-5, 10.0]


def sweep_thresholds(pairs=200, length=1000, n=100_000_000):
    """{scheme: (lambda, K, {E: {m: H}})}: a Gumbel fit per scheme, thresholds
    for m = 10 kbp and 100 kbp at each E of the E-value sweep (the scheme sweep
    uses E = 10, m = 100 kbp)."""
    out = {}
    for sc in SWEEP_SCHEMES:
        lam, K, _ = fit(pairs, length, scheme=Scheme(*sc))
        out[sc] = (lam, K, {E: {m: oracle.threshold_from_evalue(K, lam, m, n, E) for m in (10_000, 100_000)}
                           for E in SWEEP_E})
    return out


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "sweep":
        for sc, (lam, K, H) in sweep_thresholds().items():
            print(f"{sc}: lambda={lam:.4f} K={K:.4f} H={H}")
        sys.exit(0)
    pairs = int(sys.argv[1]) if len(sys.argv) > 1 else 200
    length = int(sys.argv[2]) if len(sys.argv) > 2 else 1000
    lam, K, s = fit(pairs, length)
    print(f"lambda={lam:.4f} K={K:.4f} mean={s.mean():.2f} sd={s.std(ddof=1):.2f}")
    print(thresholds(lam, K))
