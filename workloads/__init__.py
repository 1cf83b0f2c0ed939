"""Seeded synthetic inputs for exact local-alignment search.

This module only draws random sequences; it holds none of the alignment
arithmetic. Both the CPU oracle tests and the GPU path take their inputs from
here, so that the two sides see byte-identical texts and queries.

Sequences are ASCII byte arrays (numpy uint8): DNA over "ACGT", protein over
the 20 standard residues in the order "ARNDCQEGHILKMFPSTWYV".

Workload shapes (the paper measures on GRCh37 / MGSCv37 chr1 / UniParc, which
are not available here; these i.i.d. texts with planted homologous segments
stand in for them, see the design notes):

* ``dna_small``   n = 100,000 uniform ACGT; one 1,000 bp query with 5 planted,
                  mutated copies of 150-300 bp text segments; <1,-3,-5,-2>, H=30.
* ``dna_scale``   n = 100,000,000 at 41% GC; 8 queries each of 10 kbp, 100 kbp
                  and 1 Mbp, 1% of each query planted from the text at 5-15%
                  divergence; <1,-3,-5,-2>, H from E = 10 per query length.
* ``protein``     n = 50,000,000 residues at background frequencies; queries of
                  100 / 1,000 / 5,000 residues with planted homologs at 30-60%
                  identity; BLOSUM62, gap open -11, gap extend -1, H = 50.
* ``dna_batch``   4,096 queries, lengths log-uniform in [100, 20,000], against
                  the ``dna_scale`` text.
* ``dna_serve``   Poisson arrivals of queries (70% log-uniform 200-2,000 bp,
                  30% log-uniform 2,000-100,000 bp) against the same text.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

DNA = b"ACGT"
PROTEIN = b"ARNDCQEGHILKMFPSTWYV"

# Background residue frequencies in PROTEIN order (Robinson & Robinson 1991,
# PNAS 88:8880, as commonly tabulated); renormalised below.
_PROTEIN_BG = np.array([
    0.07805, 0.05129, 0.04487, 0.05364, 0.01925, 0.04264, 0.06295, 0.07377,
    0.02199, 0.05142, 0.09019, 0.05744, 0.02243, 0.03856, 0.05203, 0.07120,
    0.05841, 0.01330, 0.03216, 0.06441])
PROTEIN_BG = _PROTEIN_BG / _PROTEIN_BG.sum()

# BLOSUM62 (Henikoff & Henikoff 1992, PNAS 89:10915), rows/cols in PROTEIN order.
BLOSUM62 = np.array([
    # A   R   N   D   C   Q   E   G   H   I   L   K   M   F   P   S   T   W   Y   V
    [ 4, -1, -2, -2,  0, -1, -1,  0, -2, -1, -1, -1, -1, -2, -1,  1,  0, -3, -2,  0],  # A
    [-1,  5,  0, -2, -3,  1,  0, -2,  0, -3, -2,  2, -1, -3, -2, -1, -1, -3, -2, -3],  # R
    [-2,  0,  6,  1, -3,  0,  0,  0,  1, -3, -3,  0, -2, -3, -2,  1,  0, -4, -2, -3],  # N
    [-2, -2,  1,  6, -3,  0,  2, -1, -1, -3, -4, -1, -3, -3, -1,  0, -1, -4, -3, -3],  # D
    [ 0, -3, -3, -3,  9, -3, -4, -3, -3, -1, -1, -3, -1, -2, -3, -1, -1, -2, -2, -1],  # C
    [-1,  1,  0,  0, -3,  5,  2, -2,  0, -3, -2,  1,  0, -3, -1,  0, -1, -2, -1, -2],  # Q
    [-1,  0,  0,  2, -4,  2,  5, -2,  0, -3, -3,  1, -2, -3, -1,  0, -1, -3, -2, -2],  # E
    [ 0, -2,  0, -1, -3, -2, -2,  6, -2, -4, -4, -2, -3, -3, -2,  0, -2, -2, -3, -3],  # G
    [-2,  0,  1, -1, -3,  0,  0, -2,  8, -3, -3, -1, -2, -1, -2, -1, -2, -2,  2, -3],  # H
    [-1, -3, -3, -3, -1, -3, -3, -4, -3,  4,  2, -3,  1,  0, -3, -2, -1, -3, -1,  3],  # I
    [-1, -2, -3, -4, -1, -2, -3, -4, -3,  2,  4, -2,  2,  0, -3, -2, -1, -2, -1,  1],  # L
    [-1,  2,  0, -1, -3,  1,  1, -2, -1, -3, -2,  5, -1, -3, -1,  0, -1, -3, -2, -2],  # K
    [-1, -1, -2, -3, -1,  0, -2, -3, -2,  1,  2, -1,  5,  0, -2, -1, -1, -1, -1,  1],  # M
    [-2, -3, -3, -3, -2, -3, -3, -3, -1,  0,  0, -3,  0,  6, -4, -2, -2,  1,  3, -1],  # F
    [-1, -2, -2, -1, -3, -1, -1, -2, -2, -3, -3, -1, -2, -4,  7, -1, -1, -4, -3, -2],  # P
    [ 1, -1,  1,  0, -1,  0,  0,  0, -1, -2, -2,  0, -1, -2, -1,  4,  1, -3, -2, -2],  # S
    [ 0, -1,  0, -1, -1, -1, -1, -2, -2, -1, -1, -1, -1, -2, -1,  1,  5, -2, -2,  0],  # T
    [-3, -3, -4, -4, -2, -2, -3, -2, -2, -3, -2, -3, -1,  1, -4, -3, -2, 11,  2, -3],  # W
    [-2, -2, -2, -3, -2, -1, -2, -3,  2, -1, -1, -2, -1,  3, -3, -2, -2,  2,  7, -1],  # Y
    [ 0, -3, -3, -3, -1, -2, -2, -3, -3,  3,  1, -2,  1, -1, -2, -2,  0, -3, -1,  4],  # V
], dtype=np.int8)


@dataclass
class Scheme:
    """Scoring <s_a, s_b, s_g, s_s>, or a substitution matrix with gaps."""
    match: int = 1
    mismatch: int = -3
    gap_open: int = -5
    gap_extend: int = -2
    matrix: np.ndarray | None = None      # sigma x sigma int8, alphabet order

    def as_dict(self):
        return {"match": self.match, "mismatch": self.mismatch,
                "gap_open": self.gap_open, "gap_extend": self.gap_extend,
                "matrix": None if self.matrix is None else "BLOSUM62"}


@dataclass
class Workload:
    name: str
    alphabet: bytes
    text: np.ndarray                       # uint8 ASCII
    queries: list                          # list of uint8 ASCII arrays
    scheme: Scheme
    H: list                                # per-query threshold
    seed: int
    recipe: dict = field(default_factory=dict)
    arrivals: np.ndarray | None = None     # serving workloads: arrival times (s)

    @property
    def n(self):
        return int(self.text.size)


def iid_text(n, alphabet, probs, rng):
    """i.i.d. sequence of n letters drawn from `alphabet` with `probs`."""
    a = np.frombuffer(alphabet, dtype=np.uint8)
    cdf = np.cumsum(np.asarray(probs, dtype=np.float64))
    cdf[-1] = 1.0
    out = np.empty(n, dtype=np.uint8)
    step = 1 << 24
    for s in range(0, n, step):
        u = rng.random(min(step, n - s))
        out[s:s + u.size] = a[np.searchsorted(cdf, u, side="right")]
    return out


def gc_probs(gc):
    """ACGT probabilities for a GC fraction (A=T, C=G)."""
    at = (1.0 - gc) / 2.0
    return [at, gc / 2.0, gc / 2.0, at]


def mutate(seg, alphabet, probs, sub_p, indel_p, rng, max_indel=3):
    """Copy `seg` applying, per source position, an indel event with
    probability indel_p (insertion or deletion 50/50, length uniform in
    1..max_indel) or else a substitution with probability sub_p (uniform over
    the other letters). Inserted letters are drawn from `probs`."""
    a = np.frombuffer(alphabet, dtype=np.uint8)
    out = []
    i = 0
    L = seg.size
    while i < L:
        r = rng.random()
        if r < indel_p:
            k = int(rng.integers(1, max_indel + 1))
            if rng.random() < 0.5:                       # insertion before seg[i]
                out.extend(a[rng.choice(a.size, size=k, p=probs)].tolist())
            else:                                        # deletion of k letters
                i += k
                continue
        elif r < indel_p + sub_p:
            c = int(seg[i])
            others = a[a != c]
            out.append(int(others[rng.integers(0, others.size)]))
            i += 1
            continue
        out.append(int(seg[i]))
        i += 1
    return np.array(out, dtype=np.uint8)


def plant_query(text, m, seg_lengths, alphabet, probs, sub_p, indel_p, rng):
    """A query of exactly m letters: i.i.d. background with the mutated copies
    of len(seg_lengths) distinct random text segments placed in order, separated
    by random spacers. Returns (query, list of (text_start, length, q_start))."""
    n = text.size
    pieces, spans = [], []
    starts = set()
    for L in seg_lengths:
        while True:
            s = int(rng.integers(0, n - L))
            if all(abs(s - t) > 2 * L for t in starts):
                break
        starts.add(s)
        sp = sub_p() if callable(sub_p) else sub_p
        ip = indel_p(sp) if callable(indel_p) else indel_p
        pieces.append((s, L, mutate(text[s:s + L], alphabet, probs, sp, ip, rng)))
    body = sum(p[2].size for p in pieces)
    free = max(0, m - body)
    cuts = np.sort(rng.integers(0, free + 1, size=len(pieces)))
    gaps = np.diff(np.concatenate([[0], cuts, [free]]))
    out = []
    pos = 0
    for k, (s, L, piece) in enumerate(pieces):
        g = int(gaps[k])
        out.append(iid_text(g, alphabet, probs, rng))
        pos += g
        spans.append((s, L, pos))
        out.append(piece)
        pos += piece.size
    out.append(iid_text(int(gaps[-1]), alphabet, probs, rng))
    q = np.concatenate(out)[:m]
    if q.size < m:
        q = np.concatenate([q, iid_text(m - q.size, alphabet, probs, rng)])
    return q, spans


def _planted_lengths(total, lo, hi, rng):
    """Segment lengths uniform in [lo, hi], capped by what is left of `total`."""
    out = []
    left = total
    while left > 0:
        L = int(rng.integers(lo, hi + 1))
        L = min(L, left)
        out.append(L)
        left -= L
    return out


def dna_small(seed=20120801, n=100_000, m=1_000, copies=5):
    """Uniform ACGT text of n bp; one m bp query carrying `copies` planted
    copies of 150-300 bp text segments (lengths redrawn until their sum is at
    most m - 50), 10% substitutions and 2% indel events of length 1-3."""
    rng = np.random.default_rng(seed)
    probs = [0.25] * 4
    text = iid_text(n, DNA, probs, rng)
    while True:
        lens = rng.integers(150, 301, size=copies)
        if lens.sum() <= m - 50:
            break
    q, spans = plant_query(text, m, [int(x) for x in lens], DNA, probs, 0.10, 0.02, rng)
    return Workload("dna_small", DNA, text, [q], Scheme(), [30], seed,
                    {"n": n, "m": m, "planted": spans, "sub": 0.10, "indel": 0.02})


# Thresholds for <1,-3,-5,-2> at 41% GC and n = 1e8 from E = 10, H = ceil((ln(K m n) - ln E)/lambda),
# with lambda and K fitted on oracle maxima of random pairs (oracle/evalue_fit.py, reproduced by
# the test suite).
DNA_SCALE_H = {10_000: 19, 100_000: 21, 1_000_000: 23}

# Thresholds of the scheme sweep (Section 7.4, Fig. 9: four BLAST schemes, E = 10,
# m = 100 kbp) and of the E-value sweep (Section 7.3, Fig. 8: E = 1e-15, 1e-5, 10),
# for the 10^8-letter text at 41% GC: a Gumbel fit of the oracle's best scores on
# random pairs per scheme, frozen from `python -m oracle.evalue_fit sweep`
# (lambda, K: 1.2892, 0.2187 / 1.3044, 0.2416 / 1.0639, 0.1778 / 1.2957, 0.2394).
SWEEP_H = {
    (1, -3, -5, -2): {1e-15: {10_000: 48, 100_000: 49}, 1e-5: {10_000: 30, 100_000: 31}, 10.0: {10_000: 19, 100_000: 21}},
    (1, -4, -5, -2): {1e-15: {10_000: 47, 100_000: 49}, 1e-5: {10_000: 29, 100_000: 31}, 10.0: {10_000: 19, 100_000: 21}},
    (1, -1, -5, -2): {1e-15: {10_000: 57, 100_000: 59}, 1e-5: {10_000: 36, 100_000: 38}, 10.0: {10_000: 23, 100_000: 25}},
    (1, -3, -2, -2): {1e-15: {10_000: 47, 100_000: 49}, 1e-5: {10_000: 30, 100_000: 31}, 10.0: {10_000: 19, 100_000: 21}},
}


def dna_scale_text(seed=20120802, n=100_000_000, gc=0.41):
    rng = np.random.default_rng(seed)
    return iid_text(n, DNA, gc_probs(gc), rng)


def dna_scale_query(text, m, rng, gc=0.41, frac=0.01):
    """Query of m bp at the text's composition with `frac` of its length drawn
    from planted text segments (300-3,000 bp, capped by the budget) at a
    divergence uniform in 5-15%, split 5:1 between substitutions and indels."""
    probs = gc_probs(gc)
    lens = _planted_lengths(max(1, int(round(frac * m))), 300, 3000, rng)
    div = lambda: float(rng.uniform(0.05, 0.15))
    return plant_query(text, m, lens, DNA, probs,
                       lambda: div() * 5.0 / 6.0, lambda sp: sp / 5.0, rng)


def dna_scale(seed=20120802, n=100_000_000, lengths=(10_000, 100_000, 1_000_000),
              per_length=8, text=None):
    if text is None:
        text = dna_scale_text(seed, n)
    rng = np.random.default_rng(seed + 1)
    queries, H, spans = [], [], []
    for m in lengths:
        for _ in range(per_length):
            q, sp = dna_scale_query(text, m, rng)
            queries.append(q)
            H.append(DNA_SCALE_H.get(m, _nearest_H(m)))
            spans.append(sp)
    return Workload("dna_scale", DNA, text, queries, Scheme(), H, seed,
                    {"n": n, "lengths": list(lengths), "per_length": per_length,
                     "gc": 0.41, "planted": spans})


def dna_scale_bench(seed=20120802, n=100_000_000, lengths=(10_000, 100_000, 1_000_000), per_length=8):
    """The benchmark's scaled DNA workload: (text, queries, H, planted spans).
    Spans are (text start, length, query start) of each planted segment."""
    text = dna_scale_text(seed, n)
    rng = np.random.default_rng(seed + 1)
    queries, H, spans = [], [], []
    for m in lengths:
        for _ in range(per_length):
            q, sp = dna_scale_query(text, m, rng)
            queries.append(q)
            H.append(DNA_SCALE_H.get(m, _nearest_H(m)))
            spans.append(sp)
    return text, queries, H, spans


def _nearest_H(m):
    keys = sorted(DNA_SCALE_H)
    k = min(keys, key=lambda x: abs(math.log(x) - math.log(max(m, 1))))
    return DNA_SCALE_H[k]


def h_for_length(m):
    """Threshold used for a query of length m against the 1e8 bp text
    (log-interpolated between the fitted lengths)."""
    return _nearest_H(m)


def protein(seed=20120803, n=50_000_000, lengths=(100, 1_000, 5_000), per_length=8,
            text=None):
    """Residue text at background frequencies; queries with planted homologs
    (one per 100-residue query, ~10% of longer ones) at identity U[30%, 60%]:
    non-identical positions are redrawn from the background, plus 2% indels."""
    rng = np.random.default_rng(seed)
    if text is None:
        text = iid_text(n, PROTEIN, PROTEIN_BG, rng)
    queries, spans = [], []
    for m in lengths:
        for _ in range(per_length):
            L = min(m, max(50, m // 10)) if m > 100 else 60
            ident = float(rng.uniform(0.30, 0.60))
            q, sp = plant_query(text, m, [L], PROTEIN, PROTEIN_BG,
                                1.0 - ident, 0.02, rng)
            queries.append(q)
            spans.append(sp)
    return Workload("protein", PROTEIN, text, queries,
                    Scheme(gap_open=-11, gap_extend=-1, matrix=BLOSUM62),
                    [50] * len(queries), seed, {"n": n, "lengths": list(lengths),
                                                "planted": spans})


def log_uniform_lengths(k, lo, hi, rng):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=k)).astype(np.int64)


def dna_batch(text, seed=20120804, k=4096, lo=100, hi=20_000):
    rng = np.random.default_rng(seed)
    lens = log_uniform_lengths(k, lo, hi, rng)
    qs = [dna_scale_query(text, int(m), rng)[0] for m in lens]
    return Workload("dna_batch", DNA, text, qs, Scheme(),
                    [h_for_length(int(m)) for m in lens], seed, {"k": k, "lo": lo, "hi": hi})


def dna_serve(text, seed=20120805, k=20_000, rate=200.0):
    rng = np.random.default_rng(seed)
    short = rng.random(k) < 0.7
    lens = np.where(short, log_uniform_lengths(k, 200, 2_000, rng),
                    log_uniform_lengths(k, 2_000, 100_000, rng))
    qs = [dna_scale_query(text, int(m), rng)[0] for m in lens]
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=k))
    return Workload("dna_serve", DNA, text, qs, Scheme(),
                    [h_for_length(int(m)) for m in lens], seed,
                    {"k": k, "rate": rate}, arrivals=arrivals)


def random_pair(n, m, alphabet=DNA, probs=None, seed=0):
    """Small i.i.d. text/query pair for property tests."""
    rng = np.random.default_rng(seed)
    if probs is None:
        probs = [1.0 / len(alphabet)] * len(alphabet)
    return iid_text(n, alphabet, probs, rng), iid_text(m, alphabet, probs, rng)
