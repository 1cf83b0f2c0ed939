"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each check is chosen so that a plausible slip in the oracle (a dropped gap
state, a wrong open/extend charge, a transposed operand, an off-by-one end
index, a missing zero floor) fails at least one of them:

* exhaustive enumeration of every alignment on tiny inputs (Section 2.1's
  definition, no DP) against the full-matrix oracle, for several schemes;
* Algorithm 1 (BASIC) over the suffix-trie paths of small texts, an
  independent route to the result set;
* the worked values of Fig. 1 and the similarity example of Section 2.1;
* closed forms: exact copy, a single gap of known length, a long copy whose
  score exceeds int16;
* invariants: threshold monotonicity, text/query transpose symmetry;
* the paper's own constants for Eq. 1, Eq. 2, Lemma 4 / Eq. 4.
"""
import math
import os

import numpy as np
import pytest

import oracle
from workloads import DNA, PROTEIN, BLOSUM62, Scheme, iid_text, random_pair

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

SCHEMES = [
    Scheme(1, -3, -5, -2),      # default scheme of the paper (Section 2.1)
    Scheme(1, -1, -5, -2),      # Table 5 / Fig. 9 schemes
    Scheme(1, -3, -2, -2),
    Scheme(2, -3, -1, -1),      # s_a > 1, cheap gaps: stresses gap states
    Scheme(1, -1, 0, -1),       # zero gap open: linear gaps
]


def _dna(s):
    return np.frombuffer(s.encode(), dtype=np.uint8)


@pytest.mark.parametrize("scheme", SCHEMES, ids=lambda s: f"{s.match}{s.mismatch}{s.gap_open}{s.gap_extend}")
def test_bruteforce_matches_oracle_random(scheme):
    rng = np.random.default_rng(7)
    for case in range(6):
        n = int(rng.integers(1, 7))
        m = int(rng.integers(1, 7))
        # small alphabets make repeats, matches and gap-worthy alignments common
        alph = b"AC" if case % 2 == 0 else DNA
        T = iid_text(n, alph, [1.0 / len(alph)] * len(alph), rng)
        P = iid_text(m, alph, [1.0 / len(alph)] * len(alph), rng)
        S = oracle.local_bruteforce(T, P, scheme)
        V = oracle.sw_matrix(T, P, scheme)
        assert np.array_equal(S, V), (bytes(T), bytes(P))


def test_bruteforce_gap_cases():
    # Inputs where the best alignment needs a gap, back-to-back gaps of both
    # kinds, or ends inside a gap.
    s = Scheme(2, -3, -1, -1)
    for T, P in [("ACCA", "AA"), ("AA", "ACCA"), ("AACC", "ACAC"), ("ACGTA", "AGTCA"),
                 ("AAGGAA", "AAAA"), ("GATTACA", "GATAC")]:
        S = oracle.local_bruteforce(_dna(T), _dna(P), s)
        V = oracle.sw_matrix(_dna(T), _dna(P), s)
        assert np.array_equal(S, V), (T, P)


def test_similarity_example_section_2_1():
    # sim(AAACG, AACCG) = 1*4 + (-3) = 1 under <1,-3,-5,-2>
    assert oracle.sim_bruteforce("AAACG", "AACCG", Scheme(1, -3, -5, -2)) == 1


def _read_fig1():
    rows = []
    with open(os.path.join(GOLDEN, "fig1_mx.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append(line.split())
    return rows


def test_fig1_matrices():
    M, Ga, Gb = oracle.mx_matrices("GCTA", "GCTAG", Scheme(1, -3, -5, -2))
    assert (M[0, :] == 0).all() and (Ga[0, :] == oracle.NEG).all()
    checked = 0
    for parts in _read_fig1():
        i, j = int(parts[0]), int(parts[1])
        assert M[i, j] == int(parts[2]), (i, j)
        if parts[3] != ".":
            assert Ga[i, j] == int(parts[3]), (i, j)
        gb = oracle.NEG if parts[4] == "-inf" else int(parts[4])
        if len(parts) > 5 and parts[5].startswith("printed-typo:"):
            gb = int(parts[5].split(":")[1])
        assert Gb[i, j] == gb, (i, j)
        checked += 1
    assert checked == 24
    # The worked step of Section 2.2: M_X(4,3) = max{-5-3, -4, -14} = -4.
    assert (M[4, 3], Ga[4, 3], Gb[4, 3]) == (-4, -4, -14)


def test_theorem5_example_fgoe_scores():
    # Section 4.1's example for Theorem 5: X = GCTACCCCCTTTGGAA and two forks whose
    # query segments GCTACACCCTTT and GCTACCTCCTTT each differ from X[1..12] in one
    # letter; both first gap-open entries score 8 (11 matches, one mismatch), and the
    # common substring GGAA after them carries both on to 8 + s
    X = "GCTACCCCCTTTGGAA"
    P = "GCTACACCCTTT" + "GGAA" + "GCTACCTCCTTT" + "GGAA"
    M, _, _ = oracle.mx_matrices(X, P, Scheme(1, -3, -5, -2))
    pi1, pi2 = 1, 17
    assert M[12, pi1 + 11] == 8 and M[12, pi2 + 11] == 8
    for s in range(5):
        assert M[12 + s, pi1 + 11 + s] == M[12 + s, pi2 + 11 + s] == 8 + s


def test_basic_alg1_matches_oracle():
    rng = np.random.default_rng(11)
    for scheme in SCHEMES[:4]:
        for _ in range(4):
            T = iid_text(int(rng.integers(4, 13)), b"ACG", [0.4, 0.3, 0.3], rng)
            P = iid_text(int(rng.integers(3, 10)), b"ACG", [0.4, 0.3, 0.3], rng)
            for H in (1, 2, 3):
                A = oracle.basic_alg1(T, P, scheme, H)
                oi, oj, os_ = oracle.sw_hits(T, P, scheme, H)
                got = {(int(a), int(b)): int(c) for a, b, c in zip(oi, oj, os_)}
                assert got == A, (bytes(T), bytes(P), H)


def test_exact_copy_closed_form():
    s = Scheme(1, -3, -5, -2)
    T, _ = random_pair(2000, 1, seed=3)
    for x, L in [(0, 50), (700, 120), (1950, 50)]:
        P = T[x:x + L].copy()
        oi, oj, os_ = oracle.sw_hits(T, P, s, 1)
        hit = {(int(a), int(b)): int(c) for a, b, c in zip(oi, oj, os_)}
        # the copy ends at text position x+L-1, query position L-1, score L*s_a
        assert hit[(x + L - 1, L - 1)] == L
        # nothing can score more: P has only L letters
        assert max(hit.values()) == L


def test_single_gap_closed_form():
    s = Scheme(1, -3, -5, -2)
    rng = np.random.default_rng(5)
    U = iid_text(40, DNA, [0.25] * 4, rng)
    W = iid_text(30, DNA, [0.25] * 4, rng)
    for k in (1, 3, 6):
        V = iid_text(k, DNA, [0.25] * 4, rng)
        T = np.concatenate([iid_text(25, DNA, [0.25] * 4, rng), U, V, W])
        P = np.concatenate([U, W])
        M = oracle.sw_matrix(T, P, s)
        # U.V.W against U.W: |U|+|W| matches and one gap of k letters
        assert M[T.size - 1, P.size - 1] == s.match * (U.size + W.size) + s.gap_open + k * s.gap_extend


def test_long_copy_exceeds_int16():
    s = Scheme(1, -3, -5, -2)
    T, _ = random_pair(40_100, 1, seed=9)
    P = T[50:40_050].copy()
    oi, oj, os_ = oracle.sw_hits(T, P, s, 39_995)
    top = int(np.argmax(os_))
    assert (int(oi[top]), int(oj[top]), int(os_[top])) == (40_049, 39_999, 40_000)
    assert int(os_.max()) > 32_767


def test_threshold_monotonicity():
    s = Scheme(1, -3, -5, -2)
    T, P = random_pair(3000, 200, seed=12)
    P[40:120] = T[1000:1080]
    lo = oracle.sw_hits(T, P, s, 8)
    hi = oracle.sw_hits(T, P, s, 15)
    lo_set = {(int(a), int(b), int(c)) for a, b, c in zip(*lo) if c >= 15}
    hi_set = {(int(a), int(b), int(c)) for a, b, c in zip(*hi)}
    assert lo_set == hi_set and len(hi_set) > 0


def test_transpose_symmetry():
    for scheme in SCHEMES:
        T, P = random_pair(60, 45, seed=21)
        P[10:30] = T[5:25]
        A = oracle.sw_matrix(T, P, scheme)
        B = oracle.sw_matrix(P, T, scheme)
        assert np.array_equal(A, B.T)


def test_substitution_matrix_path():
    # BLOSUM62 is symmetric; a matrix scheme must agree with enumeration too.
    assert np.array_equal(BLOSUM62, BLOSUM62.T)
    assert int(np.diag(BLOSUM62).min()) > 0 and int(BLOSUM62.max()) == 11
    s = Scheme(gap_open=-11, gap_extend=-1, matrix=BLOSUM62)
    rng = np.random.default_rng(4)
    for _ in range(3):
        T = iid_text(5, PROTEIN, [0.05] * 20, rng)
        P = iid_text(5, PROTEIN, [0.05] * 20, rng)
        S = oracle.local_bruteforce(T, P, s, alphabet=PROTEIN)
        V = oracle.sw_matrix(T, P, s, alphabet=PROTEIN)
        assert np.array_equal(S, V)


def test_row_window_reporting():
    s = Scheme(1, -3, -5, -2)
    T, P = random_pair(400, 80, seed=31)
    P[5:60] = T[200:255]
    full = oracle.sw_hits(T, P, s, 10)
    part = oracle.sw_hits(T, P, s, 10, row_lo=230)
    want = [(a, b, c) for a, b, c in zip(*full) if a >= 230]
    got = list(zip(*part))
    assert [tuple(map(int, w)) for w in want] == [tuple(map(int, g)) for g in got]


def test_eq1_length_bound():
    # Section 3.1.1 example: P = GCTAC, H = 3: Eq. 1 gives 3 <= i <= 5 (the
    # prose's "between 3 and 4" disagrees with Eq. 1; Eq. 1 is taken).
    assert oracle.length_bound(5, 3, Scheme(1, -3, -5, -2)) == (3, 5)
    # m = 1,000 and H = 30: L_max = 1000 + floor((30 - 995) / -2) = 1482
    assert oracle.length_bound(1000, 30, Scheme(1, -3, -5, -2)) == (30, 1482)


def test_eq2_q_prefix():
    # Section 3.1.3: q = 4 for <1,-3,-5,-2>
    assert oracle.q_prefix(Scheme(1, -3, -5, -2)) == 4
    assert oracle.q_prefix(Scheme(1, -1, -5, -2)) == 2
    assert oracle.q_prefix(Scheme(2, -3, -5, -2)) == 2


def test_entry_bound_constants():
    # Section 6: for <1,-3,-5,-2> on DNA, k2 = 2.3094, log_4 k2 = 0.6038,
    # k1 = 0.4373 and the bound is 4.47 m n^0.6038.
    k1, k2, e, c = oracle.entry_bound(1, -3, 4, 4)
    assert round(k2, 4) == 2.3094 and round(e, 4) == 0.6038
    assert round(k1, 4) == 0.4373 and round(c, 2) == 4.47
    # Abstract: 4.50 mn^0.520 ... 9.05 mn^0.896 (DNA), 8.28 mn^0.364 ... 7.49 mn^0.723 (protein)
    for (sb, sigma, q), (cc, ee) in [((-4, 4, 5), (4.50, 0.520)), ((-1, 4, 2), (9.05, 0.896)),
                                     ((-4, 20, 5), (8.28, 0.364)), ((-1, 20, 2), (7.49, 0.723))]:
        _, _, e, c = oracle.entry_bound(1, sb, sigma, q)
        # the paper prints two or three decimals (0.5195 appears as 0.520)
        assert abs(c - cc) <= 0.006 and abs(e - ee) <= 0.0006


def test_evalue_threshold_is_monotone():
    a = oracle.threshold_from_evalue(0.7, 1.3, 1e4, 1e8, 10.0)
    b = oracle.threshold_from_evalue(0.7, 1.3, 1e4, 1e8, 1e-5)
    c = oracle.threshold_from_evalue(0.7, 1.3, 1e6, 1e8, 10.0)
    assert a < b and a < c


def test_dna_scale_thresholds_reproduce():
    # The workload's frozen H per query length comes from oracle.evalue_fit.
    from oracle import evalue_fit
    from workloads import DNA_SCALE_H
    lam, K, _ = evalue_fit.fit(300, 1000)
    assert evalue_fit.thresholds(lam, K) == DNA_SCALE_H


# --------------------------------------------------------------------------- suffix array (Section 2.3)

def test_oracle_suffix_array_paper_examples():
    # Section 2.3: SA of GCTAGC$ is {7, 4, 6, 2, 5, 1, 3} (1-based starts)
    t = oracle.encode(b"GCTAGC", DNA)
    assert list(oracle.suffix_array(t) + 1) == [7, 4, 6, 2, 5, 1, 3]
    # Section 5 (2): over T^-1 with positions kept the array reads {0, 4, 2, 6, 1, 5, 3}
    sa = oracle.suffix_array(t[::-1].copy())
    assert [t.size - k for k in sa] == [0, 4, 2, 6, 1, 5, 3]


def _sa_by_list_sort(codes):
    s = [int(c) for c in codes] + [-1]          # the sentinel below every letter
    return sorted(range(len(s)), key=lambda k: s[k:])


@pytest.mark.parametrize("seed", range(4))
def test_oracle_suffix_array_bruteforce(seed):
    rng = np.random.default_rng(100 + seed)
    for sigma, n in [(4, 0), (4, 1), (4, 2), (2, 40), (4, 300), (20, 200)]:
        codes = rng.integers(0, sigma, size=n).astype(np.uint8)
        if seed % 2 and n > 7:
            codes = np.tile(codes[: max(1, n // 9)], 10)[:n]
        assert list(oracle.suffix_array(codes)) == _sa_by_list_sort(codes)


def _bwt_inverse(codes, sa):
    """Text read back from the BWT of `sa` by LF steps (the Burrows-Wheeler
    inversion): right only if `sa` lists the suffixes in order."""
    n = codes.size
    bwt = np.where(sa > 0, codes[np.maximum(sa - 1, 0)].astype(np.int64), -1)
    lf = np.empty(n + 1, dtype=np.int64)
    lf[np.argsort(bwt, kind="stable")] = np.arange(n + 1)
    out = np.empty(n, dtype=np.int64)
    h = 0                                        # the row of the sentinel suffix
    for k in range(n - 1, -1, -1):
        out[k] = bwt[h]
        h = lf[h]
    return out


@pytest.mark.parametrize("kind", ["iid", "period7", "one_letter", "protein"])
def test_oracle_suffix_array_inverts_through_bwt(kind):
    rng = np.random.default_rng(7)
    n = 6000
    if kind == "protein":
        codes = rng.integers(0, 20, size=n).astype(np.uint8)
    elif kind == "one_letter":
        codes = np.zeros(n, dtype=np.uint8)
    elif kind == "period7":
        codes = np.tile(rng.integers(0, 4, size=7), n // 7 + 1)[:n].astype(np.uint8)
    else:
        codes = rng.integers(0, 4, size=n).astype(np.uint8)
    sa = oracle.suffix_array(codes)
    assert sa[0] == n and np.array_equal(np.sort(sa), np.arange(n + 1))
    assert np.array_equal(_bwt_inverse(codes, sa), codes)
    # and a misordered array fails the same check: swap two adjacent rows whose
    # BWT letters differ (equal letters would leave the BWT string unchanged)
    bwt = np.where(sa > 0, codes[np.maximum(sa - 1, 0)].astype(np.int64), -1)
    p = int(np.flatnonzero(bwt[:-1] != bwt[1:])[-1])
    bad = sa.copy()
    bad[[p, p + 1]] = bad[[p + 1, p]]
    assert not np.array_equal(_bwt_inverse(codes, bad), codes)


def test_sweep_thresholds_are_the_fits_frozen_values():
    # the scheme and E-value sweeps' thresholds (workloads.SWEEP_H) are what the
    # oracle-only fitting script gives for each scheme and E
    from oracle import evalue_fit
    from workloads import SWEEP_H
    got = evalue_fit.sweep_thresholds()
    assert set(got) == set(SWEEP_H)
    for sc, (lam, K, H) in got.items():
        assert H == SWEEP_H[sc], sc
        assert 0.5 < lam < 2.0 and 0.01 < K < 1.0
    # stricter E, higher threshold; a smaller |s_b| spreads scores, lowering lambda
    for sc in SWEEP_H:
        h = SWEEP_H[sc]
        assert h[1e-15][100_000] > h[1e-5][100_000] > h[10.0][100_000]
    assert got[(1, -1, -5, -2)][0] < got[(1, -3, -5, -2)][0]
