"""CPU oracle for exact local-alignment search — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The GPU search path neither imports nor
links it, and this package imports nothing from the GPU path.

Contents (each follows the passage it cites):

* ``sw_hits`` / ``sw_matrix`` — the plain full-matrix affine-gap
  Smith-Waterman of ``sw_oracle.c``: the local-alignment problem of Section
  2.1 (largest similarity of T[x..i] and P[y..j] for every end pair, results
  >= H as Algorithm 1 reports them). This is the oracle the GPU hits must match.
* ``sw_hits_mt`` — the same recurrence on every host core: query column
  stripes computed as a wavefront over blocks of text rows, only the edge
  column's V and F crossing between stripes. Pinned bit for bit against
  ``sw_hits`` (``tests/test_oracle_mt.py``); it times the CPU baseline and
  speeds up the large parity windows.
* ``sw_hits_starts`` — the same problem restricted to alignments that start
  at given query columns (no floor at 0, a fresh alignment begins only at an
  allowed column): the share of one part of a search whose forks are split
  over ranks. Pinned by ``local_bruteforce_starts`` (enumeration of every
  alignment from an allowed start) and by its union over a partition, which
  must equal ``sw_hits``.
* ``sim_bruteforce`` / ``local_bruteforce`` — the similarity of Section 2.1
  taken literally: every global alignment of two strings is enumerated and
  scored (no dynamic programming), then maximised over all start pairs. Used
  on inputs of at most ~7 letters to pin ``sw_hits``.
* ``mx_matrices`` — the per-substring matrices M_X, G_a, G_b of Section 2.2
  with the paper's initial conditions (no zero floor); checked against the
  worked values of Fig. 1.
* ``basic_alg1`` — Algorithm 1 (BASIC) over the distinct substrings of a small
  text, scattering max M_X scores into A(i, j); a second, independent route
  to the same result set.
* ``length_bound`` (Eq. 1), ``q_prefix`` (Eq. 2), ``entry_bound`` (Lemma 4 and
  Eq. 4) — closed forms of the paper, used as pins of the analysis.
* ``suffix_array`` — the suffix array of Section 2.3 (suffixes of the codes
  plus a smallest sentinel, in lexicographic order) as its definition: a
  library sort of the start positions with a letter-by-letter comparator
  (``sw_oracle.c``). This is what the index's device suffix array must match.

* ``mlp_oracle`` (submodule) — the work predictor's features, network,
  gradients and Adam step in fp64, with optional bfloat16 rounding of matrix
  operands; pinned in ``tests/test_mlp_oracle.py``.

Every function of this file is parity-pinned by tests in
``tests/test_oracle_pins.py`` (``sw_hits_mt`` in ``tests/test_oracle_mt.py``).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import sys
from functools import lru_cache

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile sw_oracle.c into oracle/liboracle.so (plain C, -O2)."""
    src = os.path.join(_HERE, "sw_oracle.c")
    if (not force and os.path.exists(_LIBPATH)
            and os.path.getmtime(_LIBPATH) >= os.path.getmtime(src)):
        return _LIBPATH
    tmp = _LIBPATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", src, "-o", tmp])
    os.replace(tmp, _LIBPATH)
    return _LIBPATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIBPATH)
        P = ctypes.c_void_p
        lib.ae_oracle_sw_hits.restype = ctypes.c_int64
        lib.ae_oracle_sw_hits.argtypes = [P, ctypes.c_int64, P, ctypes.c_int64, P, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int64, P, P, P, ctypes.c_int64]
        lib.ae_oracle_sw_hits_mt.restype = ctypes.c_int64
        lib.ae_oracle_sw_hits_mt.argtypes = [P, ctypes.c_int64, P, ctypes.c_int64, P, ctypes.c_int32,
                                             ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_int64, ctypes.c_int32, P, P, P, ctypes.c_int64]
        lib.ae_oracle_sw_hits_starts.restype = ctypes.c_int64
        lib.ae_oracle_sw_hits_starts.argtypes = [P, ctypes.c_int64, P, ctypes.c_int64, P, ctypes.c_int32,
                                                 ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P, P, P,
                                                 ctypes.c_int64]
        lib.ae_oracle_sw_matrix.restype = ctypes.c_int
        lib.ae_oracle_sw_matrix.argtypes = [P, ctypes.c_int64, P, ctypes.c_int64, P, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_int32, P]
        lib.ae_oracle_suffix_array.restype = ctypes.c_int
        lib.ae_oracle_suffix_array.argtypes = [P, ctypes.c_int64, P]
        _lib = lib
    return _lib


# --------------------------------------------------------------------------- scoring

def encode(seq, alphabet):
    """ASCII letters -> codes 0..sigma-1 (uint8). Raises on a foreign letter."""
    a = np.frombuffer(alphabet, dtype=np.uint8)
    lut = np.full(256, 255, dtype=np.uint8)
    lut[a] = np.arange(a.size, dtype=np.uint8)
    if isinstance(seq, str):
        seq = seq.encode()
    if isinstance(seq, (bytes, bytearray)):
        s = np.frombuffer(bytes(seq), dtype=np.uint8)
    else:
        s = np.asarray(seq, dtype=np.uint8)
    c = lut[s]
    if c.size and c.max() == 255:
        raise ValueError("letter outside the alphabet")
    return c


def subst_table(scheme, sigma):
    """delta(a, b) as a sigma x sigma int32 table (Section 2.1: s_a when the
    letters are equal, s_b otherwise; or the scheme's substitution matrix)."""
    if getattr(scheme, "matrix", None) is not None:
        return np.ascontiguousarray(np.asarray(scheme.matrix, dtype=np.int32))
    t = np.full((sigma, sigma), scheme.mismatch, dtype=np.int32)
    np.fill_diagonal(t, scheme.match)
    return t


# --------------------------------------------------------------------------- the oracle

def sw_hits(text, query, scheme, H, alphabet=b"ACGT", row_lo=0):
    """Every (text end i, query end j, score) with score >= H (0-based ends),
    row-major; rows below row_lo are computed but not reported."""
    lib = _load()
    T = np.ascontiguousarray(encode(text, alphabet))
    P = np.ascontiguousarray(encode(query, alphabet))
    sub = subst_table(scheme, len(alphabet))
    cap = max(1024, 4 * (T.size + P.size))
    while True:
        oi = np.empty(cap, dtype=np.int64)
        oj = np.empty(cap, dtype=np.int32)
        os_ = np.empty(cap, dtype=np.int32)
        cnt = lib.ae_oracle_sw_hits(T.ctypes.data, T.size, P.ctypes.data, P.size,
                                    sub.ctypes.data, len(alphabet),
                                    int(scheme.gap_open), int(scheme.gap_extend), int(H),
                                    int(row_lo), oi.ctypes.data, oj.ctypes.data,
                                    os_.ctypes.data, cap)
        if cnt < 0:
            raise RuntimeError("oracle failed")
        if cnt <= cap:
            return oi[:cnt], oj[:cnt], os_[:cnt]
        cap = int(cnt)


def host_threads():
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def sw_hits_mt(text, query, scheme, H, alphabet=b"ACGT", row_lo=0, threads=None):
    """sw_hits on `threads` host threads (default: every core this process
    may use): the same recurrence over column stripes in a wavefront, with the
    same results in the same order."""
    lib = _load()
    T = np.ascontiguousarray(encode(text, alphabet))
    P = np.ascontiguousarray(encode(query, alphabet))
    sub = subst_table(scheme, len(alphabet))
    nt = int(threads or host_threads())
    cap = max(1024, 4 * (T.size + P.size))
    while True:
        oi = np.empty(cap, dtype=np.int64)
        oj = np.empty(cap, dtype=np.int32)
        os_ = np.empty(cap, dtype=np.int32)
        cnt = lib.ae_oracle_sw_hits_mt(T.ctypes.data, T.size, P.ctypes.data, P.size,
                                       sub.ctypes.data, len(alphabet),
                                       int(scheme.gap_open), int(scheme.gap_extend), int(H),
                                       int(row_lo), nt, oi.ctypes.data, oj.ctypes.data,
                                       os_.ctypes.data, cap)
        if cnt < 0:
            raise RuntimeError("oracle failed")
        if cnt <= cap:
            return oi[:cnt], oj[:cnt], os_[:cnt]
        cap = int(cnt)


def sw_hits_starts(text, query, scheme, H, allowed, alphabet=b"ACGT"):
    """Results of the alignments that start at query columns y with
    allowed[y] (0-based): every (i, j, score >= H) of the largest similarity
    of such an alignment ending at (i, j). The union of these over a partition
    of the columns, maximised per cell, is sw_hits."""
    lib = _load()
    T = np.ascontiguousarray(encode(text, alphabet))
    P = np.ascontiguousarray(encode(query, alphabet))
    A = np.ascontiguousarray(np.asarray(allowed, dtype=np.uint8))
    if A.size != P.size:
        raise ValueError("one allowed flag per query column")
    sub = subst_table(scheme, len(alphabet))
    cap = max(1024, 4 * (T.size + P.size))
    while True:
        oi = np.empty(cap, dtype=np.int64)
        oj = np.empty(cap, dtype=np.int32)
        os_ = np.empty(cap, dtype=np.int32)
        cnt = lib.ae_oracle_sw_hits_starts(T.ctypes.data, T.size, P.ctypes.data, P.size, sub.ctypes.data,
                                           len(alphabet), int(scheme.gap_open), int(scheme.gap_extend), int(H),
                                           A.ctypes.data, oi.ctypes.data, oj.ctypes.data, os_.ctypes.data, cap)
        if cnt < 0:
            raise RuntimeError("oracle failed")
        if cnt <= cap:
            return oi[:cnt], oj[:cnt], os_[:cnt]
        cap = int(cnt)


def local_bruteforce_starts(text, query, scheme, allowed, alphabet=b"ACGT"):
    """S[i][j] = max over x <= i and allowed y <= j of sim(T[x..i], P[y..j])
    (-inf where no such pair), by enumerating every alignment: the pin of
    sw_hits_starts on small inputs."""
    T = encode(text, alphabet).tolist()
    P = encode(query, alphabet).tolist()
    delta = subst_table(scheme, len(alphabet)).tolist()
    n, m = len(T), len(P)
    S = np.full((n, m), NEG, dtype=np.int64)
    for i in range(n):
        for j in range(m):
            best = NEG
            for x in range(i + 1):
                for y in range(j + 1):
                    if not allowed[y]:
                        continue
                    v = max(_alignment_scores(T[x:i + 1], P[y:j + 1], delta, scheme.gap_open, scheme.gap_extend))
                    best = max(best, v)
            S[i, j] = best
    return S


def sw_matrix(text, query, scheme, alphabet=b"ACGT"):
    """Full n x m matrix of local-alignment cell values (int64)."""
    lib = _load()
    T = np.ascontiguousarray(encode(text, alphabet))
    P = np.ascontiguousarray(encode(query, alphabet))
    sub = subst_table(scheme, len(alphabet))
    V = np.zeros((T.size, P.size), dtype=np.int64)
    if lib.ae_oracle_sw_matrix(T.ctypes.data, T.size, P.ctypes.data, P.size, sub.ctypes.data,
                               len(alphabet), int(scheme.gap_open), int(scheme.gap_extend),
                               V.ctypes.data) != 0:
        raise RuntimeError("oracle failed")
    return V


# --------------------------------------------------------------------------- brute force

def _alignment_scores(a, b, delta, s_g, s_s):
    """Yield the score of every global alignment of code strings a and b.
    An alignment is a sequence of steps: pair a[p] with b[q], a[p] against a
    gap, or b[q] against a gap; a maximal run of r gap steps of one kind scores
    s_g + r*s_s (Section 2.1). Enumerated exhaustively, no DP."""
    la, lb = len(a), len(b)
    # stack entries: (p, q, last_kind, score); last_kind 0 = pair, 1 = gap in b, 2 = gap in a
    stack = [(0, 0, 0, 0)]
    while stack:
        p, q, last, sc = stack.pop()
        if p == la and q == lb:
            yield sc
            continue
        if p < la and q < lb:
            stack.append((p + 1, q + 1, 0, sc + delta[a[p]][b[q]]))
        if p < la:
            stack.append((p + 1, q, 1, sc + (s_s if last == 1 else s_g + s_s)))
        if q < lb:
            stack.append((p, q + 1, 2, sc + (s_s if last == 2 else s_g + s_s)))


def sim_bruteforce(A, B, scheme, alphabet=b"ACGT"):
    """sim(A, B): the best score over all global alignments of A and B."""
    a = encode(A, alphabet).tolist()
    b = encode(B, alphabet).tolist()
    delta = subst_table(scheme, len(alphabet)).tolist()
    return max(_alignment_scores(a, b, delta, scheme.gap_open, scheme.gap_extend))


def local_bruteforce(text, query, scheme, alphabet=b"ACGT"):
    """S[i][j] = max(0, max over x <= i, y <= j of sim(T[x..i], P[y..j])),
    0-based inclusive ends, by enumerating every alignment of every pair of
    non-empty substrings ending at (i, j)."""
    T = encode(text, alphabet).tolist()
    P = encode(query, alphabet).tolist()
    delta = subst_table(scheme, len(alphabet)).tolist()
    n, m = len(T), len(P)
    cache = {}
    S = np.zeros((n, m), dtype=np.int64)
    for i in range(n):
        for j in range(m):
            best = 0
            for x in range(i + 1):
                for y in range(j + 1):
                    key = (tuple(T[x:i + 1]), tuple(P[y:j + 1]))
                    v = cache.get(key)
                    if v is None:
                        v = max(_alignment_scores(list(key[0]), list(key[1]), delta,
                                                  scheme.gap_open, scheme.gap_extend))
                        cache[key] = v
                    best = max(best, v)
            S[i, j] = best
    return S


# --------------------------------------------------------------------------- Section 2.2

NEG = -(1 << 40)


def mx_matrices(X, P, scheme, alphabet=b"ACGT"):
    """(M, Ga, Gb), each (|X|+1) x (|P|+1) int64, for substring X against
    query P with the initial conditions of Section 2.2 — M(0,j)=0,
    M(i,0)=s_g+i*s_s, G_a(0,j)=G_b(i,0)=-inf — and the three recurrences
    applied for every i >= 1, j >= 1 (the range printed as "i > 1, j > 1" is
    read as i >= 1, j >= 1, which is what Fig. 1's first row and column use).
    -inf is NEG. No zero floor: M_X may be negative (Fig. 1)."""
    x = encode(X, alphabet).tolist()
    p = encode(P, alphabet).tolist()
    delta = subst_table(scheme, len(alphabet)).tolist()
    sg, ss = scheme.gap_open, scheme.gap_extend
    d, m = len(x), len(p)
    M = np.zeros((d + 1, m + 1), dtype=np.int64)
    Ga = np.full((d + 1, m + 1), NEG, dtype=np.int64)
    Gb = np.full((d + 1, m + 1), NEG, dtype=np.int64)
    for i in range(1, d + 1):
        M[i, 0] = sg + i * ss
    for i in range(1, d + 1):
        for j in range(1, m + 1):
            Ga[i, j] = max(Ga[i - 1, j] + ss, M[i - 1, j] + sg + ss)
            Gb[i, j] = max(Gb[i, j - 1] + ss, M[i, j - 1] + sg + ss)
            M[i, j] = max(M[i - 1, j - 1] + delta[x[i - 1]][p[j - 1]], Ga[i, j], Gb[i, j])
    return M, Ga, Gb


def basic_alg1(text, query, scheme, H, alphabet=b"ACGT"):
    """Algorithm 1 (BASIC): for every distinct substring X of T (a path of the
    suffix trie) with start positions t_1..t_k, every prefix length i, every
    query end j with M_X(i, j) >= H, raise A(t_h + i - 1, j) to that score;
    return {(text end, query end): score} for A >= H (0-based ends)."""
    T = bytes(np.asarray(text, dtype=np.uint8)) if not isinstance(text, (bytes, str)) else \
        (text.encode() if isinstance(text, str) else text)
    n = len(T)
    occ = {}
    for x in range(n):
        for e in range(x + 1, n + 1):
            occ.setdefault(T[x:e], []).append(x)
    A = {}
    # Every distinct substring X is one node of the suffix trie; the last row
    # of M_X is the row Algorithm 1 aligns when its walk reaches that node,
    # and `starts` are the node's occurrences t_1..t_k.
    for X, starts in occ.items():
        M, _, _ = mx_matrices(X, query, scheme, alphabet)
        i = len(X)
        for j in range(1, M.shape[1]):
            s = int(M[i, j])
            if s >= H:
                for t in starts:
                    key = (t + i - 1, j - 1)
                    if s > A.get(key, 0):
                        A[key] = s
    return {k: v for k, v in A.items() if v >= H}


# --------------------------------------------------------------------------- closed forms

def length_bound(m, H, scheme):
    """Eq. 1 (Theorem 1): rows i with ceil(H/s_a) <= i <= L_max are meaningful,
    L_max = max{m, m + floor((H - (s_a*m + s_g)) / s_s)} with the mathematical
    floor of the signed quotient. Returns (lower, L_max)."""
    sa = scheme.match if scheme.matrix is None else int(np.max(scheme.matrix))
    lo = -(-H // sa)
    L = max(m, m + math.floor((H - (sa * m + scheme.gap_open)) / scheme.gap_extend))
    return lo, L


def q_prefix(scheme):
    """Eq. 2: q = floor(min{|s_b|, |s_g + s_s|} / s_a) + 1."""
    return min(abs(scheme.mismatch), abs(scheme.gap_open + scheme.gap_extend)) // scheme.match + 1


def entry_bound(sa, sb, sigma, q):
    """Lemma 4 and Eq. 4: s = 1 + |s_b|/|s_a|,
    k1 = (1-1/s)^q ((sigma-1)/(sigma-2)) s / sqrt(2 pi (s-1)),
    k2 = s ((sigma-1)/(s-1)^(s-1))^(1/s),
    expected entries <= (k1/(k2-1) + k1 sigma^2/(sigma-k2)) m n^(log_sigma k2).
    Returns (k1, k2, exponent, coefficient)."""
    s = 1.0 + abs(sb) / abs(sa)
    k1 = (1.0 - 1.0 / s) ** q * ((sigma - 1.0) / (sigma - 2.0)) * s / math.sqrt(2.0 * math.pi * (s - 1.0))
    k2 = s * ((sigma - 1.0) / (s - 1.0) ** (s - 1.0)) ** (1.0 / s)
    expo = math.log(k2) / math.log(sigma)
    coef = k1 / (k2 - 1.0) + k1 * sigma * sigma / (sigma - k2)
    return k1, k2, expo, coef


def threshold_from_evalue(K, lam, m, n, E):
    """Section 7: H = ceil((ln(K m n) - ln E) / lambda)."""
    return int(math.ceil((math.log(K * m * n) - math.log(E)) / lam))


# --------------------------------------------------------------------------- suffix array

def suffix_array(codes):
    """Start positions of the suffixes of ``codes`` (uint8 letter codes < 255)
    followed by a sentinel smaller than every letter, in lexicographic order
    of the suffixes (Section 2.3); n + 1 entries, the first is n."""
    c = np.ascontiguousarray(np.asarray(codes, dtype=np.uint8))
    if c.size and int(c.max()) >= 255:
        raise ValueError("letter codes must be below 255")
    sa = np.empty(c.size + 1, dtype=np.int32)
    if _load().ae_oracle_suffix_array(c.ctypes.data, c.size, sa.ctypes.data) != 0:
        raise MemoryError("oracle suffix array")
    return sa
