"""q-prefix domination (Lemma 1), with the reading that a seed gram X is
dominated at query start y only if *every* occurrence of X in T is preceded by
the query letter P[y-1].  The fork starting at y is then matched cell for cell,
one match better, by the fork starting at y - 1, so dropping it changes no
result.

Checked here: on a text where it fires (a text made of a few repeated words),
the number of dropped forks equals a brute-force count over the query's seed
positions, and the results equal the oracle's with the filter on and off; on
i.i.d. text nothing is dropped.  Also checked on a collection, where a gram at
the start of a sequence has no preceding letter and so is never dominated.
"""
import numpy as np
import pytest

import oracle
from workloads import DNA, Scheme, iid_text, random_pair

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1208_0274_gb300 import ae  # noqa: E402

# q = min(6, 9) / 1 + 1 = 7 (Eq. 2), so the walk starts at depth d0 = 6
SCHEME = Scheme(1, -6, -7, -2)


def _want(T, P, H):
    oi, oj, os_ = oracle.sw_hits(T, P, SCHEME, H)
    w = np.zeros(oi.size, dtype=ae.HIT_DTYPE)
    w["text_end"], w["query_end"], w["score"] = oi, oj, os_
    return w


def _brute_dominated(seqs, P, d0):
    """Seed positions y >= 1 of P whose gram occurs in the text and every
    occurrence of which (inside one sequence) is preceded by P[y-1]."""
    prev = {}
    for T in seqs:
        t = bytes(T)
        for p in range(len(t) - d0 + 1):
            g = t[p:p + d0]
            prev.setdefault(g, set()).add(t[p - 1] if p > 0 else None)
    q = bytes(P)
    return sum(1 for y in range(1, len(q) - d0 + 1) if prev.get(q[y:y + d0]) == {q[y - 1]})


def _word_text(rng, words, n_words):
    return np.concatenate([words[int(k)] for k in rng.integers(0, len(words), size=n_words)])


def test_domination_fires_on_repetitive_text_and_keeps_results():
    rng = np.random.default_rng(31)
    words = [iid_text(40, DNA, [0.25] * 4, rng) for _ in range(6)]
    T = _word_text(rng, words, 400)
    P = _word_text(rng, words, 12)
    flip = rng.random(P.size) < 0.03
    P[flip] = np.frombuffer(DNA, dtype=np.uint8)[rng.integers(0, 4, size=int(flip.sum()))]
    H = 20
    assert ae.ae_plan(P.size, SCHEME, H)[1] == 6
    idx = ae.ae_index_build(T, ae.AE_DNA)
    want = _want(T, P, H)
    assert want.size > 100
    on, _ = ae.ae_search(idx, [P], SCHEME, [H])
    st_on = ae.ae_last_stats()
    off, _ = ae.ae_search(idx, [P], SCHEME, [H], options=ae.make_options(qprefix_domination=0))
    st_off = ae.ae_last_stats()
    assert np.array_equal(on, want) and np.array_equal(off, want)
    assert st_off["dominated"] == 0
    assert st_on["dominated"] == _brute_dominated([T], P, 6) > 50
    # fewer forks walked, fewer DP entries
    assert st_on["entries"] < st_off["entries"]
    idx.close()


def test_domination_never_fires_on_iid_text():
    T, P = random_pair(300_000, 3_000, seed=5)
    P[500:900] = T[100_000:100_400]
    idx = ae.ae_index_build(T, ae.AE_DNA)
    hits, _ = ae.ae_search(idx, [P], SCHEME, [20])
    assert ae.ae_last_stats()["dominated"] == 0
    assert np.array_equal(hits, _want(T, P, 20))
    idx.close()


def test_domination_respects_sequence_starts_in_a_collection():
    rng = np.random.default_rng(32)
    words = [iid_text(30, DNA, [0.25] * 4, rng) for _ in range(4)]
    seqs = [_word_text(rng, words, 40) for _ in range(5)]
    P = _word_text(rng, words, 10)
    H = 18
    idx = ae.ae_index_build_collection(seqs, ae.AE_DNA)
    on, c_on = ae.ae_search(idx, [P], SCHEME, [H])
    dom = ae.ae_last_stats()["dominated"]
    off, _ = ae.ae_search(idx, [P], SCHEME, [H], options=ae.make_options(qprefix_domination=0))
    assert np.array_equal(on, off)
    assert dom == _brute_dominated(seqs, P, 6) > 0
    # the oracle: each sequence on its own
    off_t = np.cumsum([0] + [s.size for s in seqs[:-1]])
    parts = []
    for s, o in zip(seqs, off_t):
        w = _want(s, P, H)
        w["text_end"] += o
        parts.append(w)
    want = np.sort(np.concatenate(parts), order=["text_end", "query_end"])
    assert np.array_equal(on, want)
    idx.close()
