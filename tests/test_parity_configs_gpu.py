"""Exact parity on the protein workload's query lengths and on the last query
columns of a 1 Mbp query, where the threshold of Theorem 2 bites.

Both cases are too large for the oracle's full matrix, so the oracle runs on
windows that provably contain every alignment a checked result can come from:

* Protein (BLOSUM62, gap -11/-1, H = 50; 1,000- and 5,000-residue queries with
  planted homologs at 30-60% identity against a 2 M-residue text).  A result
  at query end j uses at most m query letters, so by Eq. 1 (with the largest
  matrix entry g = 11 in place of s_a) its text span is at most
  L_max(m) = m + floor((H - (g m + s_g)) / s_s).  The oracle on
  T[a - L_max .. b] x P therefore gives the true value of every cell with text
  end in [a, b].

* The query tail (<1,-3,-5,-2>, H = 23: the E = 10 threshold of a 1 Mbp query
  against 10^8 letters).  The threshold thr(j) = max{0, H - 1 - (m - 1 - j) s_a}
  of Theorem 2 is positive only in the last H - 1 columns, which no window of
  the full-size test reaches.  Here the text has n_t = 60,000 letters, so an
  alignment spans at most n_t text letters and, by Eq. 1 with the roles of text
  and query swapped, at most L_max(n_t) query letters.  The oracle on
  T x P[m - J - L_max(n_t) .. m) then gives the true value of every cell with
  query end in [m - J, m).  Short planted segments end inside the last H
  columns, so the kept and the pruned states there decide real results.
"""
import numpy as np
import pytest

import oracle
from workloads import PROTEIN, Scheme, gc_probs, iid_text, mutate, protein, DNA

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1208_0274_gb300 import ae  # noqa: E402


def _search_all(idx, queries, scheme, H, opts):
    seq = np.concatenate(queries)
    offsets = np.concatenate([[0], np.cumsum([q.size for q in queries])]).astype(np.int64)
    d_seq = torch.from_numpy(seq).cuda()
    cap = 1 << 22
    while True:
        out = torch.empty(cap * 16, dtype=torch.uint8, device="cuda")
        st, counts = ae.ae_search_device(idx, d_seq.data_ptr(), offsets, scheme, H, out.data_ptr(), cap,
                                         options=opts)
        if st == ae.AE_OK:
            break
        assert st == ae.AE_EOVERFLOW
        cap = int(counts.sum()) + 1024
        del out
    hits = out[: int(counts.sum()) * 16].cpu().numpy().view(ae.HIT_DTYPE)
    starts = np.concatenate([[0], np.cumsum(counts)])
    return [hits[starts[k]:starts[k + 1]] for k in range(len(queries))]


def _as_hits(oi, oj, os_):
    w = np.zeros(oi.size, dtype=ae.HIT_DTYPE)
    w["text_end"], w["query_end"], w["score"] = oi, oj, os_
    return w


def _compare(got, want, label):
    if not np.array_equal(got, want):
        g = {(int(a), int(b)): int(c) for a, b, c in got}
        w = {(int(a), int(b)): int(c) for a, b, c in want}
        bad = [(k, g.get(k), w.get(k)) for k in set(g) | set(w) if g.get(k) != w.get(k)][:6]
        raise AssertionError(f"{label}: {len(got)} vs {len(want)} results; first differences {bad}")


def test_protein_1000_and_5000_residue_queries_windows():
    wl = protein(n=2_000_000, lengths=[1_000, 5_000], per_length=4)
    idx = ae.ae_index_build(wl.text, ae.AE_PROTEIN)
    H = 50
    per_query = _search_all(idx, wl.queries, wl.scheme, [H] * len(wl.queries), ae.make_options())
    n = wl.text.size
    rng = np.random.default_rng(5)
    checked = 0
    for qi, q in enumerate(wl.queries):
        Lmax = oracle.length_bound(q.size, H, wl.scheme)[1]
        s, L, _ = wl.recipe["planted"][qi][0]
        r = int(rng.integers(Lmax, n - 20_000))
        for a, b in [(max(0, s - 300), min(n - 1, s + L + 300)), (r, r + 20_000)]:
            a0 = max(0, a - Lmax)
            oi, oj, os_ = oracle.sw_hits_mt(wl.text[a0:b + 1], q, wl.scheme, H, alphabet=PROTEIN, row_lo=a - a0)
            want = _as_hits(oi + a0, oj, os_)
            g = per_query[qi]
            got = g[(g["text_end"] >= a) & (g["text_end"] <= b)]
            _compare(got, want, f"protein query {qi} (m={q.size}) text ends [{a}, {b}]")
            checked += want.size
    assert checked > 1_000
    idx.close()


def _tail_query(text, m, tail_end_gap, rng, probs):
    """A query of m letters (background composition) carrying a 1,500-letter
    homolog of the text ending 400 letters before the end and a short homolog
    (34-46 letters, at most two substitutions, so it scores >= 26 > H) ending
    tail_end_gap letters before the end: its results fall in the columns
    where thr(j) > 0."""
    q = iid_text(m, DNA, probs, rng)
    n = text.size
    s1 = int(rng.integers(0, n - 1_500))
    long_seg = mutate(text[s1:s1 + 1_500], DNA, probs, 0.05, 0.01, rng)
    e1 = m - 400
    q[e1 - long_seg.size:e1] = long_seg
    L2 = int(rng.integers(34, 47))
    s2 = int(rng.integers(0, n - L2))
    short_seg = text[s2:s2 + L2].copy()
    for p in rng.choice(L2, size=int(rng.integers(0, 3)), replace=False):
        short_seg[p] = [c for c in b"ACGT" if c != short_seg[p]][int(rng.integers(0, 3))]
    e2 = m - tail_end_gap
    q[e2 - L2:e2] = short_seg
    return q


def test_one_megabase_query_tail_where_threshold_bites():
    rng = np.random.default_rng(23)
    probs = gc_probs(0.41)
    n_t, m, H = 60_000, 1_000_000, 23
    text = iid_text(n_t, DNA, probs, rng)
    queries = [_tail_query(text, m, gap, rng, probs) for gap in (0, 3, 9, 17)]
    idx = ae.ae_index_build(text, ae.AE_DNA)
    scheme = Scheme(1, -3, -5, -2)
    # the benchmark's launch configuration: 2 M query letters per engine batch, leaf delay 10
    per_query = _search_all(idx, queries, scheme, [H] * len(queries),
                            ae.make_options(batch_columns=1 << 21, leaf_delay=10))
    Lq = oracle.length_bound(n_t, H, scheme)[1]
    J = 3_000
    tail_hits = 0
    for qi, q in enumerate(queries):
        y0 = m - J - Lq
        oi, oj, os_ = oracle.sw_hits_mt(text, q[y0:], scheme, H)
        oj = oj + y0
        keep = oj >= m - J
        want = _as_hits(oi[keep], oj[keep], os_[keep])
        g = per_query[qi]
        got = g[g["query_end"] >= m - J]
        _compare(got, want, f"1 Mbp query {qi}: query ends [{m - J}, {m})")
        tail_hits += int(np.sum(want["query_end"] >= m - (H - 1)))
        # nothing is reported past the query's last column
        assert g.size == 0 or int(g["query_end"].max()) < m
    # results do land in the columns where the threshold is positive
    assert tail_hits > 0
    idx.close()


def test_protein_match_mismatch_scheme_of_the_index_experiments():
    # Section 7.5 pairs protein texts with <1,-3,-11,-1>: a match/mismatch scheme over
    # 20 letters, so q-prefix seeding (Eq. 2: q = 4) and the domination filter are on,
    # unlike BLOSUM62.  Full oracle on 300 k residues.
    from workloads import PROTEIN_BG
    rng = np.random.default_rng(17)
    T = iid_text(300_000, PROTEIN, PROTEIN_BG, rng)
    scheme = Scheme(1, -3, -11, -1)
    idx = ae.ae_index_build(T, ae.AE_PROTEIN)
    qs, Hs = [], []
    for k, m in enumerate((300, 1_000, 2_500)):
        P = iid_text(m, PROTEIN, PROTEIN_BG, rng)
        L = m // 3
        x = int(rng.integers(0, T.size - L))
        seg = T[x:x + L].copy()
        flip = rng.random(L) < 0.15
        seg[flip] = iid_text(int(flip.sum()), PROTEIN, PROTEIN_BG, rng)
        P[m // 4:m // 4 + L] = seg
        qs.append(P)
        Hs.append(12 + 3 * k)
    assert ae.ae_plan(1_000, scheme, 12, ae.AE_PROTEIN)[0] == 4
    hits, counts = ae.ae_search(idx, qs, scheme, Hs)
    parts = np.split(hits, np.cumsum(counts)[:-1])
    for k, (P, H) in enumerate(zip(qs, Hs)):
        want = _as_hits(*oracle.sw_hits_mt(T, P, scheme, H, alphabet=PROTEIN))
        assert want.size > 0
        _compare(parts[k], want, f"protein <1,-3,-11,-1> query {k}")
    st = ae.ae_last_stats()
    assert st["seed_depth"] == 3
    idx.close()
