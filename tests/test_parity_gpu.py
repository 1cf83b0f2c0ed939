"""GPU search through the C ABI against the CPU oracle, hit for hit.

Every comparison is exact: the set of (text end, query end, score) results
with score >= H, sorted by (text end, query end), must be identical.
"""
import numpy as np
import pytest

import oracle
from workloads import (BLOSUM62, DNA, PROTEIN, Scheme, dna_small, iid_text, random_pair)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1208_0274_gb300 import ae  # noqa: E402


def want_hits(T, P, scheme, H, alphabet=DNA):
    oi, oj, os_ = oracle.sw_hits(T, P, scheme, H, alphabet=alphabet)
    w = np.zeros(oi.size, dtype=ae.HIT_DTYPE)
    w["text_end"], w["query_end"], w["score"] = oi, oj, os_
    return w   # row-major order == sorted by (text_end, query_end)


def split(hits, counts):
    out, s = [], 0
    for c in counts:
        out.append(hits[s:s + c])
        s += c
    return out


def assert_same(got, want, label=""):
    if not np.array_equal(got, want):
        g = {(int(a), int(b)): int(c) for a, b, c in got}
        w = {(int(a), int(b)): int(c) for a, b, c in want}
        extra = [(k, v) for k, v in g.items() if w.get(k) != v][:5]
        miss = [(k, v) for k, v in w.items() if g.get(k) != v][:5]
        raise AssertionError(f"{label}: got {len(got)} want {len(want)}; wrong/extra {extra}; missing {miss}")


def planted_pair(rng, n, m, sub=0.1):
    T, P = random_pair(n, m, seed=int(rng.integers(1 << 30)))
    if n > 40 and m > 30:
        L = int(rng.integers(10, min(n, m) // 2))
        x = int(rng.integers(0, n - L))
        y = int(rng.integers(0, m - L))
        seg = T[x:x + L].copy()
        flip = rng.random(L) < sub
        seg[flip] = np.frombuffer(DNA, dtype=np.uint8)[rng.integers(0, 4, size=int(flip.sum()))]
        P[y:y + L] = seg
    return T, P


@pytest.fixture(scope="module")
def small():
    wl = dna_small()
    idx = ae.ae_index_build(wl.text, ae.AE_DNA)
    yield wl, idx
    idx.close()


def test_dna_small_workload_full_parity(small):
    wl, idx = small
    hits, counts = ae.ae_search(idx, wl.queries, wl.scheme, wl.H)
    want = want_hits(wl.text, wl.queries[0], wl.scheme, wl.H[0])
    assert counts[0] == want.size and want.size > 1000
    assert_same(hits, want, "dna_small")
    st = ae.ae_last_stats()
    assert st["entries"] > 0 and st["hits"] == want.size and st["seed_depth"] == 3
    assert st["levels_int16"] == st["levels"]          # DNA rows never leave the int16 route here
    assert st["entries_tier"] == [0, 0, 0]             # tier counting is off by default
    # with tier_stats every entry (of the trie levels and of the sweep) falls in one tier
    hits2, _ = ae.ae_search(idx, wl.queries, wl.scheme, wl.H, options=ae.make_options(tier_stats=1))
    assert np.array_equal(hits2, hits)
    st2 = ae.ae_last_stats()
    assert sum(st2["entries_tier"]) == st2["entries"] and st2["entries_tier"][0] > 0
    # filter statistics (Eq. 5): slot candidates of the trie levels, those the filters
    # dropped, and the kept ones, which with the gap-run cells are the trie's entries
    cand, npos, nreach = st2["candidates"], st2["pruned_nonpos"], st2["pruned_reach"]
    assert cand > 0 and npos > 0 and nreach > 0 and npos + nreach < cand
    assert cand - npos - nreach <= st2["entries"] - st2["entries_leaf"]
    assert st["candidates"] == 0        # counted only with tier_stats
    # reuse at text positions (Eq. 6): rows of different starts meet along the homologs
    assert st["reused"] > 0 and st2["reused"] > 0
    assert st["reroutes"] == 0
    ae.ae_search(idx, wl.queries, wl.scheme, wl.H, options=ae.make_options(int16_limit=6))
    assert ae.ae_last_stats()["reroutes"] >= 1


@pytest.mark.parametrize("opts", [dict(qprefix_seed=0), dict(leaf_segment=1), dict(leaf_segment=7),
                                  dict(item_columns=97), dict(item_columns=250, batch_columns=300),
                                  dict(leaf_capacity=64), dict(leaf_delay=0), dict(leaf_delay=3),
                                  dict(leaf_delay=14, leaf_segment=5), dict(int16_limit=0),
                                  dict(int16_limit=6), dict(int16_limit=13, leaf_delay=14),
                                  dict(leaf_wide_rows=0), dict(leaf_wide_rows=8, leaf_delay=0),
                                  dict(leaf_wide_rows=33, leaf_segment=3)])
def test_dna_small_knobs_do_not_change_hits(small, opts):
    wl, idx = small
    want = want_hits(wl.text, wl.queries[0], wl.scheme, wl.H[0])
    hits, counts = ae.ae_search(idx, wl.queries, wl.scheme, wl.H, options=ae.make_options(**opts))
    assert_same(hits, want, str(opts))


SCHEMES = [Scheme(1, -3, -5, -2), Scheme(1, -1, -5, -2), Scheme(1, -3, -2, -2), Scheme(2, -3, -1, -1),
           Scheme(1, -4, -5, -2), Scheme(1, -2, 0, -1)]


@pytest.mark.parametrize("si", range(len(SCHEMES)))
def test_random_planted_cases(si):
    scheme = SCHEMES[si]
    rng = np.random.default_rng(100 + si)
    for case in range(8):
        n = int(rng.integers(50, 3000))
        m = int(rng.integers(5, 400))
        T, P = planted_pair(rng, n, m)
        idx = ae.ae_index_build(T, ae.AE_DNA)
        for H in (4, 9, 17):
            for seed_on in (1, 0):
                opts = ae.make_options(qprefix_seed=seed_on, leaf_segment=int(rng.integers(1, 40)),
                                       item_columns=int(rng.integers(3, 500)),
                                       leaf_delay=int(rng.integers(0, 15)),
                                       int16_limit=int(rng.choice([0, 5, 9, 32000])),
                                       general_rows=int(rng.integers(0, 2)),
                                       row_layout=int(rng.integers(0, 4)),
                                       leaf_wide_rows=int(rng.choice([0, 4, 33, 256])))
                hits, _ = ae.ae_search(idx, [P], scheme, [H], options=opts)
                assert_same(hits, want_hits(T, P, scheme, H), f"case {case} H {H} seed {seed_on}")
        idx.close()


def test_row_kernels_agree_entry_for_entry():
    """The DNA int16x2 row kernel in both layouts (one lane per parent entry
    with all children; one lane per (node, child) walking the parent row) and
    the general one (one lane per (child, parent entry)) compute the same trie
    levels: identical results, DP entries, triples and nodes, on a 1 Mbp text
    with planted homologs of several lengths and at several leaf delays."""
    rng = np.random.default_rng(11)
    T, _ = random_pair(1_000_000, 1, seed=12)
    qs = []
    for m in (300, 2_000, 20_000, 60_000):
        _, P = random_pair(1, m, seed=int(rng.integers(1 << 30)))
        for _ in range(max(1, m // 5_000)):
            L = int(rng.integers(50, min(m, 3_000)))
            x, y = int(rng.integers(0, T.size - L)), int(rng.integers(0, m - L + 1))
            seg = T[x:x + L].copy()
            flip = rng.random(L) < 0.08
            seg[flip] = np.frombuffer(DNA, dtype=np.uint8)[rng.integers(0, 4, size=int(flip.sum()))]
            P[y:y + L] = seg
        qs.append(P)
    Hs = [16, 19, 21, 23]
    scheme = Scheme(1, -3, -5, -2)
    idx = ae.ae_index_build(T, ae.AE_DNA)
    for delay in (0, 8, 14):
        got = {}
        for kind, opts in (("general", dict(general_rows=1)), ("auto", dict()),
                           ("walk", dict(row_layout=1)), ("spread", dict(row_layout=2)),
                           ("block", dict(row_layout=3))):
            hits, counts = ae.ae_search(idx, qs, scheme, Hs, options=ae.make_options(leaf_delay=delay, **opts))
            st = ae.ae_last_stats()
            got[kind] = (hits, counts, st["entries"], st["triples"], st["nodes"], st["injections"])
        ref = got["general"]
        assert ref[0].size > 1_000
        for kind, g in got.items():
            assert np.array_equal(g[0], ref[0]) and np.array_equal(g[1], ref[1]), (delay, kind)
            assert g[2:] == ref[2:], (delay, kind, g[2:], ref[2:])
    idx.close()


def test_wide_sweep_walks_on_blocks_keep_every_hit(small):
    # walks whose rows grow past leaf_wide_rows entries continue on a whole block;
    # with a low threshold most sweep walks do (and more than there are slots, so
    # some stay on their warps): the hits equal the oracle's and the warp-only run's
    wl, idx = small
    want = want_hits(wl.text, wl.queries[0], wl.scheme, wl.H[0])
    base, _ = ae.ae_search(idx, wl.queries, wl.scheme, wl.H, options=ae.make_options(leaf_wide_rows=0, leaf_delay=0))
    assert ae.ae_last_stats()["leaf_wide_walks"] == 0
    for thr in (2, 8, 40):
        hits, _ = ae.ae_search(idx, wl.queries, wl.scheme, wl.H,
                               options=ae.make_options(leaf_wide_rows=thr, leaf_delay=0, leaf_segment=2))
        st = ae.ae_last_stats()
        assert st["leaf_wide_walks"] > 0, thr
        assert_same(hits, want, f"leaf_wide_rows {thr}")
        assert np.array_equal(hits, base)
    # protein rows in the block walk
    rng = np.random.default_rng(77)
    T = iid_text(6000, PROTEIN, [0.05] * 20, rng)
    P = T[1000:1400].copy()
    P[::9] = np.frombuffer(PROTEIN, dtype=np.uint8)[rng.integers(0, 20, size=P[::9].size)]
    pidx = ae.ae_index_build(T, ae.AE_PROTEIN)
    sc = Scheme(matrix=BLOSUM62, gap_open=-11, gap_extend=-1)
    for thr in (0, 8):
        hits, _ = ae.ae_search(pidx, [P], sc, [40], options=ae.make_options(leaf_wide_rows=thr, leaf_delay=0))
        assert_same(hits, want_hits(T, P, sc, 40, alphabet=PROTEIN), f"protein, leaf_wide_rows {thr}")
    pidx.close()


def test_multi_query_batch_equals_single():
    rng = np.random.default_rng(7)
    T, _ = random_pair(5000, 1, seed=3)
    qs, Hs = [], []
    for k in range(9):
        _, P = planted_pair(rng, 5000, int(rng.integers(1, 300)))
        L = min(P.size, 60)
        if k % 2 and P.size > L:
            x = int(rng.integers(0, 5000 - L))
            P[:L] = T[x:x + L]
        qs.append(P)
        Hs.append(int(rng.integers(6, 20)))
    qs.append(np.zeros(0, dtype=np.uint8))     # an empty query
    Hs.append(5)
    scheme = Scheme(1, -3, -5, -2)
    idx = ae.ae_index_build(T, ae.AE_DNA)
    hits, counts = ae.ae_search(idx, qs, scheme, Hs)
    parts = split(hits, counts)
    for k, (P, H) in enumerate(zip(qs, Hs)):
        want = want_hits(T, P, scheme, H) if P.size else np.zeros(0, dtype=ae.HIT_DTYPE)
        assert_same(parts[k], want, f"query {k}")
        alone, c1 = ae.ae_search(idx, [P], scheme, [H])
        assert_same(alone, want, f"alone {k}")
    idx.close()


def test_protein_blosum62():
    rng = np.random.default_rng(3)
    bg = [0.05] * 20
    T = iid_text(20_000, PROTEIN, bg, rng)
    scheme = Scheme(gap_open=-11, gap_extend=-1, matrix=BLOSUM62)
    idx = ae.ae_index_build(T, ae.AE_PROTEIN)
    for m, H in [(60, 30), (200, 40), (500, 50)]:
        P = iid_text(m, PROTEIN, bg, rng)
        L = m // 2
        x = int(rng.integers(0, T.size - L))
        seg = T[x:x + L].copy()
        flip = rng.random(L) < 0.4
        seg[flip] = np.frombuffer(PROTEIN, dtype=np.uint8)[rng.integers(0, 20, size=int(flip.sum()))]
        P[m // 4:m // 4 + L] = seg
        want = want_hits(T, P, scheme, H, alphabet=PROTEIN)
        for lim in (32000, 40, 0):
            hits, _ = ae.ae_search(idx, [P], scheme, [H], options=ae.make_options(int16_limit=lim))
            assert_same(hits, want, f"protein m={m} int16_limit={lim}")
    idx.close()


def test_edge_cases():
    scheme = Scheme(1, -3, -5, -2)
    # one-letter text; H = 1 makes every equal letter pair a hit (root start)
    for T, P, H in [(b"A", b"A", 1), (b"A", b"C", 1), (b"ACGT", b"ACGT", 1), (b"ACGTACGTTT", b"GT", 1),
                    (b"ACGTTGCA" * 20, b"TTGCAACG", 3), (b"ACGT" * 50, b"ACGT" * 10, 1000)]:
        idx = ae.ae_index_build(T, ae.AE_DNA)
        hits, _ = ae.ae_search(idx, [P], scheme, [H])
        assert_same(hits, want_hits(np.frombuffer(T, np.uint8), np.frombuffer(P, np.uint8), scheme, H),
                    f"{T[:10]} {P} {H}")
        idx.close()


def test_exact_copy_and_int16_overflow_scores():
    scheme = Scheme(1, -3, -5, -2)
    T, _ = random_pair(120_000, 1, seed=8)
    P = T[30_000:70_000].copy()               # score 40,000 > int16 range
    idx = ae.ae_index_build(T, ae.AE_DNA)
    hits, _ = ae.ae_search(idx, [P], scheme, [39_990])
    want = want_hits(T, P, scheme, 39_990)
    assert_same(hits, want, "40k copy")
    top = hits[np.argmax(hits["score"])]
    assert (int(top["text_end"]), int(top["query_end"]), int(top["score"])) == (69_999, 39_999, 40_000)
    idx.close()


def test_threshold_monotonicity_on_device(small):
    wl, idx = small
    lo, _ = ae.ae_search(idx, wl.queries, wl.scheme, [22])
    hi, _ = ae.ae_search(idx, wl.queries, wl.scheme, [40])
    assert_same(hi, lo[lo["score"] >= 40], "H monotonicity")


def test_device_entry_point_and_overflow(small):
    wl, idx = small
    q = torch.from_numpy(np.concatenate(wl.queries)).cuda()
    offsets = np.array([0, wl.queries[0].size], dtype=np.int64)
    want = want_hits(wl.text, wl.queries[0], wl.scheme, wl.H[0])
    out = torch.empty((want.size + 10) * 16, dtype=torch.uint8, device="cuda")
    st, counts = ae.ae_search_device(idx, q.data_ptr(), offsets, wl.scheme, wl.H, out.data_ptr(),
                                     want.size + 10)
    assert st == ae.AE_OK and counts[0] == want.size
    got = out[:want.size * 16].cpu().numpy().view(ae.HIT_DTYPE)
    assert_same(got, want, "device")
    st, counts = ae.ae_search_device(idx, q.data_ptr(), offsets, wl.scheme, wl.H, out.data_ptr(), 5)
    assert st == ae.AE_EOVERFLOW and counts[0] == want.size


def test_large_host_results_equal_the_device_results():
    # results past 32 MB leave the device in shares copied by several host threads
    # through pinned chunks: they must equal the device entry point's results byte
    # for byte, and the returned array must keep its buffer alive on its own
    # (an exact copy of L letters at H = 30 gives about 0.4 L^2 results: past the
    # diagonal's score d, gapped extensions stay above H for gaps up to (d - H) / 2)
    rng = np.random.default_rng(77)
    T = iid_text(200_000, DNA, [0.25] * 4, rng)
    qs = [T[x:x + L].copy() for x, L in ((10_000, 2_000), (80_000, 2_011), (150_000, 1_999))]
    scheme, Hs = Scheme(), [30] * len(qs)
    idx = ae.ae_index_build(T, ae.AE_DNA)
    hits, counts = ae.ae_search(idx, qs, scheme, Hs)
    assert 32 << 20 < hits.nbytes < 160 << 20 and hits.size == counts.sum()
    d = torch.from_numpy(np.concatenate(qs)).cuda()
    off = np.concatenate([[0], np.cumsum([q.size for q in qs])]).astype(np.int64)
    out = torch.empty(hits.size * 16, dtype=torch.uint8, device="cuda")
    st, c2 = ae.ae_search_device(idx, d.data_ptr(), off, scheme, Hs, out.data_ptr(), hits.size)
    assert st == ae.AE_OK and np.array_equal(c2, counts)
    assert np.array_equal(out.cpu().numpy().view(ae.HIT_DTYPE), hits)
    tail = hits[-1000:]
    want_tail = tail.copy()
    del hits
    again, _ = ae.ae_search(idx, qs[:2], scheme, Hs[:2])
    assert again.size > 0 and np.array_equal(tail, want_tail)
    idx.close()


def test_bad_letters_rejected(small):
    wl, idx = small
    with pytest.raises(ae.AEError) as e:
        ae.ae_search(idx, [b"ACGTNACGT"], wl.scheme, [5])
    assert e.value.status == ae.AE_EINVAL
    with pytest.raises(ae.AEError) as e:
        ae.ae_search(idx, [b"ACGT"], wl.scheme, [0])
    assert e.value.status == ae.AE_EINVAL


def test_index_save_load_roundtrip(small, tmp_path):
    wl, idx = small
    p = tmp_path / "small.aeidx"
    ae.ae_index_save(idx, p)
    idx2 = ae.ae_index_load(p)
    assert ae.ae_index_info(idx2)["n"] == wl.n
    a, _ = ae.ae_search(idx, wl.queries, wl.scheme, wl.H)
    b, _ = ae.ae_search(idx2, wl.queries, wl.scheme, wl.H)
    assert_same(b, a, "reloaded index")
    idx2.close()
    raw = bytearray(p.read_bytes())
    raw[100] ^= 0xFF
    p.write_bytes(bytes(raw))
    with pytest.raises(ae.AEError) as e:
        ae.ae_index_load(p)
    assert e.value.status == ae.AE_EIO


def test_workspace_limit_splits_batches_without_changing_hits():
    # Caps below the uncapped workspace make the search split its batches; a cap
    # can also be too tight for the part that does not shrink with the batch
    # (the search's accumulated results), which must give AE_ENOMEM, never
    # different results.  At least one cap must succeed with a split.
    from workloads import dna_scale_text, dna_scale_query
    text = dna_scale_text(seed=61, n=2_000_000)
    q, _ = dna_scale_query(text, 30_000, np.random.default_rng(62), frac=0.05)
    idx = ae.ae_index_build(text, ae.AE_DNA)
    st = torch.cuda.Stream()
    base = dict(leaf_capacity=64)
    ae.ae_workspace_release(idx, st)
    want, wc = ae.ae_search(idx, [q], Scheme(), [22], options=ae.make_options(**base), stream=st)
    full, _ = ae.ae_workspace_info(idx, st)
    assert ae.ae_last_stats()["batch_splits"] == 0 and want.size > 0
    split_ok = 0
    for frac in (0.9, 0.8, 0.7, 0.6):
        ae.ae_workspace_release(idx, st)
        cap = int(full * frac)
        try:
            got, gc = ae.ae_search(idx, [q], Scheme(), [22], stream=st,
                                   options=ae.make_options(workspace_limit=cap, **base))
        except ae.AEError as e:
            assert e.status == ae.AE_ENOMEM, e
            continue
        used, _ = ae.ae_workspace_info(idx, st)
        assert used <= cap
        assert np.array_equal(wc, gc) and np.array_equal(want, got)
        split_ok += ae.ae_last_stats()["batch_splits"] >= 1
    assert split_ok >= 1
    ae.ae_workspace_release(idx, st)
    idx.close()
