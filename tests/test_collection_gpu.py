"""Collections (Section 2.3): several sequences searched as one indexed text.

The oracle of a collection is its definition: the results of the plain
full-matrix Smith-Waterman of the query against each sequence on its own, with
each sequence's text positions moved to where the sequence starts in the
concatenation.  The GPU search of the collection index must equal that union
hit for hit, so no alignment may run across a sequence boundary -- which a
query planted across a boundary would do in a plain index of the
concatenation, as the test also shows.
"""
import os
import tempfile

import numpy as np
import pytest

import oracle
from workloads import DNA, PROTEIN, Scheme, iid_text, random_pair

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1208_0274_gb300 import ae  # noqa: E402


def _oracle_collection(seqs, P, scheme, H, alphabet=DNA):
    rows = []
    off = 0
    for s in seqs:
        if s.size:
            oi, oj, os_ = oracle.sw_hits(s, P, scheme, H, alphabet=alphabet)
            rows.append((oi + off, oj, os_))
        off += s.size
    w = np.zeros(sum(r[0].size for r in rows), dtype=ae.HIT_DTYPE)
    if w.size:
        w["text_end"] = np.concatenate([r[0] for r in rows])
        w["query_end"] = np.concatenate([r[1] for r in rows])
        w["score"] = np.concatenate([r[2] for r in rows])
    return np.sort(w, order=["text_end", "query_end"])


def _collection(rng, lengths):
    return [iid_text(int(L), DNA, [0.25] * 4, rng) for L in lengths]


def test_dna_collection_matches_per_sequence_oracle():
    rng = np.random.default_rng(4)
    seqs = _collection(rng, [3_000, 1, 0, 700, 5_000, 64, 2_500, 63, 4_000])
    cat = np.concatenate(seqs)
    starts = np.concatenate([[0], np.cumsum([s.size for s in seqs])[:-1]])
    qs = []
    # a query across the boundary of sequences 0 and 3 (sequence 1 is one letter,
    # 2 is empty), one across 4 and 5 and into 6, one inside sequence 8
    q0 = np.concatenate([seqs[0][-120:], seqs[1], seqs[3][:150]])
    q1 = np.concatenate([iid_text(40, DNA, [0.25] * 4, rng), seqs[4][-90:], seqs[5], seqs[6][:80]])
    q2 = seqs[8][1_000:1_400].copy()
    q2[200] = ord("A") if q2[200] != ord("A") else ord("T")
    qs = [q0, q1, q2]
    scheme = Scheme(1, -3, -5, -2)
    Hs = [18, 20, 25]
    idx = ae.ae_index_build_collection(seqs, ae.AE_DNA)
    assert ae.ae_index_info(idx)["n"] == cat.size
    plain = ae.ae_index_build(cat, ae.AE_DNA)
    for opts in (dict(), dict(general_rows=1), dict(leaf_delay=0), dict(leaf_delay=14, qprefix_seed=0)):
        hits, counts = ae.ae_search(idx, qs, scheme, Hs, options=ae.make_options(**opts))
        parts = np.split(hits, np.cumsum(counts)[:-1])
        for k, (P, H) in enumerate(zip(qs, Hs)):
            want = _oracle_collection(seqs, P, scheme, H)
            assert want.size > 0
            assert np.array_equal(parts[k], want), (opts, k, parts[k].size, want.size)
    # the plain index of the concatenation finds alignments across the boundaries
    ph, pc = ae.ae_search(plain, qs[:2], scheme, Hs[:2])
    assert pc[0] > counts[0] and pc[1] > counts[1]
    assert int(ph["score"].max()) > int(hits["score"][: counts[0] + counts[1]].max())
    # save / load keeps the collection
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "c.aeidx")
        ae.ae_index_save(idx, path)
        idx2 = ae.ae_index_load(path)
        h2, c2 = ae.ae_search(idx2, qs, scheme, Hs)
        assert np.array_equal(h2, hits) and np.array_equal(c2, counts)
        idx2.close()
    idx.close()
    plain.close()


def test_one_sequence_collection_equals_plain_index():
    T, P = random_pair(20_000, 800, seed=8)
    P[100:600] = T[7_000:7_500]
    scheme = Scheme(1, -3, -5, -2)
    a = ae.ae_index_build_collection([T], ae.AE_DNA)
    b = ae.ae_index_build(T, ae.AE_DNA)
    ha, ca = ae.ae_search(a, [P], scheme, [20])
    hb, cb = ae.ae_search(b, [P], scheme, [20])
    assert np.array_equal(ha, hb) and ha.size > 0
    a.close()
    b.close()


def test_protein_collection_matches_per_sequence_oracle():
    rng = np.random.default_rng(9)
    from workloads import PROTEIN_BG, protein
    wl = protein(n=30_000, lengths=[300], per_length=1)
    seqs = [iid_text(int(L), PROTEIN, PROTEIN_BG, rng) for L in (4_000, 2, 6_000, 900)]
    P = np.concatenate([seqs[0][-80:], seqs[1], seqs[2][:100]])
    idx = ae.ae_index_build_collection(seqs, ae.AE_PROTEIN)
    hits, counts = ae.ae_search(idx, [P], wl.scheme, [45])
    want = _oracle_collection(seqs, P, wl.scheme, 45, alphabet=PROTEIN)
    assert want.size > 0 and np.array_equal(hits, want)
    idx.close()
