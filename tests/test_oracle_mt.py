"""The all-cores oracle (sw_hits_mt) against the one-thread oracle (sw_hits).

Both compute the full-matrix Gotoh Smith-Waterman of Section 2.1 with no
index and no filter; the threaded one cuts the query into column stripes that
run as a wavefront over blocks of text rows, handing each stripe's edge column
(V and F) to its right neighbour.  Its results must be the one-thread results,
bit for bit and in the same row-major order, for every scheme, thread count and
shape -- including stripes narrower than a thread count, text shorter than a
row block or not a multiple of it, and a window start row -- up to ~1e9 cells.
"""
import numpy as np
import pytest

import oracle
from workloads import BLOSUM62, PROTEIN, Scheme, random_pair, protein


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("threads", [1, 2, 3, 5, 8, 16])
def test_mt_matches_single_thread_dna(threads):
    T, P = random_pair(9_001, 700, seed=threads)
    P[100:400] = T[3_000:3_300]
    for sc, H in [(Scheme(1, -3, -5, -2), 12), (Scheme(2, -3, -4, -1), 20), (Scheme(1, -1, 0, -1), 9)]:
        want = oracle.sw_hits(T, P, sc, H)
        assert want[0].size > 100
        assert _same(want, oracle.sw_hits_mt(T, P, sc, H, threads=threads))


def test_mt_edge_shapes():
    sc = Scheme(1, -3, -5, -2)
    for n, m, threads in [(1, 1, 4), (255, 3, 8), (256, 7, 7), (257, 64, 3), (1_000, 2, 16), (3, 1_000, 9)]:
        T, P = random_pair(n, m, seed=n + m)
        m2 = min(n, m)
        P[:m2] = T[:m2]
        for H in (1, 3):
            assert _same(oracle.sw_hits(T, P, sc, H), oracle.sw_hits_mt(T, P, sc, H, threads=threads)), (n, m)


def test_mt_window_rows_and_protein():
    T, P = random_pair(20_000, 900, seed=9)
    P[200:700] = T[12_000:12_500]
    sc = Scheme(1, -3, -5, -2)
    assert _same(oracle.sw_hits(T, P, sc, 20, row_lo=11_000),
                 oracle.sw_hits_mt(T, P, sc, 20, row_lo=11_000, threads=6))
    wl = protein(n=30_000, lengths=[300], per_length=2)
    for q in wl.queries:
        want = oracle.sw_hits(wl.text, q, wl.scheme, 50, alphabet=PROTEIN)
        assert _same(want, oracle.sw_hits_mt(wl.text, q, wl.scheme, 50, alphabet=PROTEIN, threads=7))


def test_mt_billion_cells():
    # 1e9 cells: a 10 kbp query with two planted homologs against 100 kbp of text
    T, P = random_pair(100_000, 10_000, seed=77)
    P[1_000:2_500] = T[40_000:41_500]
    P[6_000:6_900] = T[90_000:90_900]
    sc = Scheme(1, -3, -5, -2)
    want = oracle.sw_hits(T, P, sc, 19)
    got = oracle.sw_hits_mt(T, P, sc, 19)
    assert want[0].size > 2_000 and _same(want, got)
