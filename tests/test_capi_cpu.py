"""Host-side checks of the C ABI that need no GPU: the library loads and
exports every declared symbol, the host suffix array (index build, Section
2.3 and Section 5), the planning helpers (Eq. 1, Eq. 2) and argument errors
that are rejected before any device work."""
import os
import re

import numpy as np
import pytest

from paper_1208_0274_gb300 import ae
from workloads import Scheme, random_pair, iid_text, PROTEIN

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_every_declared_symbol_is_exported():
    inc = os.path.join(ROOT, "include")
    declared = set()
    for h in sorted(os.listdir(inc)):
        if h.endswith(".h"):
            declared |= set(re.findall(r"\b(ae_[a-z0-9_]+)\s*\(", open(os.path.join(inc, h)).read()))
    assert {"ae_index_build", "ae_search", "ae_search_device", "ae_mlp_forward", "ae_int_peak"} <= declared
    for name in declared:
        assert hasattr(ae.lib, name), name


def _naive_sa(codes):
    n = len(codes)
    s = list(codes) + [-1]
    return sorted(range(n + 1), key=lambda k: s[k:])


def test_suffix_array_paper_example_forward():
    # Section 2.3: SA of GCTAGC$ is {7, 4, 6, 2, 5, 1, 3} (1-based starts)
    sa = ae.ae_suffix_array(ae.encode_codes(b"GCTAGC"), 4)
    assert list(sa + 1) == [7, 4, 6, 2, 5, 1, 3]


def test_suffix_array_paper_example_reversed():
    # Section 5 (2): T^-1 of GCTAGC with positions kept: SA[0..6] =
    # {0, 4, 2, 6, 1, 5, 3}; CG (reversed GC) has range [2, 3] whose entries
    # are the 1-based end positions 2 and 6 of GC in T.
    t = ae.encode_codes(b"GCTAGC")
    rev = t[::-1].copy()
    sa = ae.ae_suffix_array(rev, 4)
    n = t.size
    labels = [n - k for k in sa]           # position label of the suffix's first letter
    assert labels == [0, 4, 2, 6, 1, 5, 3]
    cg = [h for h in range(n + 1) if list(rev[sa[h]:sa[h] + 2]) == [1, 2]]
    assert cg == [2, 3] and sorted(labels[h] for h in cg) == [2, 6]


@pytest.mark.parametrize("seed", range(6))
def test_suffix_array_matches_naive(seed):
    rng = np.random.default_rng(seed)
    for sigma, n in [(4, 1), (4, 2), (4, 57), (2, 300), (4, 1000), (20, 500)]:
        codes = rng.integers(0, sigma, size=n).astype(np.uint8)
        if seed % 2:                         # repetitive inputs exercise SA-IS recursion
            codes = np.tile(codes[: max(1, n // 7)], 8)[:n]
        sa = ae.ae_suffix_array(codes, sigma)
        assert list(sa) == _naive_sa(codes.tolist())


def test_plan_eq1_eq2():
    s = Scheme(1, -3, -5, -2)
    q, d0, L = ae.ae_plan(5, s, 3)
    assert (q, L) == (4, 5)                 # Section 3.1.1 example (Eq. 1) and Eq. 2
    assert d0 == 2                          # below ceil(H / s_a) = 3
    q, d0, L = ae.ae_plan(1000, s, 30)
    assert (q, d0, L) == (4, 3, 1482)
    q, d0, L = ae.ae_plan(100, Scheme(gap_open=-11, gap_extend=-1, matrix=np.eye(20, dtype=np.int8) * 5 - 1),
                          50, alphabet=ae.AE_PROTEIN)
    assert (q, d0) == (0, 0)


def test_argument_errors_without_device():
    with pytest.raises(ae.AEError) as e:
        ae.ae_index_build(b"", ae.AE_DNA)
    assert e.value.status == ae.AE_EINVAL
    with pytest.raises(ae.AEError) as e:
        ae.ae_index_build(b"ACGTN", ae.AE_DNA)
    assert e.value.status == ae.AE_EINVAL
    with pytest.raises(ae.AEError) as e:
        ae.ae_index_build(b"ACGT", 7)
    assert e.value.status == ae.AE_EINVAL
    with pytest.raises(ae.AEError) as e:
        ae.ae_plan(10, Scheme(1, 2, -5, -2), 5)       # mismatch must be negative
    assert e.value.status == ae.AE_EINVAL
    with pytest.raises(ae.AEError) as e:
        ae.ae_plan(10, Scheme(1, -3, -5, 0), 5)       # gap extension must be negative
    assert e.value.status == ae.AE_EINVAL
    assert ae.strerror(ae.AE_EOVERFLOW) == "output buffer too small"


def test_options_default():
    # the defaults the header lists
    o = ae.ae_options_default()
    want = dict(qprefix_seed=1, leaf_segment=0, item_columns=1 << 24, batch_columns=1 << 20, leaf_capacity=4096,
                profile=0, leaf_delay=8, int16_limit=32000, tier_stats=0, workspace_limit=0, general_rows=0,
                qprefix_domination=1, row_layout=0, fork_parts=1, fork_part=0, leaf_wide_rows=128)
    assert {k: getattr(o, k) for k in want} == want
    assert not o.hint_hits


@pytest.mark.parametrize("kind", ["iid", "period5", "blocks", "protein"])
def test_host_suffix_array_matches_oracle_at_size(kind):
    import oracle
    rng = np.random.default_rng(31)
    sigma = 20 if kind == "protein" else 4
    if kind == "period5":
        codes = np.tile(rng.integers(0, 4, 5), 20_000).astype(np.uint8)
    elif kind == "blocks":
        codes = np.tile(rng.integers(0, 4, 3_001), 30).astype(np.uint8)
    else:
        codes = rng.integers(0, sigma, 200_003).astype(np.uint8)
    assert np.array_equal(ae.ae_suffix_array(codes, sigma), oracle.suffix_array(codes))


def test_device_suffix_array_argument_errors_without_device():
    # rejected before any device work: bad sigma, missing pointers, too long
    for args, want in [((1, 10, 0, 0, 1), ae.AE_EINVAL), ((1, 10, 4, 0, 0), ae.AE_EINVAL),
                       ((0, 10, 4, 0, 1), ae.AE_EINVAL), ((1, -1, 4, 0, 1), ae.AE_EINVAL),
                       ((1, 10, 256, 0, 1), ae.AE_EINVAL), ((1, 1 << 31, 4, 0, 1), ae.AE_EUNSUPPORTED)]:
        d_codes, n, sigma, rev, d_sa = args
        assert ae.lib.ae_suffix_array_device(d_codes or None, n, sigma, rev, d_sa or None, None) == want


def test_collection_build_rejects_bad_arguments():
    import ctypes
    t = np.frombuffer(b"ACGTACGT", dtype=np.uint8)
    out = ctypes.c_void_p(0)
    for starts in ([1, 4], [0, 5, 3], [0, 9]):
        s = np.asarray(starts, dtype=np.int64)
        st = ae.lib.ae_index_build_collection(t.ctypes.data, t.size, s.ctypes.data, s.size, ae.AE_DNA,
                                              ctypes.byref(out))
        assert st == ae.AE_EINVAL, starts
    s = np.asarray([0], dtype=np.int64)
    assert ae.lib.ae_index_build_collection(t.ctypes.data, 0, s.ctypes.data, 1, ae.AE_DNA,
                                            ctypes.byref(out)) == ae.AE_EINVAL
    bad = np.frombuffer(b"ACGNACGT", dtype=np.uint8)
    assert ae.lib.ae_index_build_collection(bad.ctypes.data, bad.size, s.ctypes.data, 1, ae.AE_DNA,
                                            ctypes.byref(out)) == ae.AE_EINVAL

