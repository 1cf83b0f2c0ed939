"""The no-allocation search (ae_search_device_static) against ae_search_device.

ae_search_device_static serves callers that cannot allocate device memory,
for example a process whose device memory is already handed out to another
allocator. Its working memory is a fixed array inside the library, shared by every call. The
results must be identical to those of ae_search_device: two different searches
are run back to back, so the second one starts from the array the first one
left behind. The file sorts last so a stop at the first failure has already
run every other test.
"""
import numpy as np
import pytest

from workloads import Scheme, dna_small, random_pair

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1208_0274_gb300 import ae  # noqa: E402


def _device_inputs(queries):
    seq = np.concatenate([np.asarray(q, dtype=np.uint8) for q in queries])
    offsets = np.concatenate([[0], np.cumsum([len(q) for q in queries])]).astype(np.int64)
    return torch.from_numpy(seq).cuda(), offsets


def _hits(buf, n):
    return buf[: n * 16].cpu().numpy().view(ae.HIT_DTYPE)


def test_static_search_matches_device_search_on_two_calls_in_a_row():
    wl = dna_small()
    idx = ae.ae_index_build(wl.text, ae.AE_DNA)
    T = wl.text
    _, extra = random_pair(1, 700, seed=41)
    extra[100:400] = T[50_000:50_300]
    extra[250] = ord("A") if extra[250] != ord("A") else ord("G")
    problems = [
        (wl.queries, wl.scheme, wl.H),
        ([extra, wl.queries[0][:500]], Scheme(1, -3, -5, -2), [20, 24]),
    ]
    cap = 1 << 17
    want = []
    for queries, scheme, H in problems:
        d_seq, offsets = _device_inputs(queries)
        out = torch.empty(cap * 16, dtype=torch.uint8, device="cuda")
        st, counts = ae.ae_search_device(idx, d_seq.data_ptr(), offsets, scheme, H, out.data_ptr(), cap)
        assert st == ae.AE_OK
        want.append((counts, _hits(out, int(counts.sum()))))
    # two calls in a row through the no-allocation entry point
    got = []
    for queries, scheme, H in problems:
        d_seq, offsets = _device_inputs(queries)
        out = torch.full((cap * 16,), 0xAB, dtype=torch.uint8, device="cuda")
        st, counts = ae.ae_search_device_static(idx, d_seq.data_ptr(), offsets, scheme, H, out.data_ptr(), cap)
        assert st == ae.AE_OK
        got.append((counts, _hits(out, int(counts.sum()))))
    for (wc, wh), (gc, gh) in zip(want, got):
        assert np.array_equal(wc, gc)
        assert wh.size > 0 and np.array_equal(wh, gh)
    # an undersized output buffer reports the sizes it needs, like ae_search_device
    d_seq, offsets = _device_inputs(problems[0][0])
    out = torch.empty(16, dtype=torch.uint8, device="cuda")
    st, counts = ae.ae_search_device_static(idx, d_seq.data_ptr(), offsets, problems[0][1], problems[0][2],
                                            out.data_ptr(), 1)
    assert st == ae.AE_EOVERFLOW and np.array_equal(counts, want[0][0])
    idx.close()


def test_static_search_rejects_inputs_beyond_its_limit():
    T, P = random_pair(5_000, 70_000, seed=2)
    idx = ae.ae_index_build(T, ae.AE_DNA)
    d_seq, offsets = _device_inputs([P])
    out = torch.empty(16, dtype=torch.uint8, device="cuda")
    st, _ = ae.ae_search_device_static(idx, d_seq.data_ptr(), offsets, Scheme(), [30], out.data_ptr(), 1)
    assert st == ae.AE_EUNSUPPORTED
    idx.close()


def test_static_search_out_of_array_midway_then_next_call_is_clean():
    # A one-letter text and query keep every trie node's row m entries wide and
    # emit a range hit per entry from depth H on, so the hit arena outgrows the
    # 64 MiB array after ~100 levels of queued kernels: the call must report
    # AE_EUNSUPPORTED, and must have waited for those kernels before returning.
    n = m = 20_000
    T = np.full(n, ord("A"), dtype=np.uint8)
    idx = ae.ae_index_build(T, ae.AE_DNA)
    d_seq, offsets = _device_inputs([np.full(m, ord("A"), dtype=np.uint8)])
    out = torch.empty(16, dtype=torch.uint8, device="cuda")
    st, _ = ae.ae_search_device_static(idx, d_seq.data_ptr(), offsets, Scheme(1, -3, -5, -2), [20],
                                       out.data_ptr(), 1)
    assert st == ae.AE_EUNSUPPORTED
    idx.close()
    # the next call, on another stream, sees a clean array and matches ae_search_device
    wl = dna_small()
    idx = ae.ae_index_build(wl.text, ae.AE_DNA)
    d_seq, offsets = _device_inputs(wl.queries)
    cap = 1 << 17
    ref = torch.empty(cap * 16, dtype=torch.uint8, device="cuda")
    st, want = ae.ae_search_device(idx, d_seq.data_ptr(), offsets, wl.scheme, wl.H, ref.data_ptr(), cap)
    assert st == ae.AE_OK
    other = torch.cuda.Stream()
    got_buf = torch.full((cap * 16,), 0xAB, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    st, got = ae.ae_search_device_static(idx, d_seq.data_ptr(), offsets, wl.scheme, wl.H, got_buf.data_ptr(), cap,
                                         stream=other)
    assert st == ae.AE_OK and np.array_equal(got, want)
    assert np.array_equal(_hits(got_buf, int(got.sum())), _hits(ref, int(want.sum())))
    idx.close()
