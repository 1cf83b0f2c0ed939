"""The no-allocation search (ae_search_device_static) against ae_search_device.

ae_search_device_static serves callers that cannot allocate device memory,
for example code running while a CUDA stream is captured into a graph. Its
working memory is a fixed array inside the library, shared by every call. The
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
