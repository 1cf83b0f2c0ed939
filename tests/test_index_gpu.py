"""The device suffix array (prefix doubling) and the index built from it,
against the oracle's suffix array (Section 2.3: the suffixes in lexicographic
order, the sentinel smallest).  Integer results, compared exactly."""
import os

import numpy as np
import pytest

import oracle
from workloads import DNA, PROTEIN, iid_text

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1208_0274_gb300 import ae  # noqa: E402


def device_sa(codes, sigma, reversed_=False):
    c = np.ascontiguousarray(codes, dtype=np.uint8)
    d_codes = torch.from_numpy(c).cuda() if c.size else torch.empty(1, dtype=torch.uint8, device="cuda")
    d_sa = torch.empty(c.size + 1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    ae.ae_suffix_array_device(d_codes.data_ptr(), c.size, sigma, d_sa.data_ptr(), reversed=reversed_)
    return d_sa.cpu().numpy()


def _cases():
    rng = np.random.default_rng(2024)
    yield "empty", np.zeros(0, np.uint8), 4
    yield "one", np.array([3], np.uint8), 4
    yield "seven", rng.integers(0, 4, 7).astype(np.uint8), 4
    # several radix tiles (2,048 keys each) and a ragged tail
    yield "iid_100003", rng.integers(0, 4, 100_003).astype(np.uint8), 4
    yield "binary", rng.integers(0, 2, 30_001).astype(np.uint8), 2
    yield "protein", rng.integers(0, 20, 50_000).astype(np.uint8), 20
    # long repeats: one doubling round per factor of two of the longest common prefix
    yield "period7", np.tile(rng.integers(0, 4, 7), 3000)[:20_000].astype(np.uint8), 4
    yield "one_letter", np.zeros(20_000, np.uint8), 4
    yield "copies", np.tile(rng.integers(0, 4, 4_093), 5).astype(np.uint8), 4


@pytest.mark.parametrize("name,codes,sigma", list(_cases()), ids=[c[0] for c in _cases()])
@pytest.mark.parametrize("reversed_", [False, True])
def test_device_suffix_array_matches_oracle(name, codes, sigma, reversed_):
    want = oracle.suffix_array(codes[::-1].copy() if reversed_ else codes)
    got = device_sa(codes, sigma, reversed_)
    assert np.array_equal(got, want), name


def test_device_suffix_array_ten_million_letters():
    codes = np.random.default_rng(5).integers(0, 4, 10_000_000).astype(np.uint8)
    assert np.array_equal(device_sa(codes, 4, True), oracle.suffix_array(codes[::-1].copy()))


def test_device_suffix_array_rejects_codes_outside_the_alphabet():
    codes = np.random.default_rng(1).integers(0, 4, 5_000).astype(np.uint8)
    codes[1234] = 4
    with pytest.raises(ae.AEError) as e:
        device_sa(codes, 4)
    assert e.value.status == ae.AE_EINVAL
    # the device is still usable
    ok = np.random.default_rng(2).integers(0, 4, 999).astype(np.uint8)
    assert np.array_equal(device_sa(ok, 4), oracle.suffix_array(ok))


@pytest.mark.parametrize("alphabet", ["dna", "protein"])
def test_index_build_text_end_array_matches_oracle(tmp_path, alphabet):
    """ae_index_build's text-end array is n - 1 - SA of the reversed text
    (Section 5 (1)-(2)), read back from the saved index file, whose last
    fields are the text-end array, the text and an 8-byte checksum."""
    rng = np.random.default_rng(11)
    if alphabet == "dna":
        letters, code = DNA, ae.AE_DNA
        text = iid_text(300_001, DNA, [0.3, 0.2, 0.2, 0.3], rng)
    else:
        letters, code = PROTEIN, ae.AE_PROTEIN
        text = iid_text(120_000, PROTEIN, [1.0 / 20] * 20, rng)
    idx = ae.ae_index_build(text, code)
    path = os.path.join(tmp_path, "i.aeidx")
    ae.ae_index_save(idx, path)
    idx.close()
    raw = open(path, "rb").read()
    n = text.size
    tend = np.frombuffer(raw[len(raw) - 8 - n - 4 * (n + 1): len(raw) - 8 - n], dtype=np.int32)
    sa = np.where(tend >= 0, n - 1 - tend, n)
    codes = oracle.encode(text, letters)
    assert np.array_equal(sa, oracle.suffix_array(codes[::-1].copy()))
