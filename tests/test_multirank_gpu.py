"""A search split into parts of its forks, merged by the per-cell maximum.

* One process: the parts (ae_options.fork_parts / fork_part) of a multi-query
  search, for 2 and 3 parts, seeded and from the root, merged on the device by
  ae_hits_merge, equal the whole search (and the oracle) hit for hit, while no
  single part does.
* Two processes on the GPU (gloo for the host exchange; their kernels never
  wait on each other): multirank.split_search on rank 0 equals the whole
  search.
"""
import datetime
import os
import socket

import numpy as np
import pytest

import oracle
from workloads import PROTEIN, Scheme, protein, random_pair

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1208_0274_gb300 import ae, multirank  # noqa: E402

SCHEME = Scheme(1, -3, -5, -2)


def _problem(seed=5):
    rng = np.random.default_rng(seed)
    T, _ = random_pair(200_000, 1, seed=seed)
    qs = []
    for k in range(4):
        _, P = random_pair(1, int(rng.integers(300, 3_000)), seed=seed * 10 + k)
        for _ in range(2):
            L = int(rng.integers(40, 250))
            x, y = int(rng.integers(0, T.size - L)), int(rng.integers(0, P.size - L))
            P[y:y + L] = T[x:x + L]
            P[y + L // 2] = ord("A") if P[y + L // 2] != ord("A") else ord("C")
        qs.append(P)
    return T, qs, [18, 20, 22, 19]


def _merge_parts(idx, qs, scheme, Hs, parts, n_text, **opts):
    recs = []
    for part in range(parts):
        h, c = ae.ae_search(idx, qs, scheme, Hs, options=ae.make_options(fork_parts=parts, fork_part=part, **opts))
        recs.append(multirank.to_records(h, c))
    rec = np.concatenate(recs)
    return multirank.merge_on_device(rec, len(qs), n_text, max(q.size for q in qs))


@pytest.mark.parametrize("parts", [2, 3])
@pytest.mark.parametrize("seeded", [1, 0])
def test_fork_parts_merge_to_the_whole_search(parts, seeded):
    T, qs, Hs = _problem()
    idx = ae.ae_index_build(T, ae.AE_DNA)
    whole, wc = ae.ae_search(idx, qs, SCHEME, Hs, options=ae.make_options(qprefix_seed=seeded))
    merged, mc = _merge_parts(idx, qs, SCHEME, Hs, parts, T.size, qprefix_seed=seeded)
    assert np.array_equal(wc, mc) and np.array_equal(whole, merged)
    for k, (P, H) in enumerate(zip(qs[:2], Hs[:2])):
        oi, oj, os_ = oracle.sw_hits(T, P, SCHEME, H)
        part = np.split(merged, np.cumsum(mc)[:-1])[k]
        assert np.array_equal(part["text_end"], oi) and np.array_equal(part["score"], os_)
    one, _ = ae.ae_search(idx, qs, SCHEME, Hs, options=ae.make_options(fork_parts=parts, fork_part=0,
                                                                       qprefix_seed=seeded))
    assert not np.array_equal(one, whole)
    idx.close()


def test_fork_parts_protein_from_the_root():
    wl = protein(n=40_000, lengths=[400], per_length=3)
    idx = ae.ae_index_build(wl.text, ae.AE_PROTEIN)
    whole, wc = ae.ae_search(idx, wl.queries, wl.scheme, wl.H)
    merged, mc = _merge_parts(idx, wl.queries, wl.scheme, wl.H, 2, wl.text.size)
    assert whole.size > 0 and np.array_equal(wc, mc) and np.array_equal(whole, merged)
    idx.close()


def test_hits_merge_rejects_bad_arguments():
    st = ae.lib.ae_hits_merge(None, None, 5, 1, 10, 10, None, None, None, None)
    assert st == ae.AE_EINVAL


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    torch.cuda.set_device(0)
    T, qs, Hs = _problem(seed=9)
    idx = ae.ae_index_build(T, ae.AE_DNA)
    r = multirank.split_search(idx, qs, SCHEME, Hs, dist)
    out.put((rank, r))
    idx.close()
    dist.destroy_process_group()


def test_two_ranks_split_search_equals_whole_search():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=300) for _ in range(2)], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    hits, counts = res[0][1]
    assert res[1][1] is None
    T, qs, Hs = _problem(seed=9)
    idx = ae.ae_index_build(T, ae.AE_DNA)
    whole, wc = ae.ae_search(idx, qs, SCHEME, Hs)
    assert whole.size > 0 and np.array_equal(wc, counts) and np.array_equal(whole, hits)
    idx.close()
