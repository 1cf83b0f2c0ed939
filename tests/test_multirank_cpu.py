"""The N > 1 host path of bench.py on CPU ranks (gloo, world size 2): queries
are sharded without overlap or loss, and the job time is the maximum and the
work the sum over ranks, as the bench reports them."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, n_items, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = bench.shard(n_items, rank, world)
    # each rank "works" for a time that depends on its shard
    ms = 100.0 + 10.0 * rank
    units = sum(1000 + k for k in mine)
    tot_ms, tot_units = bench.job_totals(ms, units, dist, device="cpu")
    out.put((rank, mine, tot_ms, tot_units))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_aggregate():
    world, n_items = 2, 25
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, n_items, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    shards = [r[1] for r in res]
    assert sorted(k for sh in shards for k in sh) == list(range(n_items))     # a partition
    assert all(set(a).isdisjoint(b) for a in shards for b in shards if a is not b)
    want_units = sum(1000 + k for k in range(n_items))
    for _, _, tot_ms, tot_units in res:
        assert tot_ms == 110.0 and tot_units == want_units          # max time, summed work


def test_single_rank_totals_are_local():
    assert bench.job_totals(12.5, 7) == (12.5, 7.0)
    assert bench.shard(5, 0, 1) == [0, 1, 2, 3, 4]
