"""The N-rank path on CPU: two gloo ranks, each reducing its own share of the
units with no exchange on the data path, then combining time (max) and
interactions (sum) as the benchmark does (paper_1404_0076_gb300/shard.py).
The reductions here are the oracle's; the host logic is the product's."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import workloads as W
from paper_1404_0076_gb300.shard import combine, partition, rank_seed
from tests import oracle_runner


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, nets, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = [nets[i] for i in partition(len(nets), rank, world)]
    res = oracle_runner.run(W.ARITH_RULES, mine, quiet=True)
    ints = sum(r["interactions"] for r in res)
    seconds = 1.0 + rank          # a stand-in for this rank's device time
    out[rank] = (list(partition(len(nets), rank, world)), ints, combine(seconds, ints, dist))
    dist.barrier()
    dist.destroy_process_group()


def test_partition_covers_every_unit_once():
    for n in (0, 1, 7, 64, 1001):
        for world in (1, 2, 3, 8):
            got = [i for r in range(world) for i in partition(n, r, world)]
            assert got == list(range(n))
            sizes = [len(partition(n, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        partition(4, 2, 2)


def test_rank_seeds_differ_and_keep_the_shape():
    a = W.config0(seed=rank_seed(W.SEED_BASE, 0))
    b = W.config0(seed=rank_seed(W.SEED_BASE, 1))
    assert len(a.nets) == len(b.nets) and a.params != b.params
    assert rank_seed(W.SEED_BASE, 0) == W.SEED_BASE


def test_two_gloo_ranks_shard_without_exchange():
    oracle_runner.build()
    nets = W.config0().nets[:96]
    whole = sum(r["interactions"] for r in oracle_runner.run(W.ARITH_RULES, nets, quiet=True))
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, nets, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    assert sorted(i for r in res.values() for i in r[0]) == list(range(len(nets)))
    assert res[0][1] + res[1][1] == whole
    for r in (0, 1):
        assert res[r][2] == (2.0, whole)    # max time, summed interactions, on every rank
