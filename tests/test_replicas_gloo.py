"""Multi-process host logic of the benchmark on CPU (gloo, world size 2): the
batch's members are split into disjoint shards that cover it, and the timed
region is the slowest rank's."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_2204_07247_gb300 import inputs as I
    from paper_2204_07247_gb300 import replicas as R
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        names = [m.name for m in I.pfc_batch(sizes=(16, 32, 64), per_size=5).members]
        mine = R.shard(names, rank, world)
        allshards = [None] * world
        dist.all_gather_object(allshards, mine)
        slowest = R.max_over_ranks(1.0 + rank, dist)
        total = R.sum_over_ranks(len(mine), dist)
        q.put((rank, allshards, names, slowest, total))
    finally:
        dist.destroy_process_group()


def test_shards_cover_the_batch_and_time_is_the_max():
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, shards, names, slowest, total in out:
        flat = [n for s in shards for n in s]
        assert sorted(flat) == sorted(names) and len(set(flat)) == len(flat)
        assert slowest == 2.0 and total == len(names)
        # every shard keeps the mix of grid sizes
        for s in shards:
            assert {n.split("_")[1] for n in s} == {"16", "32", "64"}


def test_shard_rejects_bad_rank():
    from paper_2204_07247_gb300 import replicas as R
    with pytest.raises(ValueError):
        R.shard([1, 2], 2, 2)
