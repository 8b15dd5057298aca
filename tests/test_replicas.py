"""Replica sharding of independent ACI products across ranks (CPU, gloo, world size 2).

One product does not shard (Algorithm 1 visits bonds in sequence and each pivot step needs a
global argmax), so N GPUs run independent products split by index with no data-path collective.
"""

import os

import pytest
import torch.multiprocessing as mp

from paper_2604_00037_gb300.replicas import shard


def test_shard_partitions_exactly():
    for n in range(0, 30):
        for world in range(1, 6):
            got = [list(shard(n, r, world)) for r in range(world)]
            flat = [i for g in got for i in g]
            assert flat == list(range(n))
            sizes = [len(g) for g in got]
            assert max(sizes) - min(sizes) <= 1 if n else True
    with pytest.raises(ValueError):
        shard(4, 2, 2)


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_2604_00037_gb300.replicas import gather_to_rank0, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = list(shard(7, rank, world))
    # each rank "processes" its products on the host (sum of indices stands in for the result)
    res = gather_to_rank0({"rank": rank, "items": mine, "sum": sum(mine)})
    if rank == 0:
        q.put(res)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_on_rank0():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    items = sorted(i for r in res for i in r["items"])
    assert items == list(range(7))
    assert sum(r["sum"] for r in res) == sum(range(7))
