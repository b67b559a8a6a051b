"""Multi-rank logic of the batched path on the CPU (gloo, world size 2): every
matrix lands on exactly one rank, the shards balance, and the max-over-ranks
timing reduction the benchmark uses behaves."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    from paper_1710_10989_gb300 import sharding, workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ns, _ = W.batch_spec(count=4000)
    mine = sharding.shard_indices(ns, rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put((gathered, float(t.item()), [int(n) for n in ns]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_cover_the_batch_once():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, tmax, ns = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    a, b = set(gathered[0]), set(gathered[1])
    assert not (a & b) and (a | b) == set(range(len(ns)))
    ca = sum(ns[i] ** 3 for i in a)
    cb = sum(ns[i] ** 3 for i in b)
    assert abs(ca - cb) / max(ca, cb) < 0.01
    assert tmax == 2.0


def test_shards_single_process():
    from paper_1710_10989_gb300 import sharding
    sizes = [256, 8, 64, 256, 128, 16, 200]
    shards = [sharding.shard_indices(sizes, r, 3) for r in range(3)]
    assert sorted(i for s in shards for i in s) == list(range(len(sizes)))
    assert sharding.shard_indices(sizes, 0, 1) == sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    with pytest.raises(ValueError):
        sharding.shard_indices(sizes, 3, 3)
