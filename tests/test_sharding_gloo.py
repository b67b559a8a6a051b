"""Multi-rank logic of the batched path on the CPU (gloo, world size 2): every
matrix lands on exactly one rank, the shards balance on the cost N^3 (pi_m + s)
(products of the theta rule's (m, s), Table 3), also for a norm-skewed batch,
and the max-over-ranks timing reduction the benchmark uses behaves."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


PI = {1: 0, 2: 1, 4: 2, 8: 3, 12: 4, 18: 5}   # Table 3: products of T_m in the paper's scheme


def products_of(norms):
    """pi_m + s of the theta rule's (m, s) for each norm (the oracle's selection)."""
    from oracle import oracle as O
    out = []
    for v in norms:
        m, s = O.select(float(v), "new")
        out.append(PI[m] + s)
    return out


def skewed_spec(count=600):
    """Sizes of the batched workload with 1-norms that grow with N: the largest
    matrices also need the most products, the case an N^3-only cost misjudges."""
    import numpy as np
    from paper_1710_10989_gb300 import workloads as W
    ns, _ = W.batch_spec(count=count)
    rng = np.random.default_rng(3)
    norms = np.where(rng.random(count) < 0.5, 1e-3, 1e2) * (ns / 256.0) ** 2
    return ns, norms


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    from paper_1710_10989_gb300 import sharding, workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = {}
    for name, (ns, norms) in (("uniform", W.batch_spec(count=4000)), ("skewed", skewed_spec())):
        prods = products_of(norms)
        mine = sharding.shard_indices(ns, rank, world, prods)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        res[name] = (gathered, [int(n) for n in ns], prods)
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put((res, float(t.item())))
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
    res, tmax = q.get(timeout=180)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for name, (gathered, ns, prods) in res.items():
        a, b = set(gathered[0]), set(gathered[1])
        assert not (a & b) and (a | b) == set(range(len(ns))), name
        ca = sum(ns[i] ** 3 * prods[i] for i in a)
        cb = sum(ns[i] ** 3 * prods[i] for i in b)
        assert abs(ca - cb) / max(ca, cb) < 0.01, name
    assert tmax == 2.0


def test_product_count_matters_for_skewed_norms():
    """On the norm-skewed batch, shards balanced on N^3 alone are off by more
    than the (pi_m + s)-aware ones, measured in products x N^3."""
    from paper_1710_10989_gb300 import sharding
    ns, norms = skewed_spec()
    prods = products_of(norms)
    assert min(prods) <= 3 and max(prods) >= 12

    def imbalance(assign_prods):
        loads = []
        for r in range(4):
            idx = sharding.shard_indices(ns, r, 4, assign_prods)
            loads.append(sum(int(ns[i]) ** 3 * prods[i] for i in idx))
        return max(loads) / (sum(loads) / len(loads)) - 1.0

    aware, blind = imbalance(prods), imbalance(None)
    assert aware < 0.01
    assert blind > 2 * aware
    assert sum(sharding.shard_costs(ns, 4, prods)) == sum(int(n) ** 3 * p for n, p in zip(ns, prods))


def test_shards_single_process():
    from paper_1710_10989_gb300 import sharding
    sizes = [256, 8, 64, 256, 128, 16, 200]
    shards = [sharding.shard_indices(sizes, r, 3) for r in range(3)]
    assert sorted(i for s in shards for i in s) == list(range(len(sizes)))
    assert sharding.shard_indices(sizes, 0, 1) == sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    with pytest.raises(ValueError):
        sharding.shard_indices(sizes, 3, 3)
