"""Image sharding across ranks: the LPT planner, and the multi-process path
(gloo, world size 2, on CPU): every rank derives the same plan, the shards
partition the batch, and the job time is the maximum over ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2204_07921_gb300 import shard


def test_lpt_partitions_and_balances():
    import synth
    items = synth.uneven_batch(64)
    costs = [shard.image_cost(*it.image.f.shape) for it in items]
    for world in (1, 2, 3, 4, 8):
        parts = shard.plan_lpt(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(64))
        loads = [sum(costs[i] for i in p) for p in parts]
        lower = max(max(costs), sum(costs) / world)     # no plan beats this
        assert max(loads) <= 4 / 3 * lower + 1e-9


def test_lpt_small_cases():
    assert shard.plan_lpt([5, 4, 3, 3], 2) == [[0, 3], [1, 2]]
    assert shard.plan_lpt([1.0], 3) == [[0], [], []]
    with pytest.raises(ValueError):
        shard.plan_lpt([1.0], 0)


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import synth
    items = synth.uneven_batch(16, sides=(128, 256, 512))
    costs = [shard.image_cost(*it.image.f.shape) for it in items]
    mine = shard.my_share(costs, rank, world)
    # gather every rank's shard and its (fake) time; the job time is the max
    shards = [None] * world
    dist.all_gather_object(shards, mine)
    t = torch.tensor([1.0 + rank], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    out[rank] = (shards, float(t.item()))
    dist.destroy_process_group()


def test_two_rank_gloo_sharding():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (s0, t0), (s1, t1) = out[0], out[1]
    assert s0 == s1                                     # same plan everywhere
    assert sorted(s0[0] + s0[1]) == list(range(16))     # a partition
    assert not set(s0[0]) & set(s0[1])
    assert t0 == t1 == 2.0                              # max over ranks
