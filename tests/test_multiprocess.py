"""N > 1 host logic on CPU ranks (gloo, world size 2): the LPT shard of a
batch is the same on every rank, disjoint, complete and balanced, and the
elapsed time reported is the max over ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2104_05782_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, costs, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    parts = shard.lpt_partition(costs, world)
    mine = parts[rank]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t = torch.tensor([float(10 * (rank + 1))], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put((gathered, parts, float(t.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_lpt_partition_properties():
    costs = [float((7 * i) % 13 + 1) ** 3 for i in range(100)]
    parts = shard.lpt_partition(costs, 4)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(100))
    ld = shard.loads(costs, parts)
    assert max(ld) <= (4.0 / 3.0) * max(sum(costs) / 4, max(costs))
    assert shard.lpt_partition(costs, 1) == [list(range(100))]
    with pytest.raises(ValueError):
        shard.lpt_partition(costs, 0)


def test_two_gloo_ranks_agree_on_the_shard_and_max_time():
    costs = [float(n) ** 3 for n in range(32, 512, 7)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, parts, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert gathered == parts                       # every rank computed the same partition
    assert sorted(gathered[0] + gathered[1]) == list(range(len(costs)))
    assert not set(gathered[0]) & set(gathered[1])
    assert tmax == 20.0                            # max over ranks
