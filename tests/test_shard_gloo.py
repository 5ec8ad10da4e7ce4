"""The N > 1 path on CPU: two gloo ranks shard the 512-system batch workload.

Each rank computes the partition on its own (no communication needed to agree
on it), the ranks exchange what they computed, and the test checks that they
agree, that every system is evaluated by exactly one rank, and that the
loads are balanced. The max-over-ranks reduction the benchmark applies to its
timings runs over the same process group.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = torch.distributed
mp = torch.multiprocessing


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2510_05961_gb300 import shard
    from paper_2510_05961_gb300 import workloads as W
    systems = W.batch_systems()
    parts, load = shard.shard(systems, world)
    mine = parts[rank]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    # the benchmark's timing rule: max over ranks
    t = torch.tensor([float(len(mine)) + 0.5 * rank])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    out[rank] = (parts, load, gathered, float(t.item()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_the_batch():
    from paper_2510_05961_gb300 import build
    build.build()
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    parts0, load0, gathered0, tmax0 = res[0]
    parts1, load1, gathered1, tmax1 = res[1]
    assert parts0 == parts1 and gathered0 == gathered1 == parts0
    allidx = sorted(parts0[0] + parts0[1])
    assert allidx == list(range(512))
    assert not set(parts0[0]) & set(parts0[1])
    assert max(load0) <= 1.02 * min(load0)
    assert tmax0 == tmax1 == max(len(parts0[0]), len(parts0[1]) + 0.5)


def test_shard_single_rank_and_many_ranks():
    from paper_2510_05961_gb300 import build, shard
    from paper_2510_05961_gb300 import workloads as W
    build.build()
    systems = W.batch_systems(nsys=40, seed=123)
    parts, load = shard.shard(systems, 1)
    assert parts == [list(range(40))]
    parts, load = shard.shard(systems, 8)
    assert sorted(i for p in parts for i in p) == list(range(40))
    costs = [shard.system_cost(shard.L.load(), s) for s in systems]
    # longest-processing-time bound: max load <= mean load + largest single cost
    assert max(load) <= sum(costs) / 8 + max(costs)
