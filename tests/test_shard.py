"""Instance sharding across ranks (host logic of the multi-GPU path), run as
two gloo processes on the CPU: every instance lands on exactly one rank, the
node counts balance, and the per-instance results gather on rank 0."""
import os

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2505_10171_gb300 import shard
from paper_2505_10171_gb300 import workloads as W


def test_shard_balances_and_covers():
    sizes = [w["params"]["nx"] * w["params"]["ny"] * w["params"]["nz"] for w in W.cfg4()]
    for world in (1, 2, 3, 8):
        parts = shard.shard_instances(sizes, world)
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[k] for k in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)  # greedy bound
        assert parts == shard.shard_instances(sizes, world)  # deterministic
    with pytest.raises(ValueError):
        shard.shard_instances(sizes, 0)


def _worker(rank, world, port, sizes, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard.shard_instances(sizes, world)[rank]
    local = {k: (rank, sizes[k] * 0.5) for k in mine}
    merged = shard.gather_to_rank0(local, dist, world)
    if rank == 0:
        q.put(merged)
    dist.barrier()
    dist.destroy_process_group()


def test_gather_on_two_gloo_ranks():
    sizes = [w["params"]["nx"] * w["params"]["ny"] * w["params"]["nz"] for w in W.cfg4()[:11]]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert sorted(merged) == list(range(len(sizes)))
    parts = shard.shard_instances(sizes, 2)
    for k, (rank, v) in merged.items():
        assert k in parts[rank] and v == sizes[k] * 0.5
