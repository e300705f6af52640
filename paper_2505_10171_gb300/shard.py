"""Instance sharding for runs on several GPUs (one process per GPU).

The batched workloads are independent instances, so they shard without any
data-path collective: each rank steps its own subset in one context and the
per-instance results are gathered on rank 0 at the end.  A single large domain
is not decomposed (every rank would need a halo exchange per step); several
GPUs run replicas of it instead.
"""
from __future__ import annotations

import heapq


def shard_instances(sizes, world):
    """Assign instances to ranks, balancing the node counts: largest instance
    first to the least-loaded rank (ties to the lower rank).  Returns one sorted
    list of instance indices per rank; deterministic for given sizes."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda k: (-sizes[k], k))
    heap = [(0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for k in order:
        load, r = heapq.heappop(heap)
        out[r].append(k)
        heapq.heappush(heap, (load + sizes[k], r))
    return [sorted(v) for v in out]


def gather_to_rank0(local, dist, world):
    """Gather a {instance: result} dict of every rank on rank 0 (torch.distributed
    object collective; any backend).  Returns the merged dict on rank 0 and None
    elsewhere."""
    got = [None] * world if dist.get_rank() == 0 else None
    dist.gather_object(local, got, dst=0)
    if dist.get_rank() != 0:
        return None
    merged = {}
    for part in got:
        for k, v in part.items():
            if k in merged:
                raise RuntimeError(f"instance {k} reported by two ranks")
            merged[k] = v
    return merged


def run_shard(workloads, steps, precision, rank, world, stream=None):
    """Step this rank's share of a batch of workloads in one context and
    return {instance: (particle records, FP64 diagnostics)}."""
    from paper_2505_10171_gb300 import lbm
    mine = shard_instances([w["params"]["nx"] * w["params"]["ny"] * w["params"]["nz"] for w in workloads],
                           world)[rank]
    if not mine:
        return {}
    ctx = lbm.Context([workloads[k]["params"] for k in mine], precision, stream=stream)
    for j, k in enumerate(mine):
        if workloads[k].get("particles"):
            ctx.lbm_add_particles(workloads[k]["particles"], inst=j)
        ctx.lbm_init_fields(workloads[k]["phi"], inst=j)
    ctx.lbm_step(steps)
    out = {k: (ctx.lbm_particle_forces(j), ctx.lbm_diagnostics(j)) for j, k in enumerate(mine)}
    ctx.close()
    return out
