"""Several GPUs: independent refinement instances, one per rank.

Refining one mesh on several GPUs would need the regions that cross a partition
boundary exchanged every round (Sec. 2's rounds have a global select step).
The per-round path therefore does not shard, and N GPUs run N independent
instances (replicas) of the workload, each with its own seed. The only
cross-rank step is the host-side reduction of the measurement: time is the
maximum over ranks and work is the sum. No collective touches the mesh.
"""
from __future__ import annotations

# Seeds of different ranks' instances are this far apart, so no two ranks build
# the same point set.
SEED_STRIDE = 1000


def instance_seed(seed: int, rank: int) -> int:
    """Seed of rank `rank`'s instance of a workload whose base seed is `seed`."""
    return seed + SEED_STRIDE * rank


def reduce_measurement(times, work, world: int, device="cpu"):
    """(max over ranks of each of `times`, sum over ranks of each of `work`).

    A collective call: every rank of the default process group must make it with
    lists of the same lengths. `device` is where the reduction tensors live (the
    rank's GPU under NCCL, "cpu" under gloo). With world <= 1 the inputs come
    back unchanged.
    """
    times = [float(t) for t in times]
    work = [float(w) for w in work]
    if world <= 1:
        return times, work
    import torch
    import torch.distributed as dist
    mx = torch.tensor(times, dtype=torch.float64, device=device)
    sm = torch.tensor(work, dtype=torch.float64, device=device)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return [float(v) for v in mx.cpu()], [float(v) for v in sm.cpu()]
