"""Work split across ranks (one process per GPU).

The step has no exchange between independent problems: a batch of
instances is partitioned across ranks by particle count with no collective
on the data path, and a single workload runs as one replica per rank.  The
only collectives are the bench's timing reductions (max of the per-rank
times, sum of the particle-steps).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple


def partition_instances(counts: Sequence[int], world: int) -> List[List[int]]:
    """Instances per rank, balanced by particle count: largest first, each
    to the currently lightest rank (ties to the lower rank).  Every instance
    is assigned to exactly one rank; a rank may get none when there are
    fewer instances than ranks."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    order = sorted(range(len(counts)), key=lambda q: (-int(counts[q]), q))
    for q in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(q)
        load[r] += int(counts[q])
    return [sorted(p) for p in parts]


def shard_cases(cases: Sequence, world: int, rank: int) -> list:
    """This rank's instances of a batch (partition_instances by particle
    count), in their batch order."""
    mine = partition_instances([int(c.n) for c in cases], world)[rank]
    return [cases[q] for q in mine]


def combine_timing(ms: float, particle_steps: float, dist=None) -> Tuple[float, float]:
    """Whole-job timing: the slowest rank's time and the particle-steps of
    all ranks (torch.distributed when dist is given, else this rank's)."""
    if dist is None:
        return ms, particle_steps
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    mx = torch.tensor([ms], dtype=torch.float64, device=dev)
    tot = torch.tensor([particle_steps], dtype=torch.float64, device=dev)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    return float(mx.item()), float(tot.item())
