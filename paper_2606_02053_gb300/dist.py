"""Host-side logic for running on several GPUs of one node.

With N processes each rank evolves its own grid (replicas) or its own share
of a batched scan (independent instances: no collective touches the evolved
data), or holds one z-slab of a single grid (slab.py: the ghost-plane
exchange and the exponent reduction are the only collectives).

* ``shard_instances``: contiguous, balanced split of scan instances by their
  point count (greedy over ranks, deterministic).
* ``max_over_ranks`` / ``sum_over_ranks``: reductions of host scalars
  through torch.distributed (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

from typing import List, Sequence


def shard_instances(sizes: Sequence[int], world: int) -> List[List[int]]:
    """Indices of the instances each rank owns, balancing sum(sizes).

    Largest-first greedy assignment to the least-loaded rank; ties go to the
    lowest rank.  Every instance is owned by exactly one rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    load = [0] * world
    owned: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owned[r].append(i)
        load[r] += sizes[i]
    return [sorted(o) for o in owned]


def _reduce(value: float, op_name: str) -> float:
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    backend = dist.get_backend()
    device = "cuda" if backend == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op_name))
    return float(t.item())


def max_over_ranks(value: float) -> float:
    return _reduce(value, "MAX")


def sum_over_ranks(value: float) -> float:
    return _reduce(value, "SUM")
