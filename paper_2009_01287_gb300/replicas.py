"""Multi-GPU form: independent replicas, one per rank.

A single hp-DG problem is not sharded (no halo exchange, no distributed AMG);
with N ranks every rank solves its own replica and the job's throughput is the
sum over ranks.  Timing follows the slowest rank: the per-rank seconds are
reduced with MAX over the process group (NCCL on GPUs, gloo on CPUs), the
DOF-iterations with SUM.  There is no collective on the solver's data path.
"""
from __future__ import annotations

from typing import Sequence, Tuple


def aggregate(seconds: Sequence[float], dof_iters: float, device=None) -> Tuple[list, float]:
    """Return ([max over ranks of each entry of `seconds`], sum of dof_iters).
    Works on a single process (no process group) as the identity."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(seconds), float(dof_iters)
    t = torch.tensor(list(seconds), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    d = torch.tensor([float(dof_iters)], dtype=torch.float64, device=device)
    dist.all_reduce(d, op=dist.ReduceOp.SUM)
    return [float(v) for v in t], float(d[0])
