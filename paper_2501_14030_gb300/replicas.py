"""Whole-job rate of N independent replicas (one process per GPU).

The relaxation of one grid does not shard: on N GPUs every rank solves its
own copy (weak scaling) and the only cross-rank operations are the timing
barrier and this reduction, with no collective on the data path.
"""
from __future__ import annotations


def job_rate(local_seconds: float, local_units: float, dist=None, device=None):
    """(t_max, units, rate): the slowest rank's time, the units all ranks
    processed, and units / t_max.  `dist` is torch.distributed (initialised)
    or None for one process; `device` holds the reduction tensors (a CUDA
    device under NCCL, the CPU under gloo)."""
    if dist is None:
        return local_seconds, local_units, local_units / local_seconds
    import torch
    t = torch.tensor([local_seconds], dtype=torch.float64, device=device)
    u = torch.tensor([local_units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    t_max, units = float(t.item()), float(u.item())
    return t_max, units, units / t_max
