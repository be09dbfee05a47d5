"""Multi-GPU runs as independent replicas (weak scaling).

The product y = A x has no exchange step once each GPU holds its own matrix, so
N GPUs run N independent replicas and no collective touches the data path.
The only collective is this end-of-run reduction of the timing: whole-job
throughput = units processed by all ranks / the slowest rank's time.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def aggregate(local_units: float, local_seconds: float, device=None):
    """(total_units, max_seconds, units_per_second) over all ranks.

    Without an initialised process group this is the single-rank identity.
    `device` must be a CUDA device for the NCCL backend; gloo works on CPU.
    """
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(local_units), float(local_seconds), float(local_units) / float(local_seconds)
    dev = device if device is not None else torch.device("cpu")
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=dev)
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total, tmax = float(u.item()), float(t.item())
    return total, tmax, total / tmax
