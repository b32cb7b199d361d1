"""Independent replicas on several GPUs: the only cross-rank steps of a run.

The update does not shard (a lattice fits one GPU many times over), so N
GPUs run N independent replicas.  Ranks meet only at a barrier around the
timed region and at the end, where the slowest rank's time and the sum of
the units processed give the whole-job throughput.  Launched by torchrun
(RANK / LOCAL_RANK / WORLD_SIZE / MASTER_* in the environment); the backend
is NCCL on GPUs and gloo elsewhere.
"""
from __future__ import annotations

import os
from typing import Tuple


def world() -> Tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment (1, 0, 0 without one)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str, device=None) -> None:
    import torch.distributed as dist

    if world()[0] > 1 and not dist.is_initialized():
        if backend == "nccl":
            dist.init_process_group("nccl", device_id=device)
        else:
            dist.init_process_group(backend)


def barrier() -> None:
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def combine(ms: float, units: float, device=None) -> Tuple[float, float]:
    """(slowest rank's time, units summed over ranks); the identity on one rank."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return ms, units
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def finish() -> None:
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()
