"""Host logic of the multi-GPU run: independent replicas, one per rank.

The deflated solve has no data-path exchange between GPUs at these sizes (one
system fits one GPU; a batch of systems is split by system), so N GPUs run N
independent solves of the same workload, each on its own seeded field.  The
only collectives are the bench's timing ones: a barrier on both sides of the
timed region and the maximum of the per-rank step times.

Ranks are launched by torch.distributed.run (RANK, LOCAL_RANK, WORLD_SIZE,
MASTER_ADDR, MASTER_PORT in the environment); NCCL on GPUs, gloo on CPU.
"""
from __future__ import annotations

import os


def dist_env():
    """(world size, rank, local rank) from the launcher's environment."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def init(cuda: bool):
    """Join the process group when there is more than one rank."""
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl" if cuda else "gloo")
    return world, rank, local


def barrier(cuda: bool):
    """All ranks here, and (on GPUs) this rank's queued work finished."""
    import torch
    world, _, _ = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    if cuda:
        torch.cuda.synchronize()


def max_over_ranks(value: float, cuda: bool) -> float:
    """The largest of the ranks' values (the job's step time)."""
    world, _, _ = dist_env()
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device="cuda" if cuda else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank: int, base: int = 1) -> int:
    """Seed of the rank's workload: every replica solves its own field."""
    return base + rank


def finish():
    world, _, _ = dist_env()
    if world > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()
