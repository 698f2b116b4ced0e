"""Multi-GPU as replicas: one process per GPU, independent work, no data-path collective.

Every transform and vector op of this library is independent, so N GPUs run N shards of the
job list (or N copies of a benchmark step): a batch of uneven jobs is split by estimated cost, a
served request stream round-robin by arrival (each rank serves its own requests).  The process group is used only to line the ranks
up before and after a timed region and to combine per-rank numbers (max of times, sum of work).
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def world() -> tuple[int, int, int]:
    """(world_size, rank, local_rank) from the torchrun environment (1, 0, 0 when absent)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str = "nccl") -> None:
    ws, _, _ = world()
    if ws > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend)


def barrier() -> None:
    if dist.is_initialized():
        dist.barrier()


def _reduce(x: float, op, device) -> float:
    if not dist.is_initialized():
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x: float, device="cpu") -> float:
    return _reduce(x, dist.ReduceOp.MAX, device)


def sum_over_ranks(x: float, device="cpu") -> float:
    return _reduce(x, dist.ReduceOp.SUM, device)


def shard(items, rank: int, world_size: int):
    """Round-robin share of a job list for one rank (disjoint, together complete)."""
    return list(items)[rank::world_size]


def shard_balanced(items, rank: int, world_size: int, cost):
    """Share of a list of uneven jobs for one rank, balanced by estimated cost: jobs in order of
    decreasing cost (ties by position) go one at a time to the rank with the least cost so far
    (ties to the lowest rank).  Every rank computes the same assignment without communicating and
    keeps its own jobs in their original order, so the shares are disjoint and together complete."""
    items = list(items)
    if world_size <= 1:
        return items
    order = sorted(range(len(items)), key=lambda i: (-cost(items[i]), i))
    load = [0.0] * world_size
    owner = [0] * len(items)
    for i in order:
        r = min(range(world_size), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += cost(items[i])
    return [it for i, it in enumerate(items) if owner[i] == rank]


def job_cost(job) -> float:
    """Relative device work of one job (for balancing only): transforms n log2 n L^2 (a cyclic
    product three transforms), element-wise jobs n L^2."""
    limbs = job.width // 32
    if job.op in ("ntt_fwd", "ntt_inv", "polymul"):
        lg = max(1, int(job.n).bit_length() - 1)
        return job.n * lg * limbs * limbs * (3 if job.op == "polymul" else 1)
    return job.n * limbs * limbs


def finalize() -> None:
    if dist.is_initialized():
        dist.destroy_process_group()
