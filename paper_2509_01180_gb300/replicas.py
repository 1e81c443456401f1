"""Replica sharding for several GPUs: the alignment of different subtomograms never exchanges data, so
N GPUs run N independent replicas.  Only the timing is combined (max over ranks), with torch.distributed
(NCCL on GPUs, gloo on CPU)."""
from __future__ import annotations


def shard_first(rank: int, per_rank: int) -> int:
    """Index of the first subtomogram of `rank` when every rank aligns `per_rank` of its own (weak scaling)."""
    if rank < 0 or per_rank < 0:
        raise ValueError("rank and per_rank must be >= 0")
    return rank * per_rank


def max_over_ranks(values, device=None):
    """Element-wise maximum of a list of floats over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()
