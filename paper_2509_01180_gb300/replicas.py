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


def particle_cost(Nb: int, V: int, S: int, steps: int, stages) -> float:
    """Work of one subtomogram: the expansion's V * Nb products plus S * (1 + steps) evaluations per marching
    band, each over E(L) = sum_{l<=L} (2l+1)^2 Wigner entries."""
    ev = sum(sum((2 * l + 1) ** 2 for l in range(L + 1)) for L in stages)
    return float(V) * Nb + float(S) * (1 + steps) * ev


def balanced_partition(costs, world: int) -> list[list[int]]:
    """Cost-balanced assignment of subtomograms to `world` ranks (longest-processing-time greedy: by
    decreasing cost, each goes to the least-loaded rank; ties to the lowest rank).  Deterministic, so every
    rank computes the same assignment without communication.  Indices are ascending within a rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    import heapq
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(p) for p in parts]


def gather_results(indices, quat, score, total: int):
    """Host-side gather of per-subtomogram results (quaternion, score: 20 bytes each) from every rank into the
    original order on every rank; the only cross-rank data of the replicas.  Without a process group the
    local results are scattered into place."""
    import numpy as np
    import torch.distributed as dist
    local = (list(map(int, indices)), np.asarray(quat, np.float32).reshape(-1, 4), np.asarray(score, np.float32).ravel())
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        allp = [None] * dist.get_world_size()
        dist.all_gather_object(allp, local)
    else:
        allp = [local]
    Q = np.full((total, 4), np.nan, np.float32)
    Sc = np.full((total,), np.nan, np.float32)
    seen = np.zeros(total, dtype=bool)
    for idx, q, s in allp:
        if len(idx) != len(q) or len(idx) != len(s):
            raise ValueError("indices and results differ in length")
        for j, i in enumerate(idx):
            if seen[i]:
                raise ValueError(f"subtomogram {i} returned by two ranks")
            seen[i] = True
            Q[i], Sc[i] = q[j], s[j]
    return Q, Sc, seen
