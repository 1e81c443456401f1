"""Multi-GPU host logic on CPU: world_size-2 gloo ranks shard subtomograms without overlap and agree on
the max-over-ranks timing (the only cross-rank step of the replicas)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2509_01180_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first = replicas.shard_first(rank, 1024)
    times = replicas.max_over_ranks([10.0 + rank, 5.0 - rank])
    replicas.barrier()
    q.put((rank, first, times))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [0, 1024]
    assert out[0][2] == out[1][2] == [11.0, 5.0]


def test_single_process_is_identity():
    assert replicas.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]
    assert replicas.shard_first(3, 7) == 21
    with pytest.raises(ValueError):
        replicas.shard_first(-1, 7)
