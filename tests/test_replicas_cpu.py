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


def test_balanced_partition_covers_once_and_balances():
    import random
    rng = random.Random(5)
    # mixed-box costs: 3000 x 24^3 (l <= 12), 2000 x 40^3 (l <= 20), 1000 x 64^3 (l <= 32) in a shuffled order
    costs = ([replicas.particle_cost(1323, 7123, 16, 30, [3, 6, 12])] * 300 +
             [replicas.particle_cost(5886, 33371, 16, 30, [5, 10, 20])] * 200 +
             [replicas.particle_cost(23536, 137059, 32, 30, [8, 16, 32])] * 100)
    rng.shuffle(costs)
    for world in (1, 2, 3, 8):
        parts = replicas.balanced_partition(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs) + 1e-6 * sum(costs)
        assert parts == replicas.balanced_partition(costs, world)  # deterministic on every rank
    with pytest.raises(ValueError):
        replicas.balanced_partition(costs, 0)


def _gather_worker(rank, world, port, q):
    import numpy as np
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    costs = [float((7 * i) % 11 + 1) for i in range(23)]
    mine = replicas.balanced_partition(costs, world)[rank]
    quat = np.array([[i, 0, 0, 1] for i in mine], np.float32).reshape(-1, 4)
    score = np.array([10.0 * i for i in mine], np.float32)
    Q, S, seen = replicas.gather_results(mine, quat, score, len(costs))
    q.put((rank, Q.tolist(), S.tolist(), bool(seen.all())))
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_results_in_order():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gather_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, Q, S, all_seen in out:
        assert all_seen
        assert [row[0] for row in Q] == list(range(23))
        assert S == [10.0 * i for i in range(23)]


def test_mixed_batch_shards_cover_every_particle_once():
    import numpy as np

    from paper_2509_01180_gb300 import mixed, synth
    classes = synth.make_mixed(scale=0.01, distinct=3)
    for world in (1, 2, 3):
        seen = [np.zeros(cw.B, dtype=int) for cw in classes]
        for rank in range(world):
            sub, idx = mixed.shard_classes(classes, rank, world)
            for ci, (cw, sc, ix) in enumerate(zip(classes, sub, idx)):
                seen[ci][ix] += 1
                assert sc.B == len(ix)
                assert (np.diff(sc.S) >= 0).all()  # start-count groups stay contiguous
                assert np.array_equal(sc.vols, cw.vols[ix])
        assert all((s == 1).all() for s in seen)
