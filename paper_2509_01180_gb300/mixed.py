"""Batched uneven alignment: subtomograms of several box edges, templates and start counts in ONE CUDA-graph
launch.

Each box class has its own plan (basis table) and its own branch of the graph: expansion of all of its
subtomograms, then one alignment launch per start-count group (particles are sorted by start count, so a
group is a contiguous slice).  The branches run concurrently on separate streams, so small-band classes
fill the SMs that a large-band class leaves idle.  Kernel variants (lanes per start, GEMM tile) are chosen
per (class, group) by bh_autotune before capture.  Marshalling only: all arithmetic is in libbh.
"""
from __future__ import annotations

import numpy as np

from . import bh


class MixedBatch:
    def __init__(self, classes, device, mode: int = bh.BH_MODE_BF16_SPLIT, autotune: bool = True):
        import torch
        self.classes = classes
        self.device = device
        self.parts = []
        for cw in classes:
            plan = bh.bh_plan_create(cw.N, cw.Lmax, cw.lam_max, mode, max_batch=min(cw.B, 2048))
            tv = torch.from_numpy(cw.templates).to(device)
            tmpl = bh.bh_expand(plan, tv).contiguous()  # (n_templates, Nb, 2)
            vols = torch.from_numpy(cw.vols).to(device)
            coef = torch.empty((cw.B, plan.Nb, 2), dtype=torch.float32, device=device)
            tidx = torch.from_numpy(cw.tmpl_index.astype(np.int32)).to(device)
            quat = torch.empty((cw.B, 4), dtype=torch.float32, device=device)
            score = torch.empty((cw.B,), dtype=torch.float32, device=device)
            groups = []
            for first, count, S in cw.groups():
                starts = torch.from_numpy(np.ascontiguousarray(cw.starts[first:first + count, :S])).to(device)
                tune = bh.bh_autotune(plan, count, S, cw.stages, cw.steps) if autotune else None
                groups.append((first, count, S, starts, tune))
            self.parts.append(dict(cw=cw, plan=plan, tmpl=tmpl, vols=vols, coef=coef, tidx=tidx, quat=quat,
                                   score=score, groups=groups, stream=torch.cuda.Stream(device)))
        self.graph = None

    def _launch_class(self, p, stream):
        cw = p["cw"]
        bh.bh_expand(p["plan"], p["vols"], p["coef"], stream=stream)
        for first, count, S, starts, _ in p["groups"]:
            bh.bh_align_batch(p["plan"], p["tmpl"], p["coef"][first:first + count], starts, cw.stages, cw.steps,
                              tmpl_index=p["tidx"][first:first + count], n_templates=p["tmpl"].shape[0],
                              quat_out=p["quat"][first:first + count], score_out=p["score"][first:first + count],
                              stream=stream)

    def run_eager(self):
        """All classes on their own streams, joined into the current stream."""
        import torch
        cur = torch.cuda.current_stream(self.device)
        ev = torch.cuda.Event()
        ev.record(cur)
        for p in self.parts:
            p["stream"].wait_event(ev)
            self._launch_class(p, p["stream"])
            e = torch.cuda.Event()
            e.record(p["stream"])
            cur.wait_event(e)

    def capture(self):
        """Record the whole batch (every class's expansion and alignment launches) into one CUDA graph."""
        import torch
        self.run_eager()  # warm-up outside capture (kernel attributes, lazy module loading)
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run_eager()
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def launches_per_replay(self) -> int:
        n = 0
        for p in self.parts:
            passes = -(-p["cw"].B // p["plan"].max_batch)
            n += 3 * passes + len(p["groups"])
        return n

    def results(self):
        return [(p["quat"].cpu().numpy(), p["score"].cpu().numpy()) for p in self.parts]

    @property
    def total(self) -> int:
        return sum(p["cw"].B for p in self.parts)

    def destroy(self):
        for p in self.parts:
            p["plan"].destroy()


def shard_classes(classes, rank: int, world: int):
    """This rank's share of one mixed batch split over `world` GPUs: subtomograms assigned by a cost-balanced
    partition (expansion V * Nb plus S (1 + steps) Wigner evaluations per band), classes kept, particles kept
    in start-count order.  Returns (classes restricted to the share, per-class original indices)."""
    import copy

    from . import replicas
    costs, owner = [], []
    for ci, cw in enumerate(classes):
        L = cw.Lmax
        # basis size (FP64 roots on the host) and in-ball voxel count (centre N/2, r < 1) of the class
        N = cw.N
        K, _, _ = bh.bh_basis_roots(L, cw.lam_max)
        Nb = int(sum((2 * l + 1) * int(K[l]) for l in range(L + 1)))
        c = (np.arange(N) - N / 2) / (N / 2)
        V = int(np.count_nonzero((c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2) < 1.0))
        for b in range(cw.B):
            costs.append(replicas.particle_cost(Nb, V, int(cw.S[b]), cw.steps, cw.stages))
            owner.append((ci, b))
    mine = replicas.balanced_partition(costs, world)[rank]
    out, index = [], []
    for ci, cw in enumerate(classes):
        sel = np.array([owner[i][1] for i in mine if owner[i][0] == ci], dtype=np.int64)
        sub = copy.copy(cw)
        sub.vols, sub.tmpl_index, sub.q_true = cw.vols[sel], cw.tmpl_index[sel], cw.q_true[sel]
        sub.S, sub.starts = cw.S[sel], cw.starts[sel]
        out.append(sub)
        index.append(sel)
    return out, index
