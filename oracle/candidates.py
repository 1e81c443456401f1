"""Candidate starts from local maxima of the lowest marching band, FP64 (oracle; test infrastructure).

Only tests/, the smoke check and the benchmark's CPU-baseline leg may import this module.

Paper passage: Sec. III picks the initial candidate rotations as the local maxima of Eq. 2 truncated at
the lowest selected band (L = 7 there), then refines them through the higher bands.

Readings where the paper is silent:
  * The band-L score is evaluated on a given finite rotation grid (the paper names no grid; the inputs
    use super-Fibonacci spirals).  Rotations are unit quaternions; q and -q are the same rotation.
  * Neighbours: j != i with geodesic angle 2 acos|q_i . q_j| <= rho, decided as
    |q_i . q_j| >= cos(rho / 2).  The dot product is summed in the order w, x, y, z in FP64 (the
    products of float32 grid coordinates are exact in FP64), so the relation is reproducible.
  * Order: grid point i ranks above j when its score is larger, or equal with i < j.  A grid point is a
    local maximum when it ranks above every neighbour.
  * Candidates: the local maxima in rank order; if there are fewer than S, the remaining slots take the
    highest-ranked other grid points.  The first S are returned.
"""
from __future__ import annotations

import math

import numpy as np

from .align import align_particle, build_xi, score


def grid_scores(xi: list[np.ndarray], grid: np.ndarray, L: int) -> np.ndarray:
    """Eq. 2 truncated at band L at every grid rotation (FP64)."""
    return np.array([score(xi, q, L) for q in np.asarray(grid, dtype=np.float64)])


def grid_neighbors(grid: np.ndarray, radius: float) -> list[np.ndarray]:
    """Indices j != i with |q_i . q_j| >= cos(radius / 2), ascending, for every grid point i."""
    q = np.asarray(grid, dtype=np.float32).astype(np.float64)
    c = math.cos(radius / 2)
    out = []
    for i in range(len(q)):
        d = q[i, 0] * q[:, 0] + q[i, 1] * q[:, 1] + q[i, 2] * q[:, 2] + q[i, 3] * q[:, 3]
        nb = np.nonzero(np.abs(d) >= c)[0]
        out.append(nb[nb != i])
    return out


def _ranks_above(s: np.ndarray, i: int, j: int) -> bool:
    return s[i] > s[j] or (s[i] == s[j] and i < j)


def local_maxima(scores: np.ndarray, neighbors: list[np.ndarray]) -> np.ndarray:
    """Boolean mask of the grid points that rank above all of their neighbours."""
    return np.array([all(_ranks_above(scores, i, int(j)) for j in nb) for i, nb in enumerate(neighbors)])


def candidates(scores: np.ndarray, neighbors: list[np.ndarray], S: int) -> np.ndarray:
    """The first S grid indices: local maxima by rank, then the other grid points by rank."""
    scores = np.asarray(scores)
    is_max = local_maxima(scores, neighbors)
    order = sorted(range(len(scores)), key=lambda i: (not is_max[i], -scores[i], i))
    return np.array(order[:S], dtype=np.int64)


def align_from_candidates(basis, t_hat, f_hat, grid, radius: float, S: int, stages: list[int], steps: int):
    """Sec. III pipeline for one pair: band-stages[0] scores on the grid, S candidates from its local maxima,
    then the marching ascent (Sec. II-C) from those candidates."""
    xi = build_xi(basis, t_hat, f_hat, max(stages))
    sc = grid_scores(xi, grid, stages[0])
    idx = candidates(sc, grid_neighbors(grid, radius), S)
    starts = np.asarray(grid, dtype=np.float64)[idx]
    return idx, align_particle(basis, t_hat, f_hat, starts, stages, steps)

