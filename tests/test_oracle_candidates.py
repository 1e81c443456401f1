"""Pins of the oracle's candidate starts: local maxima of the lowest band on a rotation grid (Sec. III).

CPU only."""
import math

import numpy as np
import pytest

from oracle import align, ball, candidates, wigner
from oracle.wigner import quat_conj
from paper_2509_01180_gb300 import synth
from tests.test_oracle_wigner import rand_quats


def matrix_angle(qa, qb) -> float:
    """Geodesic angle between two rotations from their matrices: acos((tr(Ra^T Rb) - 1) / 2)."""
    Ra, Rb = wigner.quat_to_matrix(np.asarray(qa, np.float64)), wigner.quat_to_matrix(np.asarray(qb, np.float64))
    return math.acos(max(-1.0, min(1.0, (np.trace(Ra.T @ Rb) - 1) / 2)))


def test_super_fibonacci_grid_is_unit_and_covers_so3():
    g = synth.super_fibonacci(1000).astype(np.float64)
    assert np.abs(np.linalg.norm(g, axis=1) - 1).max() < 1e-6
    assert (g[:, 0] >= 0).all()
    probe = rand_quats(300, 5)
    worst = max(min(matrix_angle(p, q) for q in g[::1]) for p in probe[:60])
    assert worst < math.radians(25.0), math.degrees(worst)


def test_neighbors_are_the_rotations_within_the_radius():
    """Neighbour relation vs the rotation-matrix angle (an independent formula; q and -q agree)."""
    g = synth.super_fibonacci(300)
    radius = math.radians(40.0)
    nb = candidates.grid_neighbors(g, radius)
    checked = 0
    for i in range(0, 300, 7):
        for j in range(300):
            if j == i:
                continue
            a = matrix_angle(g[i], g[j])
            if abs(a - radius) < 1e-6:
                continue
            assert (j in set(nb[i].tolist())) == (a <= radius), (i, j, math.degrees(a))
            checked += 1
    assert checked > 10000
    assert all((np.diff(n) > 0).all() for n in nb)
    assert all(len(n) > 0 for n in nb)


def test_candidate_order_hand_example():
    """Local maxima by rank, then the rest by rank; equal scores rank by lower index."""
    sc = np.array([3.0, 5.0, 5.0, 1.0, 4.0])
    nb = [np.array([1]), np.array([0, 2]), np.array([1]), np.array([4]), np.array([3])]
    assert candidates.local_maxima(sc, nb).tolist() == [False, True, False, False, True]
    assert candidates.candidates(sc, nb, 5).tolist() == [1, 4, 2, 0, 3]
    assert candidates.candidates(sc, nb, 2).tolist() == [1, 4]


def test_local_maxima_of_two_bumps():
    """Score = two separated bumps on SO(3): the first two candidates are the grid points nearest to the
    higher and to the lower bump centre (the neighbour radius exceeds twice the covering radius)."""
    g = synth.super_fibonacci(1000).astype(np.float64)
    A, B = rand_quats(1, 31)[0], None
    for q in rand_quats(50, 32):
        if matrix_angle(A, q) > math.radians(120.0):
            B = q
            break
    dA = np.array([matrix_angle(A, q) for q in g])
    dB = np.array([matrix_angle(B, q) for q in g])
    sig = math.radians(25.0)
    sc = np.exp(-(dA / sig) ** 2) + 0.8 * np.exp(-(dB / sig) ** 2)
    nb = candidates.grid_neighbors(g, math.radians(50.0))
    c = candidates.candidates(sc, nb, 4)
    assert c[0] == int(np.argmin(dA)) and c[1] == int(np.argmin(dB))
    is_max = candidates.local_maxima(sc, nb)
    assert is_max[c[0]] and is_max[c[1]]


def test_candidates_find_the_known_rotation():
    """Exactly rotated coefficients (f_hat = D(R) t_hat): the best grid candidate at band L1 lies near
    R^{-1}, and the marching ascent from the candidates reaches R^{-1}."""
    Bs = ball.make_basis(6, 6 * math.pi)
    rng = np.random.default_rng(41)
    t = rng.normal(size=Bs.Nb) + 1j * rng.normal(size=Bs.Nb)
    q_true = rand_quats(1, 42)[0]
    f = align.rotate_coeffs(Bs, t, q_true)
    g = synth.super_fibonacci(1000)
    idx, res = candidates.align_from_candidates(Bs, t, f, g, math.radians(50.0), 4, [2, 4, 6], 40)
    assert matrix_angle(g[idx[0]], quat_conj(q_true)) < math.radians(25.0)
    assert wigner.geodesic_angle(res.q, quat_conj(q_true)) < 1e-3
    assert res.best == 0 or abs(res.start_score[0] - res.score) < 1e-6 * abs(res.score)


@pytest.mark.parametrize("mutant", ["no_abs", "half_radius"])
def test_neighbor_pin_catches_mistakes(monkeypatch, mutant):
    orig = candidates.grid_neighbors

    def bad(grid, radius):
        if mutant == "half_radius":
            return orig(grid, radius / 2)
        q = np.asarray(grid, np.float32).astype(np.float64)
        c = math.cos(radius / 2)
        out = []
        for i in range(len(q)):
            d = q @ q[i]
            nb = np.nonzero(d >= c)[0]
            out.append(nb[nb != i])
        return out

    monkeypatch.setattr(candidates, "grid_neighbors", bad)
    with pytest.raises(AssertionError):
        test_neighbors_are_the_rotations_within_the_radius()


@pytest.mark.parametrize("mutant", ["minima", "ties_high"])
def test_order_pin_catches_mistakes(monkeypatch, mutant):
    if mutant == "minima":
        monkeypatch.setattr(candidates, "_ranks_above", lambda s, i, j: s[i] < s[j] or (s[i] == s[j] and i < j))
    else:
        monkeypatch.setattr(candidates, "_ranks_above", lambda s, i, j: s[i] > s[j] or (s[i] == s[j] and i > j))
    with pytest.raises(AssertionError):
        test_candidate_order_hand_example()
