"""Rotational cross-correlation, its gradient and the marching ascent, FP64 (oracle; test infrastructure).

Paper passages:
  * Eq. 1: the cross-correlation C_{f,t}(s, g) = int t(x) [R_g f](x + s) dx; here s = 0
    (subtomograms are centred), so C(g) = <t, R_g f> for real t, f.
  * Eq. 2: C^L(s, g) = sum_{l<=L} sum_{m,m'} xi^s_{l,m,m'} D^l_{m,m'}(g), with xi
    built from t_hat and f_hat_s.
  * Sec. II-C: closed-form derivative of Eq. 2 in g; gradient-based maximisation
    combined with frequency marching (the band L raised in stages); the
    exhaustive grid evaluation is the most accurate (used as a brute-force pin).
  * Fig. 1 caption: energy ratio Ratio(L).

Readings where the paper is silent, garbled or ambiguous:
  * xi^l_{mm'} = sum_k conj(t_hat_klm) f_hat_klm' (Eq. 2 names xi without defining it).
    With orthonormal psi, <t, R f> = Re sum_l sum_{m,m'} xi^l_{mm'} D^l_{mm'}(R).
    Its maximiser is R* = R_true^{-1} when f = R_true t.
  * Gradient: right perturbation R exp(eps J_i), i in {x, y, z} (body axes), giving
    g_i = Re sum_l sum_{m,m'} xi^l_{mm'} [D^l(R) (-i J_i)]_{mm'}.
  * Ascent step rule (the paper names gradient-based steps only): per stage with band L,
    h0 = pi/(2L), hmax = pi/L; each of T steps: stop if |g| <= 1e-12 |S|; else u = g/|g|,
    trial R' = R exp(h u.J); accept if S(R') > S(R) (then h <- min(1.5 h, hmax)), else h <- h/2.
    Quaternions are renormalised after every accepted product.
  * Marching: stages L1 < L2 < ... truncate in l only (all k kept); every start is
    carried through every stage; each stage restarts h at h0 and re-evaluates S, g.
  * Selection: argmax over starts of the final-stage score; ties within 1e-12 |S|
    go to the lowest start index.
  * Energy ratio: the Fig. 1 caption omits the sums over m, m'; the reading sums them.
  * Band selection (Sec. II-C: the energy ratio picks high-energy bands; Sec. III: L_set chosen with it;
    no rule is printed): for thresholds tau_1 > tau_2 > ... > tau_n in (0, 1) and a lowest band L_min >= 1,
    band j is the smallest L >= L_min whose remaining energy Ratio(L) is at most tau_j (Ratio(Lmax) = 0,
    so it exists); equal consecutive bands are kept once, so the marching schedule is strictly increasing.
  * Newton steps (Sec. III names them, without details): the Hessian is the second derivative of
    S(R exp(eps.J)) at eps = 0, H_ij = -Re sum xi^l_{mm'} [D^l(R) (J_i J_j + J_j J_i) / 2]_{mm'}.
    Per stage with band L, T iterations: stop if |g| <= 1e-12 |S|; if H is negative definite the
    direction is d = -H^{-1} g, else the gradient step d = (pi/(2L)) g/|g|; d is clipped to length
    pi/L and scaled by a damping factor lam (1 at the stage start); the trial R exp(d.J) is accepted if
    it raises S (then lam <- min(1, 2 lam)), else lam <- lam/2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .ball import Basis, split_by_degree
from .wigner import _j, quat_mul, wigner_D


def build_xi(basis: Basis, t_hat: np.ndarray, f_hat: np.ndarray, L: int | None = None) -> list[np.ndarray]:
    """xi[l][m+l, m'+l] = sum_k conj(t_hat_klm) f_hat_klm' for l <= L (Eq. 2)."""
    L = basis.Lmax if L is None else L
    T = split_by_degree(basis, t_hat)
    F = split_by_degree(basis, f_hat)
    return [np.conj(T[l]).T @ F[l] for l in range(L + 1)]


def score(xi: list[np.ndarray], q, L: int) -> float:
    """Eq. 2 at s = 0, truncated at band L: Re sum_{l<=L} sum_{m,m'} xi^l_{mm'} D^l_{mm'}(q)."""
    return float(sum(np.real(np.sum(xi[l] * wigner_D(l, q))) for l in range(L + 1)))


def score_grad(xi: list[np.ndarray], q, L: int) -> tuple[float, np.ndarray]:
    """Eq. 2 and its closed-form derivative along R(q) exp(eps J_i) for i = x, y, z (Sec. II-C)."""
    S = 0.0
    g = np.zeros(3)
    for l in range(L + 1):
        D = wigner_D(l, q)
        S += float(np.real(np.sum(xi[l] * D)))
        J = _j(l)
        for i in range(3):
            g[i] += float(np.real(np.sum(xi[l] * (D @ (-1j * J[i])))))
    return S, g


def score_grad_hess(xi: list[np.ndarray], q, L: int) -> tuple[float, np.ndarray, np.ndarray]:
    """Eq. 2, its body-frame gradient and Hessian along R(q) exp(eps.J) (Newton steps, Sec. III)."""
    S = 0.0
    g = np.zeros(3)
    H = np.zeros((3, 3))
    for l in range(L + 1):
        D = wigner_D(l, q)
        J = _j(l)
        S += float(np.real(np.sum(xi[l] * D)))
        for i in range(3):
            g[i] += float(np.real(np.sum(xi[l] * (D @ (-1j * J[i])))))
            for k in range(3):
                H[i, k] -= 0.5 * float(np.real(np.sum(xi[l] * (D @ (J[i] @ J[k] + J[k] @ J[i])))))
    return S, g, H


def _normalize(q):
    q = np.asarray(q, dtype=np.float64)
    return q / np.linalg.norm(q)


@dataclass
class StartResult:
    q: np.ndarray
    score: float
    accepted: int
    evals: int


def ascend(xi: list[np.ndarray], q0, stages: list[int], steps: int) -> StartResult:
    """Multi-stage gradient ascent of one start with frequency marching (Sec. II-C)."""
    q = _normalize(q0)
    S = 0.0
    accepted = 0
    evals = 0
    for L in stages:
        if L < 1:
            raise ValueError("marching bands must be >= 1")
        h0, hmax = math.pi / (2 * L), math.pi / L
        S, g = score_grad(xi, q, L)
        evals += 1
        h = h0
        for _ in range(steps):
            gn = float(np.linalg.norm(g))
            if gn <= 1e-12 * abs(S):
                break
            u = g / gn
            step = np.array([math.cos(h / 2), *(math.sin(h / 2) * u)])
            qt = _normalize(quat_mul(q, step))
            St, gt = score_grad(xi, qt, L)
            evals += 1
            if St > S:
                q, S, g = qt, St, gt
                h = min(1.5 * h, hmax)
                accepted += 1
            else:
                h = h / 2
    return StartResult(q, S, accepted, evals)


def newton(xi: list[np.ndarray], q0, stages: list[int], steps: int) -> StartResult:
    """Damped Newton iteration of one start with frequency marching (Sec. III, Sec. II-C)."""
    q = _normalize(q0)
    S = 0.0
    accepted = 0
    evals = 0
    for L in stages:
        if L < 1:
            raise ValueError("marching bands must be >= 1")
        h0, hmax = math.pi / (2 * L), math.pi / L
        S, g, H = score_grad_hess(xi, q, L)
        evals += 1
        lam = 1.0
        for _ in range(steps):
            gn = float(np.linalg.norm(g))
            if gn <= 1e-12 * abs(S):
                break
            if np.linalg.eigvalsh(H).max() < 0:
                d = -np.linalg.solve(H, g)
            else:
                d = h0 * g / gn
            dn = float(np.linalg.norm(d))
            if dn > hmax:
                d = d * (hmax / dn)
                dn = hmax
            d = lam * d
            dn = lam * dn
            step = np.array([math.cos(dn / 2), *(math.sin(dn / 2) * d / dn)]) if dn > 0 else np.array([1.0, 0, 0, 0])
            qt = _normalize(quat_mul(q, step))
            St, gt, Ht = score_grad_hess(xi, qt, L)
            evals += 1
            if St > S:
                q, S, g, H = qt, St, gt, Ht
                lam = min(1.0, 2 * lam)
                accepted += 1
            else:
                lam = lam / 2
    return StartResult(q, S, accepted, evals)


def select_best(scores: np.ndarray) -> int:
    """Index of the largest final score; ties within 1e-12 |S| go to the lowest index."""
    best = 0
    for s in range(1, len(scores)):
        if scores[s] > scores[best] + 1e-12 * abs(scores[best]):
            best = s
    return best


@dataclass
class AlignResult:
    q: np.ndarray  # best rotation (w, x, y, z)
    score: float
    start_q: np.ndarray  # (S, 4) final rotation of every start
    start_score: np.ndarray  # (S,)
    best: int


def align_particle(basis: Basis, t_hat, f_hat, starts: np.ndarray, stages: list[int], steps: int,
                   method: str = "ascent") -> AlignResult:
    """One template/subtomogram pair: xi, every start's marching ascent (or Newton iteration), selection."""
    xi = build_xi(basis, t_hat, f_hat, max(stages))
    run = {"ascent": ascend, "newton": newton}[method]
    res = [run(xi, q0, stages, steps) for q0 in starts]
    sc = np.array([r.score for r in res])
    qs = np.array([r.q for r in res])
    b = select_best(sc)
    return AlignResult(qs[b], float(sc[b]), qs, sc, b)


def energy_ratio(xi: list[np.ndarray]) -> np.ndarray:
    """Ratio(L) = sum_{l>L} |xi^l|^2 / sum_{l<=Lmax} |xi^l|^2 for L = 0..Lmax (Fig. 1 caption)."""
    e = np.array([float(np.sum(np.abs(x) ** 2)) for x in xi])
    tot = e.sum()
    tail = np.concatenate([np.cumsum(e[::-1])[::-1][1:], [0.0]])
    return tail / tot if tot > 0 else np.zeros_like(e)


def choose_bands(xi: list[np.ndarray], thresholds, L_min: int = 1) -> list[int]:
    """Marching bands picked by the energy ratio of Fig. 1 (reading above): for each threshold tau_j, in the
    given (decreasing) order, the smallest L >= L_min with Ratio(L) <= tau_j; repeats dropped."""
    r = energy_ratio(xi)
    Lmax = len(r) - 1
    if not 1 <= L_min <= Lmax:
        raise ValueError("L_min must lie in 1..Lmax")
    bands = []
    for tau in thresholds:
        L = next(L for L in range(L_min, Lmax + 1) if r[L] <= tau)
        if not bands or L > bands[-1]:
            bands.append(L)
    return bands


def rotate_coeffs(basis: Basis, coeffs: np.ndarray, q) -> np.ndarray:
    """Coefficients of R(q) f from those of f: (R f)^_{klm} = sum_m' D^l_{mm'}(q) f^_{klm'} (Sec. II-A steerability)."""
    out = np.array(coeffs, dtype=np.complex128, copy=True)
    for l in range(basis.Lmax + 1):
        D = wigner_D(l, q)
        o0, o1 = basis.offsets[l], basis.offsets[l + 1]
        blk = out[o0:o1].reshape(-1, 2 * l + 1)
        out[o0:o1] = (blk @ D.T).ravel()
    return out


@dataclass
class ShiftResult:
    shift: int  # index of the best shift
    q: np.ndarray
    score: float
    per_shift: list


def align_shifts(basis: Basis, t_hat, vol, shifts, starts: np.ndarray, stages: list[int], steps: int) -> ShiftResult:
    """Eq. 1 over a grid of shifts (Sec. II-C): for each shift s, expand f_s(x) = f(x + s) and maximise Eq. 2
    from the same starts; keep the (shift, rotation) with the largest final score (ties: lowest shift index)."""
    from .ball import expand, shift_volume
    res = []
    for s in shifts:
        f_hat = expand(basis, shift_volume(vol, s))[0]
        res.append(align_particle(basis, t_hat, f_hat, starts, stages, steps))
    best = select_best(np.array([r.score for r in res]))
    return ShiftResult(best, res[best].q, res[best].score, res)
