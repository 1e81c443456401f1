"""Missing-wedge constrained correlation (Sec. II-B), FP64 (oracle; test infrastructure).

Only tests/, the smoke check and the benchmark's CPU legs may import this module.

Paper passage: Sec. II-B counters the missing wedge by measuring the correlation only in the region of
Fourier space that both volumes sample (the constrained correlation of Foerster et al., 2008).

Readings where the paper is silent:
  * Wedge geometry (the synthetic data's): tilt axis y, beam z; the subtomogram f samples the Fourier
    directions with |k_z| <= tan(a) |k_x| (a = tilt half-angle); W is that indicator on the unit sphere.
    The template t is complete.
  * Rotating f by R rotates its sampled region: W_R(k) = W(R^{-1} k).  The part of t's Fourier transform
    inside W_R is all that <t, R f> sees, so the constrained score is C(R) = S(R) / sqrt(Dn(R)) with
    S(R) of Eq. 2 and Dn(R) = ||W_R t||^2; ||f|| does not depend on R and is dropped.
  * Dn on the voxel grid: Dn(R) = |T(0)|^2 + sum over DFT frequencies 0 < |k| < N/2 of
    W_L(R^{-1} k/|k|) |T(k)|^2, T the unnormalised DFT of the template restricted to the ball, W_L the
    spherical-harmonic expansion of W truncated at the marching band L of the stage (so Dn is
    band-limited like S).
    Then Dn(R) = |T(0)|^2 + Re sum_{l<=L} sum_{m,m'} q_lm w_lm' D^l_{mm'}(R),
    q_lm = sum_k Y_l^m(k^) |T(k)|^2,  w_lm = <Y_l^m, W> on the sphere:
    Eq. 2's form with xi'^l_{mm'} = q_lm w_lm' (one radial index per degree).
  * w_lm: with x = cos(theta), W restricts phi to |cos phi| >= |cot theta| / tan(a); the phi integral is
    closed-form and the x integral is taken in the variable phi0 = arccos(|cot theta| / tan(a)), where
    the integrand is smooth (Gauss-Legendre).
  * Constrained ascent: the step rule of the ascent (align.ascend) applied to C, with
    grad C = grad S / sqrt(Dn) - S grad Dn / (2 Dn^{3/2}).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .align import StartResult, _normalize, build_xi, score_grad, select_best
from .ball import assoc_legendre_normalized, sph_harm_all, voxel_ball
from .wigner import quat_mul


def wedge_indicator(kdir: np.ndarray, half_angle_deg: float) -> np.ndarray:
    """1 where the direction (x, y, z) is sampled (|k_z| <= tan(a) |k_x|), else 0."""
    t = math.tan(math.radians(half_angle_deg))
    return (np.abs(kdir[..., 2]) <= t * np.abs(kdir[..., 0])).astype(np.float64)


def wedge_sh(L: int, half_angle_deg: float, n_gl: int = 96) -> list[np.ndarray]:
    """w[l][m+l] = integral over the sphere of W conj(Y_l^m), l <= L."""
    a = math.radians(half_angle_deg)
    T = math.tan(a)
    u, wu = np.polynomial.legendre.leggauss(n_gl)
    phi0 = (u + 1) * (math.pi / 4)  # [0, pi/2]
    wq = wu * (math.pi / 4)
    c = np.cos(phi0)
    x = T * c / np.sqrt(1 + (T * c) ** 2)  # cos(theta) on the upper half, x in [0, sin a]
    jac = T * np.sin(phi0) / (1 + (T * c) ** 2) ** 1.5  # |dx/dphi0|
    P = assoc_legendre_normalized(L, x)  # P[l][m] normalised so that Y_l^m = P_lm e^{i m phi}
    out = []
    for l in range(L + 1):
        row = np.zeros(2 * l + 1, dtype=np.complex128)
        for m in range(0, l + 1):
            if (l + m) % 2 or m % 2:
                continue  # the integrand is odd in x (l + m odd) or the two phi arcs cancel (m odd)
            Phi = 4 * phi0 if m == 0 else 4 * np.sin(m * phi0) / m
            val = 2 * float(np.sum(wq * P[l, m] * Phi * jac))  # both hemispheres
            row[m + l] = val
            if m > 0:
                row[-m + l] = (-1) ** m * val
        out.append(row)
    return out


def dft_power(tvol: np.ndarray) -> tuple[np.ndarray, np.ndarray, float]:
    """Directions k/|k| and |T(k)|^2 over the DFT frequencies 0 < |k| < N/2 of the ball-restricted
    template, and |T(0)|^2."""
    N = tvol.shape[0]
    flat, _ = voxel_ball(N)
    tb = np.zeros(N ** 3)
    tb[flat] = np.asarray(tvol, np.float64).ravel()[flat]
    T = np.fft.fftn(tb.reshape(N, N, N))
    k = np.fft.fftfreq(N) * N
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    r = np.sqrt(kx * kx + ky * ky + kz * kz)
    sel = (r > 0) & (r < N / 2)
    dirs = np.stack([kx[sel], ky[sel], kz[sel]], axis=1) / r[sel][:, None]
    return dirs, np.abs(T[sel]) ** 2, float(np.abs(T[0, 0, 0]) ** 2)


def power_sh(dirs: np.ndarray, pw: np.ndarray, L: int) -> list[np.ndarray]:
    """q[l][m+l] = sum_k Y_l^m(k^) |T(k)|^2."""
    Y = sph_harm_all(L, dirs)  # Y[l] of shape (points, 2l+1)
    return [Y[l].T @ pw for l in range(L + 1)]


@dataclass
class Wedge:
    L: int
    q: list
    w: list
    c0: float

    def xi(self, L: int | None = None) -> list[np.ndarray]:
        L = self.L if L is None else L
        return [np.outer(self.q[l], self.w[l]) for l in range(L + 1)]


def make_wedge(tvol: np.ndarray, half_angle_deg: float, L: int) -> Wedge:
    dirs, pw, c0 = dft_power(np.asarray(tvol, np.float64))
    return Wedge(L, power_sh(dirs, pw, L), wedge_sh(L, half_angle_deg), c0)


def denominator(wd: Wedge, q, L: int) -> tuple[float, np.ndarray]:
    """Dn(R) = ||W_R t||^2 at band L and its body-frame gradient."""
    D, g = score_grad(wd.xi(L), q, L)
    return wd.c0 + D, g


def constrained_score_grad(xi, wd: Wedge, q, L: int) -> tuple[float, np.ndarray]:
    """C(R) = S(R) / sqrt(Dn(R)) and its body-frame gradient, both at band L."""
    S, gS = score_grad(xi, q, L)
    Dn, gD = denominator(wd, q, L)
    r = 1.0 / math.sqrt(Dn)
    return S * r, gS * r - 0.5 * S * r * r * r * gD


def ascend_constrained(xi, wd: Wedge, q0, stages: list[int], steps: int) -> StartResult:
    """The ascent's step rule and marching on C(R)."""
    q = _normalize(q0)
    C = 0.0
    accepted = evals = 0
    for L in stages:
        h0, hmax = math.pi / (2 * L), math.pi / L
        C, g = constrained_score_grad(xi, wd, q, L)
        evals += 1
        h = h0
        for _ in range(steps):
            gn = float(np.linalg.norm(g))
            if gn <= 1e-12 * abs(C):
                break
            u = g / gn
            qt = _normalize(quat_mul(q, np.array([math.cos(h / 2), *(math.sin(h / 2) * u)])))
            Ct, gt = constrained_score_grad(xi, wd, qt, L)
            evals += 1
            if Ct > C:
                q, C, g = qt, Ct, gt
                h = min(1.5 * h, hmax)
                accepted += 1
            else:
                h = h / 2
    return StartResult(q, C, accepted, evals)


def align_constrained(basis, t_hat, f_hat, wd: Wedge, starts, stages: list[int], steps: int):
    """One pair: every start's constrained ascent, then the best final constrained score."""
    from .align import AlignResult
    xi = build_xi(basis, t_hat, f_hat, max(stages))
    res = [ascend_constrained(xi, wd, q0, stages, steps) for q0 in starts]
    sc = np.array([r.score for r in res])
    qs = np.array([r.q for r in res])
    b = select_best(sc)
    return AlignResult(qs[b], float(sc[b]), qs, sc, b)
