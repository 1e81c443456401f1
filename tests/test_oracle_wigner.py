"""Pins of the oracle's Wigner matrices (Sec. II-A steerability; Eq. 2's D^l_{mm'}(g)).  CPU only."""
import math

import numpy as np
import pytest
from numpy.polynomial.legendre import legval

from oracle import align, ball, wigner
from oracle.wigner import quat_mul
from tests.test_oracle_basis import ball_quadrature


def rand_quats(n, seed):
    rng = np.random.default_rng(seed)
    q = rng.normal(size=(n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def zyz(alpha, beta, gamma):
    qa, qb, qc = wigner.axis_rotation(2, alpha), wigner.axis_rotation(1, beta), wigner.axis_rotation(2, gamma)
    return quat_mul(quat_mul(qa, qb), qc)


@pytest.mark.parametrize("l", [0, 1, 2, 7, 16, 32])
def test_unitary(l):
    for q in rand_quats(3, l):
        D = wigner.wigner_D(l, q)
        assert np.allclose(D @ D.conj().T, np.eye(2 * l + 1), atol=1e-12)


def test_identity_and_homomorphism():
    for l in (1, 3, 8, 12):
        assert np.allclose(wigner.wigner_D(l, [1, 0, 0, 0]), np.eye(2 * l + 1), atol=1e-15)
        q1, q2 = rand_quats(2, 100 + l)
        assert np.allclose(wigner.wigner_D(l, quat_mul(q1, q2)), wigner.wigner_D(l, q1) @ wigner.wigner_D(l, q2),
                           atol=1e-12)
        # q and -q are the same rotation, and integer l sees no sign
        assert np.allclose(wigner.wigner_D(l, -q1), wigner.wigner_D(l, q1), atol=1e-12)


@pytest.mark.parametrize("l", [0, 1, 2, 5, 10, 20, 32])
def test_d00_is_legendre(l):
    for beta in (0.0, 0.3, 1.1, 2.0, math.pi):
        c = np.zeros(l + 1)
        c[l] = 1
        assert abs(wigner.wigner_d(l, beta)[l, l] - legval(math.cos(beta), c)) < 1e-12


def test_d1_closed_form():
    # rows/columns ordered m = -1, 0, 1; d^1_{mm'}(beta) = <1 m| exp(-i beta J_y) |1 m'>
    for beta in (0.2, 1.3, 2.9):
        c, s = math.cos(beta), math.sin(beta)
        r2 = math.sqrt(2)
        ref = np.array([
            [(1 + c) / 2, s / r2, (1 - c) / 2],   # m = -1
            [-s / r2, c, s / r2],                  # m = 0
            [(1 - c) / 2, -s / r2, (1 + c) / 2],  # m = 1
        ])
        assert np.allclose(wigner.wigner_d(1, beta), ref, atol=1e-14)


def wigner_small_d_explicit(l, m, mp, beta):
    """Wigner's explicit sum for d^l_{m m'}(beta) (row m, column m')."""
    tot = 0.0
    f = math.factorial
    pre = math.sqrt(f(l + m) * f(l - m) * f(l + mp) * f(l - mp))
    for s in range(0, 2 * l + 1):
        a, b, c, d = l + mp - s, s, m - mp + s, l - m - s
        if min(a, b, c, d) < 0:
            continue
        tot += (-1) ** (m - mp + s) / (f(a) * f(b) * f(c) * f(d)) * \
            math.cos(beta / 2) ** (2 * l + mp - m - 2 * s) * math.sin(beta / 2) ** (m - mp + 2 * s)
    return pre * tot


@pytest.mark.parametrize("l", [1, 2, 3, 5, 8])
def test_d_matches_wigner_explicit_sum(l):
    for beta in (0.1, 0.9, 1.7, 3.0):
        d = wigner.wigner_d(l, beta)
        for m in range(-l, l + 1):
            for mp in range(-l, l + 1):
                assert abs(d[m + l, mp + l] - wigner_small_d_explicit(l, m, mp, beta)) < 1e-12


def test_zyz_factorisation():
    # D(Rz(a) Ry(b) Rz(c)) = diag(e^{-i m a}) d(b) diag(e^{-i m' c})
    a, b, c = 0.7, 1.9, -2.3
    for l in (1, 4, 9):
        m = np.arange(-l, l + 1)
        ref = np.exp(-1j * m * a)[:, None] * wigner.wigner_d(l, b) * np.exp(-1j * m * c)[None, :]
        assert np.allclose(wigner.wigner_D(l, zyz(a, b, c)), ref, atol=1e-12)


def test_steerability_exact_rotation():
    """A volume synthesised from random f_hat and sampled at R^{-1} x expands to D(R) f_hat (Sec. II-A).

    Synthesis and re-expansion use a product quadrature on the ball that integrates the band-limited
    products to ~1e-12, so the identity holds to quadrature accuracy; a wrong D convention
    (transpose, conjugate, inverse rotation) fails it by O(1)."""
    Bs = ball.make_basis(4, 4.5 * math.pi)
    rng = np.random.default_rng(7)
    coef = rng.normal(size=Bs.Nb) + 1j * rng.normal(size=Bs.Nb)
    pts, W = ball_quadrature(120, 4)
    for q in rand_quats(3, 8):
        Rinv = wigner.quat_to_matrix(q).T
        f_rot = ball.psi_at(Bs, pts @ Rinv.T) @ coef  # (R f)(x) = f(R^{-1} x)
        got = (ball.psi_at(Bs, pts).conj().T * W[None, :]) @ f_rot
        ref = align.rotate_coeffs(Bs, coef, q)
        assert np.allclose(got, ref, atol=1e-9)


def test_rotation_direction_of_a_dipole():
    # f(x) = x-coordinate; rotating by +90 degrees about z maps the x axis to the y axis:
    # (R f)(x) = f(R^{-1} x) = y.  In degree 1: x ~ (Y_1^{-1} - Y_1^1), y ~ i (Y_1^{-1} + Y_1^1).
    q = wigner.axis_rotation(2, math.pi / 2)
    fx = np.array([1.0, 0.0, -1.0], dtype=complex)  # coefficients of x (m = -1, 0, 1), up to scale
    fy = np.array([1j, 0.0, 1j])
    assert np.allclose(wigner.wigner_D(1, q) @ fx, fy, atol=1e-14)
