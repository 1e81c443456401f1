"""Wigner matrices D^l(g), FP64 (oracle; test infrastructure).

Paper passages:
  * Sec. II-A: rotating the ball-harmonic coefficients is an exact linear map
    within each degree l, given by Wigner D-matrices ("steerable" basis).
  * Eq. 2: D^l_{m,m'}(g), degree l, orders m, m', g in SO(3).
  * Sec. II-C: D^l is smooth and its derivative exists in closed form.

Readings where the paper is silent (convention fixed by the steerability pin
in the tests, not by transcription):
  * A rotation acts on functions by (R f)(x) = f(R^{-1} x) and
    D^l_{mm'}(R) = <Y_l^m, R Y_l^{m'}>, so (R f)^_{klm} = sum_m' D^l_{mm'}(R) f^_{klm'}.
  * Rotations are unit quaternions q = (w, x, y, z) = (cos(t/2), sin(t/2) n),
    the rotation by angle t about the unit axis n; R(q1 q2) = R(q1) R(q2).
  * With J the spin-l angular-momentum matrices in the basis m = -l..l
    (J_z = diag(m), J_+ |m> = sqrt(l(l+1) - m(m+1)) |m+1>, J_x = (J_+ + J_-)/2,
    J_y = (J_+ - J_-)/(2i)), the representation is D^l(q) = expm(-i t n.J).
    This is the definition of the rotation operator; no Euler angles are used.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import expm


def jmats(l: int):
    """(J_x, J_y, J_z) of degree l, rows/columns ordered m = -l..l (complex128)."""
    n = 2 * l + 1
    m = np.arange(-l, l + 1)
    Jp = np.zeros((n, n), dtype=np.complex128)
    for i in range(n - 1):
        Jp[i + 1, i] = math.sqrt(l * (l + 1) - m[i] * (m[i] + 1))
    Jm = Jp.conj().T
    Jx = (Jp + Jm) / 2.0
    Jy = (Jp - Jm) / 2.0j
    Jz = np.diag(m).astype(np.complex128)
    return Jx, Jy, Jz


_JCACHE: dict = {}


def _j(l):
    if l not in _JCACHE:
        _JCACHE[l] = jmats(l)
    return _JCACHE[l]


def axis_angle(q) -> tuple[float, np.ndarray]:
    """Angle t in [0, 2pi] and unit axis n of a unit quaternion (w, x, y, z)."""
    q = np.asarray(q, dtype=np.float64)
    v = q[1:]
    s = float(np.linalg.norm(v))
    t = 2.0 * math.atan2(s, float(q[0]))
    n = v / s if s > 0 else np.array([0.0, 0.0, 1.0])
    return t, n


def wigner_D(l: int, q) -> np.ndarray:
    """D^l(q) = expm(-i t n.J^(l)) for the rotation q (Eq. 2's D^l_{mm'}(g)); rows m, columns m', both -l..l."""
    t, n = axis_angle(q)
    Jx, Jy, Jz = _j(l)
    return expm(-1j * t * (n[0] * Jx + n[1] * Jy + n[2] * Jz))


def wigner_d(l: int, beta: float) -> np.ndarray:
    """Reduced matrix d^l(beta) = D^l of the rotation by beta about the y axis (real)."""
    _, Jy, _ = _j(l)
    return expm(-1j * beta * Jy).real


def quat_mul(p, q) -> np.ndarray:
    """Hamilton product p q (rotation R(p) R(q))."""
    pw, px, py, pz = p
    qw, qx, qy, qz = q
    return np.array([
        pw * qw - px * qx - py * qy - pz * qz,
        pw * qx + px * qw + py * qz - pz * qy,
        pw * qy - px * qz + py * qw + pz * qx,
        pw * qz + px * qy - py * qx + pz * qw,
    ])


def quat_conj(q) -> np.ndarray:
    return np.array([q[0], -q[1], -q[2], -q[3]], dtype=np.float64)


def quat_to_matrix(q) -> np.ndarray:
    """3x3 rotation matrix of a unit quaternion (w, x, y, z)."""
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def axis_rotation(axis: int, eps: float) -> np.ndarray:
    """Quaternion of the rotation by eps about coordinate axis 0=x, 1=y, 2=z."""
    q = np.zeros(4)
    q[0] = math.cos(eps / 2)
    q[1 + axis] = math.sin(eps / 2)
    return q


def geodesic_angle(q1, q2) -> float:
    """Angle (radians) of the rotation R(q1)^T R(q2)."""
    d = abs(float(np.dot(np.asarray(q1, float), np.asarray(q2, float))))
    return 2.0 * math.acos(min(1.0, d))
