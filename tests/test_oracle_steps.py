"""Pins of the oracle's step control (Sec. II-C gradient ascent with marching; Sec. III Newton steps),
hand-traced on an objective whose every step has a closed form.  CPU only.

Objective: xi^0 = 0, xi^1 = I (3 x 3) and xi^2 = 0, so Eq. 2 is S(R) = Re tr D^1(R) = 1 + 2 cos(theta), the
character of degree 1 (theta = rotation angle), and S depends on theta alone.  For R = rotation by theta
about a unit axis a (theta in (-pi, pi)), the body-frame gradient is g = -2 sin(theta) a, and the Hessian
along R exp(eps u) is H = 2 sin^2(theta/2) a a^T - 2 cos^2(theta/2) I (eigenvalue -2 cos(theta) along a).
So every step stays on the axis a:
  * ascent: the trial rotation R exp(h u.J), u = g/|g| = -sign(theta) a, has angle theta - h sign(theta);
    it is accepted iff |theta - h sign(theta)| < |theta|;
  * Newton: where -H is positive definite (cos(theta) > 0) d = -H^{-1} g = -tan(theta) a, else the gradient
    step of length pi/(2L) along -sign(theta) a; |d| is clipped to pi/L and scaled by the damping lam.
The expected angles below were traced by hand from the step rule (h0 = pi/(2L), hmax = pi/L, x1.5 on accept,
x1/2 on reject, h restarted per band; Newton: lam = 1 per band, min(1, 2 lam) on accept, lam/2 on reject).
"""
import math

import numpy as np
import pytest

from oracle import align

AXIS = np.array([1.0, 2.0, 2.0]) / 3.0


def xi_character():
    """xi^0 = 0, xi^1 = I, xi^2 = 0 (so the band-2 stage sees the same objective)."""
    return [np.zeros((1, 1), dtype=np.complex128), np.eye(3, dtype=np.complex128), np.zeros((5, 5), dtype=np.complex128)]


def q_of(theta):
    return np.array([math.cos(theta / 2), *(math.sin(theta / 2) * AXIS)])


def signed_angle(q):
    """Angle of q about AXIS (q must lie on that axis)."""
    q = np.asarray(q, dtype=np.float64)
    v = q[1:]
    assert np.linalg.norm(v - np.dot(v, AXIS) * AXIS) < 1e-12  # still a rotation about AXIS
    return 2.0 * math.atan2(float(np.dot(v, AXIS)), float(q[0]))


def test_character_objective():
    """The closed forms the traces rest on: S = 1 + 2 cos(theta), g = -2 sin(theta) a."""
    xi = xi_character()
    for th in (2.0, 0.4, -1.1):
        S, g = align.score_grad(xi, q_of(th), 1)
        assert abs(S - (1 + 2 * math.cos(th))) < 1e-12
        assert np.allclose(g, -2 * math.sin(th) * AXIS, atol=1e-12)
        _, _, H = align.score_grad_hess(xi, q_of(th), 1)
        ref = 2 * math.sin(th / 2) ** 2 * np.outer(AXIS, AXIS) - 2 * math.cos(th / 2) ** 2 * np.eye(3)
        assert np.allclose(H, ref, atol=1e-12)


# ascent from theta0 = 2, band 1 (h0 = pi/2, hmax = pi):
#   step 1: h = pi/2    trial 2 - pi/2 = 0.429      accept, h -> 3pi/4
#   step 2: h = 3pi/4   trial -1.927                reject, h -> 3pi/8
#   step 3: h = 3pi/8   trial -0.749                reject, h -> 3pi/16
#   step 4: h = 3pi/16  trial 2 - 11pi/16 = -0.160  accept, h -> 9pi/32
#   step 5: h = 9pi/32  trial 0.724                 reject, h -> 9pi/64
# band 2 (h restarts at pi/4, hmax = pi/2):
#   step 1: h = pi/4    trial 0.626 reject;  step 2: h = pi/8  trial 0.233 reject;
#   step 3: h = pi/16   trial 2 - 5pi/8 = 0.0365 accept, h -> 3pi/32;
#   step 4: h = 3pi/32  trial -0.258 reject;  step 5: h = 3pi/64  trial -0.111 reject
ASCENT_BAND1 = [2 - math.pi / 2, 2 - math.pi / 2, 2 - math.pi / 2, 2 - 11 * math.pi / 16, 2 - 11 * math.pi / 16]
ASCENT_ACCEPTED = [1, 1, 1, 2, 2]


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_ascent_steps_band1(k):
    r = align.ascend(xi_character(), q_of(2.0), [1], k)
    assert abs(signed_angle(r.q) - ASCENT_BAND1[k - 1]) < 1e-9, (k, signed_angle(r.q))
    assert r.accepted == ASCENT_ACCEPTED[k - 1] and r.evals == 1 + k


def test_ascent_two_bands():
    r = align.ascend(xi_character(), q_of(2.0), [1, 2], 5)
    assert abs(signed_angle(r.q) - (2 - 5 * math.pi / 8)) < 1e-9, signed_angle(r.q)
    assert r.accepted == 3 and r.evals == 2 + 10
    assert abs(r.score - (1 + 2 * math.cos(2 - 5 * math.pi / 8))) < 1e-12


# Newton from theta0 = 1.3 (cos > 0: -H positive definite), band 1 (hmax = pi):
#   it 1: d = tan(1.3) = 3.60 clipped to pi, lam 1: trial 1.3 - pi    reject, lam -> 1/2
#   it 2: same d, lam 1/2: trial 1.3 - pi/2 = -0.271                   accept, lam -> 1
#   it 3: d = -tan(theta): trial theta - tan(theta) = 0.00682          accept
# band 2 after one band-1 iteration: lam restarts at 1, |d| clipped to pi/2: trial 1.3 - pi/2.
# From theta0 = 2 (cos < 0: gradient step pi/2): 2 - pi/2 = 0.429, then the Newton step with lam 1:
# 0.429 - tan(0.429) = -0.0285.
NEWTON_BAND1 = [1.3, 1.3 - math.pi / 2, (1.3 - math.pi / 2) - math.tan(1.3 - math.pi / 2)]


@pytest.mark.parametrize("k", [1, 2, 3])
def test_newton_steps_band1(k):
    r = align.newton(xi_character(), q_of(1.3), [1], k)
    assert abs(signed_angle(r.q) - NEWTON_BAND1[k - 1]) < 1e-9, (k, signed_angle(r.q))


def test_newton_damping_restarts_per_band():
    r = align.newton(xi_character(), q_of(1.3), [1, 2], 1)
    assert abs(signed_angle(r.q) - (1.3 - math.pi / 2)) < 1e-9, signed_angle(r.q)


def test_newton_gradient_step_then_newton_step():
    t1 = 2 - math.pi / 2
    for k, ref in ((1, t1), (2, t1 - math.tan(t1))):
        r = align.newton(xi_character(), q_of(2.0), [1], k)
        assert abs(signed_angle(r.q) - ref) < 1e-9, (k, signed_angle(r.q))
