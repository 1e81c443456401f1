"""Pins of the oracle's score, gradient and marching ascent (Eq. 2, Sec. II-C).  CPU only."""
import math

import numpy as np
import pytest

from oracle import align, ball, wigner
from oracle.wigner import quat_conj, quat_mul
from paper_2509_01180_gb300 import synth
from tests.test_oracle_basis import ball_quadrature
from tests.test_oracle_wigner import rand_quats


@pytest.fixture(scope="module")
def small():
    Bs = ball.make_basis(6, 6 * math.pi)
    rng = np.random.default_rng(11)
    t = rng.normal(size=Bs.Nb) + 1j * rng.normal(size=Bs.Nb)
    f = rng.normal(size=Bs.Nb) + 1j * rng.normal(size=Bs.Nb)
    return Bs, t, f


def test_score_at_identity_is_coefficient_inner_product(small):
    Bs, t, f = small
    xi = align.build_xi(Bs, t, f)
    assert abs(align.score(xi, [1, 0, 0, 0], Bs.Lmax) - np.real(np.vdot(t, f))) < 1e-10


def test_score_is_eq1_inner_product_of_rotated_volume():
    """Eq. 2 equals Eq. 1 at s = 0: <t, R f> computed by quadrature of the synthesised functions."""
    Bs = ball.make_basis(3, 3.5 * math.pi)
    rng = np.random.default_rng(12)
    ct = rng.normal(size=Bs.Nb) + 1j * rng.normal(size=Bs.Nb)
    cf = rng.normal(size=Bs.Nb) + 1j * rng.normal(size=Bs.Nb)
    pts, W = ball_quadrature(100, 3)
    tv = ball.psi_at(Bs, pts) @ ct
    for q in rand_quats(2, 13):
        Rinv = wigner.quat_to_matrix(q).T
        fv_rot = ball.psi_at(Bs, pts @ Rinv.T) @ cf
        ref = np.real(np.sum(W * np.conj(tv) * fv_rot))
        xi = align.build_xi(Bs, ct, cf)
        assert abs(align.score(xi, q, Bs.Lmax) - ref) < 1e-9 * max(1, abs(ref))


def test_gradient_matches_central_differences(small):
    Bs, t, f = small
    xi = align.build_xi(Bs, t, f)
    eps = 1e-5
    for q in rand_quats(3, 14):
        S, g = align.score_grad(xi, q, Bs.Lmax)
        assert abs(S - align.score(xi, q, Bs.Lmax)) < 1e-12 * max(1, abs(S))
        for i in range(3):
            qp = quat_mul(q, wigner.axis_rotation(i, eps))
            qm = quat_mul(q, wigner.axis_rotation(i, -eps))
            fd = (align.score(xi, qp, Bs.Lmax) - align.score(xi, qm, Bs.Lmax)) / (2 * eps)
            assert abs(fd - g[i]) < 1e-7 * max(1.0, np.linalg.norm(g)), (i, fd, g[i])


def test_maximum_at_known_rotation(small):
    """For exactly rotated coefficients f_hat = D(R) t_hat, max_R Eq. 2 = ||t_hat||^2 at R^{-1}."""
    Bs, t, _ = small
    q_true = rand_quats(1, 15)[0]
    f = align.rotate_coeffs(Bs, t, q_true)
    xi = align.build_xi(Bs, t, f)
    S, g = align.score_grad(xi, quat_conj(q_true), Bs.Lmax)
    assert abs(S - np.vdot(t, t).real) < 1e-9 * np.vdot(t, t).real
    assert np.linalg.norm(g) < 1e-8 * S
    for q in rand_quats(20, 16):
        assert align.score(xi, q, Bs.Lmax) < S


def test_ascent_recovers_exact_rotation(small):
    Bs, t, _ = small
    q_true = rand_quats(1, 17)[0]
    f = align.rotate_coeffs(Bs, t, q_true)
    starts = rand_quats(6, 18)
    res = align.align_particle(Bs, t, f, starts, [2, 4, 6], 40)
    assert wigner.geodesic_angle(res.q, quat_conj(q_true)) < 1e-3
    assert abs(res.score - np.vdot(t, t).real) < 1e-6 * np.vdot(t, t).real


def so3_grid(n_axis_angles):
    """Brute-force SO(3) grid: ZYZ Euler angles on a regular lattice."""
    a = np.linspace(0, 2 * np.pi, n_axis_angles, endpoint=False)
    b = np.arccos(np.linspace(1, -1, n_axis_angles // 2 + 1))
    qs = []
    for al in a:
        for be in b:
            for ga in a:
                qa, qb, qc = wigner.axis_rotation(2, al), wigner.axis_rotation(1, be), wigner.axis_rotation(2, ga)
                qs.append(quat_mul(quat_mul(qa, qb), qc))
    return np.array(qs)


def test_brute_force_grid_agrees_with_ascent():
    """Exhaustive evaluation on a grid (Sec. II-C: the most accurate, most expensive way) vs the ascent."""
    Bs = ball.make_basis(3, 4 * math.pi)
    rng = np.random.default_rng(19)
    t = rng.normal(size=Bs.Nb) + 1j * rng.normal(size=Bs.Nb)
    f = align.rotate_coeffs(Bs, t, rand_quats(1, 20)[0]) + 0.3 * (rng.normal(size=Bs.Nb) + 1j * rng.normal(size=Bs.Nb))
    xi = align.build_xi(Bs, t, f)
    grid = so3_grid(24)
    Dl = [np.array([wigner.wigner_D(l, q) for q in grid]) for l in range(4)]
    sc = sum(np.real(np.einsum("mn,gmn->g", xi[l], Dl[l])) for l in range(4))
    gbest = grid[int(np.argmax(sc))]
    res = align.align_particle(Bs, t, f, rand_quats(8, 21), [1, 2, 3], 60)
    assert res.score >= sc.max() - 1e-9
    assert wigner.geodesic_angle(res.q, gbest) < math.radians(15.0)  # grid spacing 15 degrees


def test_selection_tie_goes_to_lowest_index():
    assert align.select_best(np.array([1.0, 3.0, 3.0, 2.0])) == 1
    assert align.select_best(np.array([5.0, 5.0 * (1 + 1e-14), 4.0])) == 0
    assert align.select_best(np.array([-2.0, -1.0])) == 1


def test_energy_ratio():
    xi = [np.full((2 * l + 1, 2 * l + 1), 1.0 + 0j) for l in range(3)]  # |xi^l|^2 sums: 1, 9, 25
    r = align.energy_ratio(xi)
    assert np.allclose(r, [34 / 35, 25 / 35, 0.0])


def _xi_with_energies(e):
    """xi^l with sum_{m,m'} |xi^l_{mm'}|^2 = e[l] (constant entries)."""
    return [np.full((2 * l + 1, 2 * l + 1), math.sqrt(e[l]) / (2 * l + 1) + 0j) for l in range(len(e))]


def test_band_choice_hand_example():
    """Energies 8, 4, 2, 1, 1 over l = 0..4 (total 16): Ratio(L) = 8/16, 4/16, 2/16, 1/16, 0 for L = 0..4.
    Thresholds 0.3, 0.1, 0.01: the first L with Ratio <= 0.3 is 1 (0.25), with <= 0.1 it is 3 (0.0625), with
    <= 0.01 it is 4 (0).  A lowest band of 2 moves the first band to 2; thresholds that pick the same band
    give it once."""
    xi = _xi_with_energies([8.0, 4.0, 2.0, 1.0, 1.0])
    assert np.allclose(align.energy_ratio(xi), [0.5, 0.25, 0.125, 0.0625, 0.0])
    assert align.choose_bands(xi, [0.3, 0.1, 0.01]) == [1, 3, 4]
    assert align.choose_bands(xi, [0.3, 0.1, 0.01], L_min=2) == [2, 3, 4]
    assert align.choose_bands(xi, [0.3, 0.26, 0.2]) == [1, 2]
    assert align.choose_bands(xi, [0.25, 0.0625]) == [1, 3]  # Ratio equal to the threshold qualifies
    assert align.choose_bands(xi, [0.9]) == [1]  # bands start at 1 even when Ratio(0) is below tau


def test_marching_on_noiseless_voxel_phantom():
    """Plain method, FP64, one noiseless 16^3 pair (l <= 8, 2-4-8, 8 starts, 50 steps): the recovered
    rotation is R_true^{-1} up to the voxelisation and truncation bias (reported, loosely gated)."""
    w = synth.make_workload("pair16")
    Bs = ball.make_basis(w.Lmax, w.lam_max)
    t = ball.expand(Bs, w.template.astype(np.float64))[0]
    f = ball.expand(Bs, w.vols[0].astype(np.float64))[0]
    res = align.align_particle(Bs, t, f, w.starts[0].astype(np.float64), w.stages, w.steps)
    err = math.degrees(wigner.geodesic_angle(res.q, quat_conj(w.q_true[0])))
    assert err < 3.0, err


def test_shift_search_recovers_shift_and_rotation():
    """Eq. 1 over a shift grid: a noiseless phantom rotated by R and displaced by s_true is matched at
    s_true (f_s(x) = f(x + s) undoes the displacement) with R close to R_true^{-1}."""
    w = synth.make_workload("pair16")
    tpl = synth.blob_template(synth.rng_for(1, 0), 20, 1.2, 6.0)
    s_true = (1, 0, -1)
    vol = synth.render(16, tpl, w.q_true[0], offset=s_true)
    Bs = ball.make_basis(8, 8 * math.pi)
    t = ball.expand(Bs, synth.render(16, tpl))[0]
    shifts = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 0, -1), (1, 0, -1), (-1, 0, 1)]
    res = align.align_shifts(Bs, t, vol, shifts, w.starts[0].astype(np.float64), [2, 4, 8], 30)
    assert shifts[res.shift] == s_true
    assert math.degrees(wigner.geodesic_angle(res.q, quat_conj(w.q_true[0]))) < 3.0


def _exp_step(q, eps):
    """q * exp(eps.J) for a rotation vector eps (body frame)."""
    n = float(np.linalg.norm(eps))
    if n == 0:
        return np.asarray(q, np.float64)
    return quat_mul(q, np.array([math.cos(n / 2), *(math.sin(n / 2) * np.asarray(eps) / n)]))


def test_hessian_matches_mixed_differences(small):
    """H = second derivatives of f(eps) = S(R exp(eps.J)) at 0, by central and mixed differences of S."""
    Bs, t, f = small
    xi = align.build_xi(Bs, t, f)
    h = 1e-4
    for q in rand_quats(3, 51):
        S, g, H = align.score_grad_hess(xi, q, Bs.Lmax)
        assert np.allclose(H, H.T, atol=0)
        fq = lambda e: align.score(xi, _exp_step(q, e), Bs.Lmax)  # noqa: E731
        E = np.eye(3) * h
        ref = np.zeros((3, 3))
        for i in range(3):
            ref[i, i] = (fq(E[i]) - 2 * S + fq(-E[i])) / h ** 2
            for j in range(i + 1, 3):
                ref[i, j] = ref[j, i] = (fq(E[i] + E[j]) - fq(E[i] - E[j]) - fq(E[j] - E[i]) + fq(-E[i] - E[j])) / (4 * h * h)
        scale = max(1.0, np.abs(H).max())
        assert np.abs(H - ref).max() < 1e-5 * scale, (H, ref)


def test_hessian_negative_definite_at_known_maximum(small):
    Bs, t, _ = small
    q_true = rand_quats(1, 52)[0]
    xi = align.build_xi(Bs, t, align.rotate_coeffs(Bs, t, q_true))
    S, g, H = align.score_grad_hess(xi, quat_conj(q_true), Bs.Lmax)
    assert np.linalg.norm(g) < 1e-8 * S
    assert np.linalg.eigvalsh(H).max() < 0


def test_newton_converges_quadratically(small):
    """From 4 degrees off the exact maximum, Newton steps reach it to 1e-10 rad in a few iterations, where the
    gradient ascent with the same number of steps is still far (linear convergence)."""
    Bs, t, _ = small
    q_true = rand_quats(1, 53)[0]
    xi = align.build_xi(Bs, t, align.rotate_coeffs(Bs, t, q_true))
    target = quat_conj(q_true)
    q0 = _exp_step(target, np.radians(4.0) * np.array([0.6, -0.48, 0.64]))
    r_n = align.newton(xi, q0, [Bs.Lmax], 6)
    r_g = align.ascend(xi, q0, [Bs.Lmax], 6)
    assert wigner.geodesic_angle(r_n.q, target) < 1e-10
    assert wigner.geodesic_angle(r_g.q, target) > 1e-6


def test_newton_marching_recovers_exact_rotation(small):
    Bs, t, _ = small
    q_true = rand_quats(1, 54)[0]
    f = align.rotate_coeffs(Bs, t, q_true)
    res = align.align_particle(Bs, t, f, rand_quats(6, 55), [2, 4, 6], 15, method="newton")
    assert wigner.geodesic_angle(res.q, quat_conj(q_true)) < 1e-8
    assert abs(res.score - np.vdot(t, t).real) < 1e-9 * np.vdot(t, t).real
