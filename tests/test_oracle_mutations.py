"""Planted mistakes: each plausible error in the oracle must fail one of its pins (CPU only).

The mistakes are planted in the oracle (monkeypatched), never in the CUDA path."""
import math

import numpy as np
import pytest

from oracle import align, ball, wigner
from tests import test_oracle_align as ta
from tests import test_oracle_basis as tb
from tests import test_oracle_wigner as tw


def _fails(fn, *a):
    try:
        fn(*a)
    except AssertionError:
        return True
    return False


@pytest.mark.parametrize("mutant", ["transpose", "conjugate", "inverse"])
def test_steerability_pin_catches_wrong_D_convention(monkeypatch, mutant):
    orig = wigner.wigner_D

    def bad(l, q):
        D = orig(l, q)
        return {"transpose": D.T, "conjugate": D.conj(), "inverse": D.conj().T}[mutant]

    monkeypatch.setattr(wigner, "wigner_D", bad)
    monkeypatch.setattr(align, "wigner_D", bad)
    assert _fails(tw.test_steerability_exact_rotation)


def test_gradient_pin_catches_sign_error(monkeypatch):
    orig = wigner._j

    def bad(l):
        Jx, Jy, Jz = orig(l)
        return Jx, -Jy, Jz

    monkeypatch.setattr(align, "_j", bad)
    Bs = ball.make_basis(4, 5 * math.pi)
    rng = np.random.default_rng(1)
    small = (Bs, rng.normal(size=Bs.Nb) + 1j * rng.normal(size=Bs.Nb), rng.normal(size=Bs.Nb) + 1j * rng.normal(size=Bs.Nb))
    assert _fails(ta.test_gradient_matches_central_differences, small)


def test_orthonormality_pin_catches_wrong_constant(monkeypatch):
    monkeypatch.setattr(ball, "norm_const", lambda l, lam: 1.0 / abs(float(ball.sph_jn(l + 1, lam))))
    assert _fails(tb.test_ball_basis_orthonormal)


def test_ylm_pin_catches_missing_condon_shortley_phase(monkeypatch):
    orig = ball.assoc_legendre_normalized

    def bad(L, x):
        P = orig(L, x)
        for m in range(L + 1):
            P[:, m] *= (-1) ** m
        return P

    monkeypatch.setattr(ball, "assoc_legendre_normalized", bad)
    assert _fails(tb.test_ylm_closed_forms)


def test_xi_pin_catches_swapped_conjugation(monkeypatch):
    orig = align.build_xi

    def bad(basis, t, f, L=None):
        return orig(basis, np.conj(t), np.conj(f), L)

    monkeypatch.setattr(align, "build_xi", bad)
    assert _fails(ta.test_score_is_eq1_inner_product_of_rotated_volume)


@pytest.mark.parametrize("mutant", ["one_sided", "sign", "no_half"])
def test_hessian_pin_catches_mistakes(monkeypatch, mutant):
    def bad(xi, q, L):
        S, g = align.score_grad(xi, q, L)
        H = np.zeros((3, 3))
        for l in range(L + 1):
            D = wigner.wigner_D(l, q)
            J = wigner._j(l)
            for i in range(3):
                for k in range(3):
                    sym = J[i] @ J[k] + J[k] @ J[i]
                    prod = {"one_sided": J[i] @ J[k], "sign": -sym / 2, "no_half": sym}[mutant]
                    H[i, k] -= float(np.real(np.sum(xi[l] * (D @ prod))))
        return S, g, H

    monkeypatch.setattr(align, "score_grad_hess", bad)
    Bs = ball.make_basis(4, 5 * math.pi)
    rng = np.random.default_rng(2)
    small = (Bs, rng.normal(size=Bs.Nb) + 1j * rng.normal(size=Bs.Nb), rng.normal(size=Bs.Nb) + 1j * rng.normal(size=Bs.Nb))
    assert _fails(ta.test_hessian_matches_mixed_differences, small)


# ---------------------------------------------------------------------------- step control (Sec. II-C, Sec. III)
def _mutant(module, name, old, new):
    """`module.name` recompiled from its source with one text change (the planted mistake)."""
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(getattr(module, name)))
    assert src.count(old) == 1, old
    ns = dict(vars(module))
    exec(compile(src.replace(old, new), f"<mutant of {name}>", "exec"), ns)
    return ns[name]


def _step_pins_fail(kind):
    from tests import test_oracle_steps as ts
    if kind == "ascend":
        runs = [(ts.test_ascent_steps_band1, k) for k in range(1, 6)] + [(ts.test_ascent_two_bands,)]
    else:
        runs = [(ts.test_newton_steps_band1, k) for k in range(1, 4)] + [
            (ts.test_newton_damping_restarts_per_band,), (ts.test_newton_gradient_step_then_newton_step,)]
    return any(_fails(*r) for r in runs)


@pytest.mark.parametrize("old,new", [
    ("h = min(1.5 * h, hmax)", "h = min(2.0 * h, hmax)"),                       # growth x2 instead of x1.5
    ("h = h / 2", "h = h / 4"),                                                 # shrink x1/4 instead of x1/2
    ("        h = h0\n", "        h = h if L != stages[0] else h0\n"),          # no restart of h per band
    ("math.pi / (2 * L), math.pi / L", "math.pi / (2 * L), math.pi / (2 * L)"),  # hmax = pi/(2L)
    ("math.pi / (2 * L), math.pi / L", "math.pi / L, math.pi / L"),              # h0 = pi/L
])
def test_step_pins_catch_ascent_mistakes(monkeypatch, old, new):
    monkeypatch.setattr(align, "ascend", _mutant(align, "ascend", old, new))
    assert _step_pins_fail("ascend")


@pytest.mark.parametrize("old,new", [
    ("lam = min(1.0, 2 * lam)", "lam = 2 * lam"),                              # damping not capped at 1
    ("lam = lam / 2", "lam = lam / 4"),                                        # shrink x1/4 instead of x1/2
    ("        lam = 1.0\n", "        lam = lam if L != stages[0] else 1.0\n"),  # no restart of lam per band
    ("math.pi / (2 * L), math.pi / L", "math.pi / (2 * L), math.pi / (2 * L)"),  # clip at pi/(2L)
    ("if np.linalg.eigvalsh(H).max() < 0:", "if True:"),                        # Newton step without the test
])
def test_step_pins_catch_newton_mistakes(monkeypatch, old, new):
    monkeypatch.setattr(align, "newton", _mutant(align, "newton", old, new))
    assert _step_pins_fail("newton")


# ---------------------------------------------------------------------------- DFT power of the template (Sec. II-B)
@pytest.mark.parametrize("old,new", [
    ("tb[flat] = np.asarray(tvol, np.float64).ravel()[flat]", "tb[:] = np.asarray(tvol, np.float64).ravel()"),  # no ball
    ("sel = (r > 0) & (r < N / 2)", "sel = (r > 0) & (r <= N / 2)"),            # |k| = N/2 kept
    ('kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")', 'kx, ky, kz = np.meshgrid(k, k, k, indexing="ij")'),  # axes
])
def test_dft_power_pin_catches_mistakes(monkeypatch, old, new):
    from oracle import wedge
    from tests import test_oracle_wedge as twd
    monkeypatch.setattr(wedge, "dft_power", _mutant(wedge, "dft_power", old, new))
    assert _fails(twd.test_dft_power_is_the_direct_dft_of_the_ball_restricted_volume)


# ---------------------------------------------------------------------------- band choice (Fig. 1, Sec. III)
@pytest.mark.parametrize("old,new", [
    ("if r[L] <= tau)", "if r[L] < tau)"),                      # strict comparison
    ("range(L_min, Lmax + 1)", "range(0, Lmax + 1)"),           # band 0 allowed
    ("if not bands or L > bands[-1]:", "if True:"),             # repeats kept
    ("if r[L] <= tau)", "if 1.0 - r[L] <= tau)"),               # captured instead of remaining energy
])
def test_band_choice_pin_catches_mistakes(monkeypatch, old, new):
    monkeypatch.setattr(align, "choose_bands", _mutant(align, "choose_bands", old, new))
    try:
        ta.test_band_choice_hand_example()
    except (AssertionError, StopIteration):  # a wrong band, or no band found at all
        return
    raise AssertionError("the planted mistake passed the pin")
