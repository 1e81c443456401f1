"""Pins of the oracle's missing-wedge constrained correlation (Sec. II-B).  CPU only."""
import math

import numpy as np
import pytest

from oracle import align, ball, wedge, wigner
from oracle.wigner import quat_conj, quat_mul
from paper_2509_01180_gb300 import synth
from tests.test_oracle_wigner import rand_quats


@pytest.fixture(scope="module")
def pair():
    w = synth.make_workload("pair16")
    return w, wedge.make_wedge(w.template.astype(np.float64), 60.0, 8)


def test_wedge_coefficient_l0_is_the_sampled_area():
    """The sampled directions |k_z| <= tan(a)|k_x| cover the fraction 2a/pi of the sphere: w_00 = 8a/sqrt(4 pi)."""
    for a in (30.0, 60.0, 75.0):
        w = wedge.wedge_sh(4, a)
        assert abs(w[0][0] - 8 * math.radians(a) / math.sqrt(4 * math.pi)) < 1e-12


def test_wedge_coefficients_match_direct_quadrature():
    """Against a dense product rule over the indicator itself (no change of variables; error ~1e-4 from
    the discontinuity)."""
    L, a = 6, 60.0
    w = wedge.wedge_sh(L, a)
    x, wx = np.polynomial.legendre.leggauss(500)
    nph = 1000
    ph = (np.arange(nph) + 0.5) * 2 * math.pi / nph
    X, PH = np.meshgrid(x, ph, indexing="ij")
    st = np.sqrt(1 - X ** 2)
    dirs = np.stack([st * np.cos(PH), st * np.sin(PH), X], -1).reshape(-1, 3)
    wts = (wx[:, None] * np.full((1, nph), 2 * math.pi / nph)).ravel() * wedge.wedge_indicator(dirs, a)
    Y = ball.sph_harm_all(L, dirs)
    for l in range(L + 1):
        ref = np.conj(Y[l]).T @ wts
        assert np.abs(ref - w[l]).max() < 2e-3, (l, ref, w[l])


def test_denominator_equals_the_sum_over_dft_samples(pair):
    """Dn(R) from the Wigner sum equals sum_k W_L(R^{-1} k^) |T(k)|^2 + |T(0)|^2 with W_L synthesised
    directly from its coefficients at the rotated directions."""
    w, wd = pair
    dirs, pw, c0 = wedge.dft_power(w.template.astype(np.float64))
    L = 8
    for q in rand_quats(3, 61):
        rd = dirs @ wigner.quat_to_matrix(q)  # rows: R^{-1} k^
        Y = ball.sph_harm_all(L, rd)
        WL = sum(Y[l] @ wd.w[l] for l in range(L + 1)).real
        Dn, _ = wedge.denominator(wd, q, L)
        assert abs(c0 + float(np.sum(WL * pw)) - Dn) < 1e-11 * Dn


def test_denominator_has_the_wedge_symmetries(pair):
    """The sampled region is invariant under pi rotations about x, y and z, so Dn(R Q) = Dn(R) for those Q."""
    _, wd = pair
    for q in rand_quats(2, 62):
        D0, _ = wedge.denominator(wd, q, 8)
        for ax in range(3):
            D1, _ = wedge.denominator(wd, quat_mul(q, wigner.axis_rotation(ax, math.pi)), 8)
            assert abs(D1 - D0) < 1e-10 * D0


def test_denominator_approaches_the_sharp_wedge(pair):
    """With the indicator itself in place of W_L the sum is ||W_R t||^2; the band-limited form tends to it."""
    w, _ = pair
    dirs, pw, c0 = wedge.dft_power(w.template.astype(np.float64))
    q = rand_quats(1, 63)[0]
    sharp = c0 + float(np.sum(wedge.wedge_indicator(dirs @ wigner.quat_to_matrix(q), 60.0) * pw))
    errs = []
    for L in (4, 8, 16):
        wd = wedge.make_wedge(w.template.astype(np.float64), 60.0, L)
        errs.append(abs(wedge.denominator(wd, q, L)[0] - sharp) / sharp)
    assert errs[-1] < errs[0] and errs[-1] < 0.05, errs


def test_constrained_gradient_matches_central_differences(pair):
    w, wd = pair
    Bs = ball.make_basis(8, 8 * math.pi)
    t = ball.expand(Bs, w.template.astype(np.float64))[0]
    f = ball.expand(Bs, w.vols[0].astype(np.float64))[0]
    xi = align.build_xi(Bs, t, f)
    eps = 1e-5
    for q in rand_quats(3, 64):
        C, g = wedge.constrained_score_grad(xi, wd, q, 8)
        for i in range(3):
            cp, _ = wedge.constrained_score_grad(xi, wd, quat_mul(q, wigner.axis_rotation(i, eps)), 8)
            cm, _ = wedge.constrained_score_grad(xi, wd, quat_mul(q, wigner.axis_rotation(i, -eps)), 8)
            assert abs((cp - cm) / (2 * eps) - g[i]) < 1e-7 * max(1.0, np.linalg.norm(g))


def test_constrained_ascent_recovers_a_wedged_phantom():
    """Noiseless phantom with a +-60 deg missing wedge: the constrained ascent finds R_true^{-1}."""
    w = synth.make_workload("pair16", snr=None, wedge=60.0)
    wd = wedge.make_wedge(w.template.astype(np.float64), 60.0, 8)
    Bs = ball.make_basis(8, 8 * math.pi)
    t = ball.expand(Bs, w.template.astype(np.float64))[0]
    f = ball.expand(Bs, w.vols[0].astype(np.float64))[0]
    res = wedge.align_constrained(Bs, t, f, wd, w.starts[0].astype(np.float64), [2, 4, 8], 40)
    assert math.degrees(wigner.geodesic_angle(res.q, quat_conj(w.q_true[0]))) < 5.0


@pytest.mark.parametrize("mutant", ["one_arc", "conj_q"])
def test_wedge_pins_catch_mistakes(monkeypatch, mutant, pair):
    if mutant == "one_arc":  # the phi integral keeps only one of the two sampled arcs for m != 0
        orig = wedge.wedge_sh

        def bad(L, a, n_gl=96):
            w = orig(L, a, n_gl)
            for l in range(L + 1):
                w[l] = np.array([v if m == 0 else v / 2 for m, v in zip(range(-l, l + 1), w[l])])
            return w

        monkeypatch.setattr(wedge, "wedge_sh", bad)
        with pytest.raises(AssertionError):
            test_wedge_coefficients_match_direct_quadrature()
    else:
        w, wd = pair
        bad = wedge.Wedge(wd.L, [np.conj(x) for x in wd.q], wd.w, wd.c0)
        with pytest.raises(AssertionError):
            test_denominator_equals_the_sum_over_dft_samples((w, bad))


def direct_dft_power(vol: np.ndarray):
    """|T(k)|^2 by the definition T(k) = sum_{voxels v in the ball} t(v) exp(-2 pi i k.v / N), for every integer
    frequency vector k = (kx, ky, kz) in [-N/2, N/2)^3 with 0 < |k| < N/2 (kx along the array's last axis),
    returned as rows (k/|k|, |T(k)|^2), and |T(0)|^2.  O(N^6), for tiny N only."""
    N = vol.shape[0]
    h = N // 2
    rows = []
    idx = np.arange(N)
    z, y, x = np.meshgrid(idx, idx, idx, indexing="ij")
    ball = (x - h) ** 2 + (y - h) ** 2 + (z - h) ** 2 < h * h
    tv, xs, ys, zs = vol[ball], x[ball], y[ball], z[ball]
    for kz in range(-h, h):
        for ky in range(-h, h):
            for kx in range(-h, h):
                r2 = kx * kx + ky * ky + kz * kz
                if r2 == 0 or r2 >= h * h:
                    continue
                T = np.sum(tv * np.exp(-2j * np.pi * (kx * xs + ky * ys + kz * zs) / N))
                r = math.sqrt(r2)
                rows.append((kx / r, ky / r, kz / r, abs(T) ** 2))
    return np.array(rows), abs(np.sum(tv)) ** 2


def test_dft_power_is_the_direct_dft_of_the_ball_restricted_volume():
    """dft_power against the DFT written out on an 8^3 volume with no symmetry (random values): the same
    multiset of (direction, power) pairs, the same count of frequencies, and the same |T(0)|^2."""
    rng = np.random.default_rng(64)
    vol = rng.normal(size=(8, 8, 8)) + np.linspace(0, 1, 8)[None, None, :]  # a ramp along x breaks symmetry
    dirs, pw, c0 = wedge.dft_power(vol)
    ref, c0_ref = direct_dft_power(vol)
    assert len(pw) == len(ref)
    got = np.concatenate([dirs, pw[:, None]], axis=1)
    key = lambda a: np.lexsort((a[:, 3], np.round(a[:, 2], 9), np.round(a[:, 1], 9), np.round(a[:, 0], 9)))
    got, ref = got[key(got)], ref[key(ref)]
    assert np.allclose(got[:, :3], ref[:, :3], atol=1e-12)
    assert np.allclose(got[:, 3], ref[:, 3], rtol=1e-10, atol=1e-10 * ref[:, 3].max())
    assert abs(c0 - c0_ref) < 1e-10 * c0_ref
