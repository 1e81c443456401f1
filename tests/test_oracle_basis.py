"""Pins of the oracle's basis and expansion against what the paper and the mathematics fix (CPU only).

Basis display of Sec. II-A: psi_klm = c_lk j_l(lambda_lk r) Y_l^m chi_[0,1)(r), orthonormal
eigenfunctions of the Dirichlet Laplacian on the unit ball.
"""
import math

import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss
from scipy import special

from oracle import ball


# ---------------------------------------------------------------- spherical Bessel j_l

def test_spherical_bessel_closed_forms():
    x = np.linspace(0.3, 60.0, 97)
    j0 = np.sin(x) / x
    j1 = np.sin(x) / x ** 2 - np.cos(x) / x
    j2 = (3 / x ** 2 - 1) * np.sin(x) / x - 3 * np.cos(x) / x ** 2
    for l, ref in ((0, j0), (1, j1), (2, j2)):
        assert np.allclose(ball.sph_jn(l, x), ref, rtol=0, atol=1e-14)


@pytest.mark.parametrize("l", [0, 3, 8, 16, 24, 32])
def test_spherical_bessel_vs_half_integer_bessel(l):
    # j_l(x) = sqrt(pi / (2x)) J_{l+1/2}(x): a different library routine
    x = np.linspace(0.5, 110.0, 211)
    ref = np.sqrt(np.pi / (2 * x)) * special.jv(l + 0.5, x)
    assert np.allclose(ball.sph_jn(l, x), ref, rtol=1e-9, atol=1e-15)


# ---------------------------------------------------------------- roots lambda_lk

def test_roots_of_j0_are_multiples_of_pi():
    r = ball.bessel_roots(0, 8 * math.pi)
    assert len(r) == 8  # the endpoint k = 8 is included (lambda_max = pi N / 2 at N = 16)
    assert np.allclose(r, math.pi * np.arange(1, 9), rtol=0, atol=1e-13)


@pytest.mark.parametrize("l", [1, 2, 5, 9, 16, 32])
def test_roots_are_zeros(l):
    r = ball.bessel_roots(l, 32 * math.pi)
    assert len(r) > 0
    # |j_l(lambda)| at a simple root ~ |j_l'| * eps * lambda
    assert np.max(np.abs(ball.sph_jn(l, r))) < 1e-13
    # Sturm comparison: for order l + 1/2 > 1/2 consecutive zeros are more than pi apart and
    # their spacing decreases towards pi
    d = np.diff(r)
    assert np.all(d > math.pi) and np.all(np.diff(d) < 0)


def test_roots_interlace():
    # lambda_{l,k} < lambda_{l+1,k} < lambda_{l,k+1}
    lam_max = 20 * math.pi
    roots = [ball.bessel_roots(l, lam_max) for l in range(0, 20)]
    for l in range(19):
        a, b = roots[l], roots[l + 1]
        for k in range(len(b)):
            assert a[k] < b[k]
            if k + 1 < len(a):
                assert b[k] < a[k + 1]


def test_index_set_sizes_match_root_counting():
    # N_b = sum_l K_l (2l+1) with K_l = #{k: lambda_lk <= pi N / 2}; cross-checked with the
    # sign-change count of sqrt(pi/2x) J_{l+1/2} on a fine grid (a different routine).
    for N, L in ((16, 8), (32, 16)):
        lam_max = math.pi * N / 2
        B = ball.make_basis(L, lam_max)
        for l in range(L + 1):
            x = np.arange(max(l, 0.5), lam_max + 1e-9, 1e-3)
            v = special.jv(l + 0.5, x)
            cnt = int(np.sum(v[:-1] * v[1:] < 0))
            if l == 0:  # j_0 has its root k = N/2 exactly at lambda_max
                cnt = N // 2
            assert B.K[l] == cnt, (N, l)
    assert ball.make_basis(8, 8 * math.pi).Nb == 408
    assert ball.make_basis(16, 16 * math.pi).Nb == 3050


# ---------------------------------------------------------------- c_lk and radial orthonormality

@pytest.mark.parametrize("l", [0, 1, 4, 9])
def test_radial_profiles_orthonormal(l):
    # int_0^1 c_lk j_l(lambda_lk r) c_lk' j_l(lambda_lk' r) r^2 dr = delta_kk'
    x, w = leggauss(400)
    r = 0.5 * (x + 1.0)
    w = 0.5 * w * r ** 2
    lam = ball.bessel_roots(l, 12 * math.pi)
    c = np.array([ball.norm_const(l, v) for v in lam])
    R = c[:, None] * ball.sph_jn(l, lam[:, None] * r[None, :])
    G = (R * w[None, :]) @ R.T
    assert np.allclose(G, np.eye(len(lam)), atol=1e-12)


# ---------------------------------------------------------------- spherical harmonics

def _dirs(theta, phi):
    return np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], axis=1)


def test_ylm_closed_forms():
    rng = np.random.default_rng(0)
    th, ph = np.arccos(rng.uniform(-1, 1, 50)), rng.uniform(0, 2 * np.pi, 50)
    Y = ball.sph_harm_all(2, _dirs(th, ph))
    ct, st, e = np.cos(th), np.sin(th), np.exp(1j * ph)
    ref = {
        (0, 0): np.full_like(ct, 0.5 / math.sqrt(math.pi)),
        (1, 0): math.sqrt(3 / (4 * math.pi)) * ct,
        (1, 1): -math.sqrt(3 / (8 * math.pi)) * st * e,
        (1, -1): math.sqrt(3 / (8 * math.pi)) * st / e,
        (2, 0): math.sqrt(5 / (16 * math.pi)) * (3 * ct ** 2 - 1),
        (2, 1): -math.sqrt(15 / (8 * math.pi)) * st * ct * e,
        (2, 2): math.sqrt(15 / (32 * math.pi)) * st ** 2 * e ** 2,
        (2, -2): math.sqrt(15 / (32 * math.pi)) * st ** 2 / e ** 2,
    }
    for (l, m), v in ref.items():
        assert np.allclose(Y[l][:, m + l], v, atol=1e-14), (l, m)


def test_ylm_orthonormal_on_product_quadrature():
    L = 20
    x, wt = leggauss(L + 2)
    nphi = 2 * L + 3
    ph = 2 * np.pi * np.arange(nphi) / nphi
    TH, PH = np.meshgrid(np.arccos(x), ph, indexing="ij")
    W = (wt[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).ravel()
    Y = ball.sph_harm_all(L, _dirs(TH.ravel(), PH.ravel()))
    A = np.concatenate(Y, axis=1)
    G = (A.conj().T * W[None, :]) @ A
    assert np.allclose(G, np.eye(A.shape[1]), atol=1e-12)


def test_ylm_addition_theorem():
    rng = np.random.default_rng(1)
    d = rng.normal(size=(40, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = ball.sph_harm_all(32, d)
    for l in range(33):
        assert np.allclose(np.sum(np.abs(Y[l]) ** 2, axis=1), (2 * l + 1) / (4 * np.pi), rtol=1e-12)


def test_ylm_vs_scipy():
    if not hasattr(special, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    rng = np.random.default_rng(2)
    th, ph = np.arccos(rng.uniform(-1, 1, 30)), rng.uniform(0, 2 * np.pi, 30)
    Y = ball.sph_harm_all(24, _dirs(th, ph))
    for l in (0, 1, 5, 13, 24):
        for m in range(-l, l + 1):
            ref = special.sph_harm_y(l, m, th, ph)
            assert np.allclose(Y[l][:, m + l], ref, atol=1e-12), (l, m)


# ---------------------------------------------------------------- the ball basis

def ball_quadrature(nr, L):
    """Product rule on the unit ball: Gauss-Legendre in r (weight r^2) x in cos(theta) x uniform phi."""
    xr, wr = leggauss(nr)
    r = 0.5 * (xr + 1.0)
    wr = 0.5 * wr * r ** 2
    xt, wt = leggauss(L + 2)
    nphi = 2 * L + 3
    ph = 2 * np.pi * np.arange(nphi) / nphi
    R, CT, PH = np.meshgrid(r, xt, ph, indexing="ij")
    W = (wr[:, None, None] * wt[None, :, None] * np.full(nphi, 2 * np.pi / nphi)[None, None, :]).ravel()
    st = np.sqrt(1 - CT ** 2)
    pts = np.stack([(R * st * np.cos(PH)).ravel(), (R * st * np.sin(PH)).ravel(), (R * CT).ravel()], axis=1)
    return pts, W


def test_ball_basis_orthonormal():
    B = ball.make_basis(5, 5 * math.pi)
    pts, W = ball_quadrature(160, 5)
    P = ball.psi_at(B, pts)
    G = (P.conj().T * W[None, :]) @ P
    assert np.allclose(G, np.eye(B.Nb), atol=1e-10)


def test_voxel_grid_geometry():
    flat, pts = ball.voxel_ball(16)
    assert len(flat) == 2103
    assert np.all(np.linalg.norm(pts, axis=1) < 1.0)
    # voxel (z=8, y=8, x=8) is the centre
    assert np.any(np.all(pts == 0.0, axis=1))
    assert flat[np.flatnonzero(np.all(pts == 0.0, axis=1))[0]] == 8 * 256 + 8 * 16 + 8
    assert len(ball.voxel_ball(32)[0]) == 17071


def test_expand_matches_pointwise_definition():
    # a_klm = h^3 sum_v f(x_v) conj(c_lk j_l(lambda_lk r_v) Y_l^m(x_v)), evaluated one coefficient at a
    # time with scipy's own j_l and Y_l^m (independent of the oracle's Legendre recurrence and layout code)
    if not hasattr(special, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    N = 12
    B = ball.make_basis(4, math.pi * N / 2)
    rng = np.random.default_rng(3)
    vol = rng.normal(size=(N, N, N))
    a = ball.expand(B, vol)[0]
    flat, pts = ball.voxel_ball(N)
    f = vol.ravel()[flat]
    r = np.linalg.norm(pts, axis=1)
    th = np.arccos(np.clip(np.where(r > 0, pts[:, 2] / np.where(r > 0, r, 1), 1.0), -1, 1))
    ph = np.arctan2(pts[:, 1], pts[:, 0])
    h3 = (2.0 / N) ** 3
    for (l, k, m) in [(0, 0, 0), (0, 5, 0), (1, 0, -1), (1, 2, 1), (3, 1, 2), (4, 0, -4), (4, 2, 3)]:
        lam = B.roots[l][k]
        c = math.sqrt(2) / abs(special.spherical_jn(l + 1, lam))
        psi = c * special.spherical_jn(l, lam * r) * special.sph_harm_y(l, m, th, ph)
        ref = h3 * np.sum(f * np.conj(psi))
        got = a[B.offsets[l] + k * (2 * l + 1) + m + l]
        assert abs(got - ref) < 1e-12 * max(1.0, abs(ref)), (l, k, m)


def test_expand_real_volume_conjugate_symmetry():
    B = ball.make_basis(6, 8 * math.pi)
    rng = np.random.default_rng(4)
    a = ball.expand(B, rng.normal(size=(16, 16, 16)))[0]
    for l in range(7):
        blk = ball.split_by_degree(B, a)[l]
        for m in range(1, l + 1):
            assert np.allclose(blk[:, -m + l], (-1) ** m * np.conj(blk[:, m + l]), atol=1e-13)
        assert np.allclose(blk[:, l].imag, 0, atol=1e-13)


def test_expand_is_linear():
    B = ball.make_basis(4, 6 * math.pi)
    rng = np.random.default_rng(5)
    u, v = rng.normal(size=(2, 12, 12, 12))
    a = ball.expand(B, np.stack([u, v, 2 * u - 3 * v]))
    assert np.allclose(a[2], 2 * a[0] - 3 * a[1], atol=1e-12)


def test_voxel_expansion_converges_to_projection():
    # On finer voxel grids the discrete inner product tends to the L2 one: the coefficients of a
    # smooth band-limited function approach its exact coefficients (error reported, decreasing).
    B = ball.make_basis(2, 3 * math.pi)
    rng = np.random.default_rng(6)
    coef = rng.normal(size=B.Nb) + 1j * rng.normal(size=B.Nb)
    errs = []
    for N in (16, 32, 64):
        flat, pts = ball.voxel_ball(N)
        f = np.zeros(N ** 3, dtype=np.complex128)
        f[flat] = ball.psi_at(B, pts) @ coef
        a = np.zeros(B.Nb, dtype=np.complex128)
        # complex f: expand real and imaginary parts separately (expand is linear)
        a = ball.expand(B, f.real.reshape(N, N, N))[0] + 1j * ball.expand(B, f.imag.reshape(N, N, N))[0]
        errs.append(np.linalg.norm(a - coef) / np.linalg.norm(coef))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.05


def test_shift_volume_definition():
    rng = np.random.default_rng(8)
    v = rng.normal(size=(8, 8, 8))
    s = (2, -1, 3)
    out = ball.shift_volume(v, s)
    for z, y, x in ((0, 1, 0), (4, 4, 4), (2, 7, 5)):
        zz, yy, xx = z + s[2], y + s[1], x + s[0]
        ref = v[zz, yy, xx] if (0 <= zz < 8 and 0 <= yy < 8 and 0 <= xx < 8) else 0.0
        assert out[z, y, x] == ref
    # shifting back restores the overlap
    back = ball.shift_volume(out, (-2, 1, -3))
    assert np.array_equal(back[3:8, 0:7, 2:8], v[3:8, 0:7, 2:8])
