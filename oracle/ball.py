"""Ball-harmonic basis and voxel expansion, FP64 (oracle; test infrastructure).

Paper passages (Sec. II-A, "Ball Harmonics"):
  * basis display:   psi_{k,l,m}(r,theta,phi) = c_lk j_l(lambda_lk r) Y_l^m(theta,phi) chi_[0,1)(r),
                     m in {-l..l}, l >= 0, k >= 1, c_lk > 0 "normalization constants",
                     j_l spherical Bessel of the first kind, lambda_lk the k-th positive root of j_l.
  * expansion display: f(x) = sum_{(k,l,m) in I} f_hat_klm psi_klm, for a finite index set I.
  * frequency ordering by the eigenvalue lambda_lk^2 (lowpass = zero high-lambda coefficients).

Readings where the paper is silent:
  * c_lk makes psi orthonormal on the unit ball B.  Since the integral of
    j_l(lambda r)^2 r^2 over [0,1] equals j_{l+1}(lambda)^2 / 2 at a root of j_l,
    c_lk = sqrt(2) / |j_{l+1}(lambda_lk)|.
  * Y_l^m is the complex spherical harmonic, orthonormal on the sphere, with the
    Condon-Shortley phase, so that Y_l^{-m} = (-1)^m conj(Y_l^m).
  * The index set I is {(k,l,m): l <= Lmax, lambda_lk <= lambda_max}; a root is
    included when lambda_lk <= lambda_max + ROOT_SLACK (the default
    lambda_max = pi N / 2 coincides with the root k = N/2 of j_0 = sin x / x).
  * Voxel grid of an N^3 box (N even), array order vol[z, y, x]: voxel i along
    an axis sits at (i - N/2) / (N/2); the ball is the set of voxels with
    (ix-N/2)^2 + (iy-N/2)^2 + (iz-N/2)^2 < (N/2)^2 (strict, exact in integers).
  * Coefficients are the discrete L2 inner product (quadrature, weight h^3,
    h = 2/N): f_hat_klm = h^3 sum_v f(x_v) conj(psi_klm(x_v)).  The paper's own
    expansion uses a fast transform of the same inner product; on a voxel grid
    this is the plain definition.
  * Coefficient layout: complex vector ordered [l][k][m + l], l = 0..Lmax.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.optimize import brentq
from scipy.special import spherical_jn

ROOT_SLACK = 1e-9


def sph_jn(l: int, x):
    """Spherical Bessel function of the first kind j_l(x) (basis display, Sec. II-A).

    A library routine serves as this step."""
    return spherical_jn(l, x)


def bessel_roots(l: int, lam_max: float) -> np.ndarray:
    """All positive roots lambda_lk of j_l with lambda_lk <= lam_max (+ROOT_SLACK), ascending.

    Sec. II-A defines lambda_lk as the k-th positive zero of j_l.  Roots are bracketed
    by sign changes on a fine scan (spacing of consecutive roots is about pi) and
    refined by Brent's method.  The first root of j_l exceeds l, so the scan
    starts at l (at 0.5 for l = 0, where j_0 = sin(x)/x)."""
    x0 = 0.5 if l == 0 else float(l)
    hi = lam_max + 0.5
    xs = np.arange(x0, hi + 0.05, 0.05)
    vals = sph_jn(l, xs)
    roots = []
    for i in range(len(xs) - 1):
        a, b = vals[i], vals[i + 1]
        if a == 0.0:
            roots.append(xs[i])
        elif a * b < 0.0:
            roots.append(brentq(lambda t: sph_jn(l, t), xs[i], xs[i + 1], xtol=1e-15, rtol=8.9e-16, maxiter=200))
    roots = np.array([r for r in roots if r <= lam_max + ROOT_SLACK])
    return roots


def norm_const(l: int, lam: float) -> float:
    """c_lk = sqrt(2)/|j_{l+1}(lambda_lk)|: the positive constant making psi orthonormal on B."""
    return math.sqrt(2.0) / abs(float(sph_jn(l + 1, lam)))


def assoc_legendre_normalized(L: int, x: np.ndarray) -> np.ndarray:
    """Pbar[l, m, :] for 0 <= m <= l <= L with Y_l^m(theta, phi) = Pbar_l^m(cos theta) e^{i m phi}.

    Textbook recurrences for the sphere-normalised associated Legendre functions
    with the Condon-Shortley phase:
        Pbar_0^0 = 1/sqrt(4 pi)
        Pbar_m^m = -sqrt((2m+1)/(2m)) sqrt(1-x^2) Pbar_{m-1}^{m-1}
        Pbar_{m+1}^m = sqrt(2m+3) x Pbar_m^m
        Pbar_l^m = a_lm (x Pbar_{l-1}^m - Pbar_{l-2}^m / a_{l-1,m}),  a_lm = sqrt((4l^2-1)/(l^2-m^2)).
    """
    x = np.asarray(x, dtype=np.float64)
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    P = np.zeros((L + 1, L + 1) + x.shape)
    P[0, 0] = 1.0 / math.sqrt(4.0 * math.pi)
    for m in range(1, L + 1):
        P[m, m] = -math.sqrt((2 * m + 1) / (2.0 * m)) * s * P[m - 1, m - 1]
    for m in range(0, L):
        P[m + 1, m] = math.sqrt(2 * m + 3) * x * P[m, m]
    for m in range(0, L + 1):
        for l in range(m + 2, L + 1):
            a_l = math.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
            a_lm1 = math.sqrt((4.0 * (l - 1) ** 2 - 1.0) / ((l - 1) ** 2 - m * m))
            P[l, m] = a_l * (x * P[l - 1, m] - P[l - 2, m] / a_lm1)
    return P


def sph_harm_all(L: int, pts: np.ndarray) -> list[np.ndarray]:
    """Complex Y_l^m at unit-or-zero direction vectors; returns [Y_l of shape (n, 2l+1)] with column m+l.

    Directions come from Cartesian points: cos(theta) = z/r, e^{i phi} = (x+iy)/rho.
    At r = 0 (and on the z axis for the azimuth) theta = phi = 0 by convention;
    only l = 0 survives there in the basis because j_l(0) = 0 for l >= 1."""
    pts = np.asarray(pts, dtype=np.float64)
    r = np.linalg.norm(pts, axis=1)
    rho = np.hypot(pts[:, 0], pts[:, 1])
    ct = np.where(r > 0, pts[:, 2] / np.where(r > 0, r, 1.0), 1.0)
    eiphi = np.where(rho > 0, (pts[:, 0] + 1j * pts[:, 1]) / np.where(rho > 0, rho, 1.0), 1.0 + 0j)
    P = assoc_legendre_normalized(L, ct)
    out = []
    for l in range(L + 1):
        Y = np.zeros((pts.shape[0], 2 * l + 1), dtype=np.complex128)
        for m in range(0, l + 1):
            ym = P[l, m] * eiphi ** m
            Y[:, m + l] = ym
            if m > 0:
                Y[:, -m + l] = (-1) ** m * np.conj(ym)
        out.append(Y)
    return out


@dataclass
class Basis:
    """The truncated index set I and its radial data (Sec. II-A)."""

    Lmax: int
    lam_max: float
    roots: list  # roots[l] = array of lambda_lk, k = 1..K_l
    consts: list  # consts[l] = array of c_lk
    offsets: np.ndarray = field(default=None)  # offsets[l] = start of degree l in the [l][k][m+l] layout

    @property
    def K(self):
        return [len(r) for r in self.roots]

    @property
    def Nb(self) -> int:
        return int(self.offsets[-1])


def make_basis(Lmax: int, lam_max: float) -> Basis:
    """Index set I = {(k,l,m): l <= Lmax, lambda_lk <= lam_max} with c_lk (Sec. II-A)."""
    roots, consts = [], []
    for l in range(Lmax + 1):
        r = bessel_roots(l, lam_max)
        roots.append(r)
        consts.append(np.array([norm_const(l, lam) for lam in r]))
    offs = [0]
    for l in range(Lmax + 1):
        offs.append(offs[-1] + len(roots[l]) * (2 * l + 1))
    return Basis(Lmax, lam_max, roots, consts, np.array(offs, dtype=np.int64))


def psi_at(basis: Basis, pts: np.ndarray) -> np.ndarray:
    """psi_klm at Cartesian points (n, 3) inside the closed unit ball; returns (n, Nb) complex in [l][k][m+l] order.

    psi = c_lk j_l(lambda_lk r) Y_l^m(theta, phi) chi_[0,1)(r) (basis display, Sec. II-A)."""
    pts = np.asarray(pts, dtype=np.float64)
    r = np.linalg.norm(pts, axis=1)
    chi = (r < 1.0).astype(np.float64)
    Y = sph_harm_all(basis.Lmax, pts)
    out = np.zeros((pts.shape[0], basis.Nb), dtype=np.complex128)
    for l in range(basis.Lmax + 1):
        for k, (lam, c) in enumerate(zip(basis.roots[l], basis.consts[l])):
            rad = c * sph_jn(l, lam * r) * chi
            o = basis.offsets[l] + k * (2 * l + 1)
            out[:, o:o + 2 * l + 1] = rad[:, None] * Y[l]
    return out


def voxel_ball(N: int):
    """In-ball voxel indices (flat, into vol[z,y,x]) and their centres in unit-ball coordinates (x, y, z)."""
    if N % 2:
        raise ValueError("box edge N must be even")
    h = N // 2
    i = np.arange(N) - h
    z, y, x = np.meshgrid(i, i, i, indexing="ij")
    inside = (x * x + y * y + z * z) < h * h
    flat = np.flatnonzero(inside.ravel())
    pts = np.stack([x.ravel()[flat], y.ravel()[flat], z.ravel()[flat]], axis=1).astype(np.float64) / h
    return flat, pts


def expand(basis: Basis, vols: np.ndarray) -> np.ndarray:
    """Coefficients f_hat_klm = h^3 sum_v f(x_v) conj(psi_klm(x_v)) of B volumes (B, N, N, N) -> (B, Nb) complex.

    The expansion display of Sec. II-A, with the discrete inner product on the
    voxel grid (h = 2/N).  psi factors into the radial profile c_lk j_l(lambda_lk r)
    times Y_l^m, which the loop over (l, k) uses directly; the sum over voxels is a
    matrix product."""
    vols = np.asarray(vols, dtype=np.float64)
    if vols.ndim == 3:
        vols = vols[None]
    B, N = vols.shape[0], vols.shape[1]
    flat, pts = voxel_ball(N)
    X = vols.reshape(B, -1)[:, flat]
    r = np.linalg.norm(pts, axis=1)
    Y = sph_harm_all(basis.Lmax, pts)
    h3 = (2.0 / N) ** 3
    out = np.zeros((B, basis.Nb), dtype=np.complex128)
    for l in range(basis.Lmax + 1):
        Yc = np.conj(Y[l])
        for k, (lam, c) in enumerate(zip(basis.roots[l], basis.consts[l])):
            rad = c * sph_jn(l, lam * r)
            o = basis.offsets[l] + k * (2 * l + 1)
            out[:, o:o + 2 * l + 1] = h3 * ((X * rad[None, :]) @ Yc)
    return out


def split_by_degree(basis: Basis, coeffs: np.ndarray) -> list[np.ndarray]:
    """View a coefficient vector (Nb,) as [(K_l, 2l+1) arrays], row k, column m+l."""
    out = []
    for l in range(basis.Lmax + 1):
        o0, o1 = basis.offsets[l], basis.offsets[l + 1]
        out.append(np.asarray(coeffs[o0:o1]).reshape(len(basis.roots[l]), 2 * l + 1))
    return out


def shift_volume(vol: np.ndarray, s) -> np.ndarray:
    """f_s(x) = f(x + s) on the voxel grid for an integer shift s = (sx, sy, sz) voxels, zero where x + s
    leaves the box (Eq. 1's shifted subtomogram; array order [z][y][x])."""
    vol = np.asarray(vol)
    N = vol.shape[0]
    sx, sy, sz = (int(v) for v in s)
    out = np.zeros_like(vol)
    i = np.arange(N)
    ox, oy, oz = i + sx, i + sy, i + sz
    vx, vy, vz = (ox >= 0) & (ox < N), (oy >= 0) & (oy < N), (oz >= 0) & (oz < N)
    out[np.ix_(vz, vy, vx)] = vol[np.ix_(oz[vz], oy[vy], ox[vx])]
    return out
