"""Parity of the FP32 evaluation of Eq. 2 and its closed-form derivatives (Sec. II-C) at the bands the
workloads march to (16 at 32^3, 32 at 64^3), and of the FP32 marching ascent at 64^3, against the FP64
oracle.  Coefficients are drawn directly in the real-volume symmetry f_{k,l,-m} = (-1)^m conj(f_klm), so no
64^3 expansion is needed for the evaluation tests.

Tolerances:
  * score: |S_gpu - S_ref| <= 1e-4 ||t_<=L|| ||f_<=L|| (the Cauchy-Schwarz bound of |S|) everywhere, and
    <= 1e-4 |S_ref| wherever |S_ref| >= 0.1 ||t_<=L|| ||f_<=L|| (relative, where S is not near zero);
  * gradient <= 1e-4 (L+1) ||t|| ||f||, Hessian <= 1e-4 (L+1)^2 ||t|| ||f|| (sin beta > 0.2), as at low bands;
  * rotations: the oracle's optimum from the same starts within 0.1 degree unless its two best starts are
    tied (score gap < 1e-4 relative).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import align, ball, wigner  # noqa: E402
from paper_2509_01180_gb300 import bh, synth  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    bh.lib()
    return torch.device("cuda:0")


_plans, _bases = {}, {}


def match_plan(N):
    if N not in _plans:
        _plans[N] = bh.bh_plan_create(N, N // 2, math.pi * N / 2, bh.BH_MODE_FP32, flags=bh.BH_PLAN_MATCH_ONLY)
    return _plans[N]


def basis(N):
    if N not in _bases:
        _bases[N] = ball.make_basis(N // 2, math.pi * N / 2)
    return _bases[N]


def to_f32(c):
    return torch.from_numpy(np.stack([c.real, c.imag], -1).astype(np.float32))


def real_symmetric(Bs, rng, decay=1.0):
    """Random coefficients of a real volume: f_{k,l,-m} = (-1)^m conj(f_klm) (f_kl0 real), amplitude falling
    like 1/(1+l)^decay as in the phantoms' spectra; rounded to FP32 (what the GPU holds)."""
    c = np.zeros(Bs.Nb, dtype=np.complex128)
    for l in range(Bs.Lmax + 1):
        for k in range(len(Bs.roots[l])):
            o = Bs.offsets[l] + k * (2 * l + 1) + l
            a = 1.0 / (1 + l) ** decay
            c[o] = a * rng.normal()
            for m in range(1, l + 1):
                z = a * (rng.normal() + 1j * rng.normal()) / math.sqrt(2)
                c[o + m] = z
                c[o - m] = (-1) ** m * np.conj(z)
    return c.astype(np.complex64).astype(np.complex128)


def correlated_pair(Bs, rng):
    """Template t and f = R0 t + noise, so that Eq. 2 is large near R0^{-1} (where the relative check bites)."""
    t = real_symmetric(Bs, rng)
    q0 = synth.uniform_quaternions(rng, 1)[0]
    f = align.rotate_coeffs(Bs, t, q0) + 0.3 * real_symmetric(Bs, rng)
    return t, f.astype(np.complex64).astype(np.complex128), q0


def eval_rotations(rng, q0, n_near, n_far):
    """Rotations near R0^{-1} (a few degrees away) and uniform ones, all with sin(beta) > 0.2."""
    out = []
    base = wigner.quat_conj(q0)
    while len(out) < n_near:
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        ang = math.radians(rng.uniform(0.5, 6.0))
        q = wigner.quat_mul(base, np.array([math.cos(ang / 2), *(math.sin(ang / 2) * ax)]))
        if 2 * math.hypot(q[1], q[2]) * math.hypot(q[0], q[3]) > 0.2:
            out.append(q)
    while len(out) < n_near + n_far:
        q = synth.uniform_quaternions(rng, 1)[0]
        if 2 * math.hypot(q[1], q[2]) * math.hypot(q[0], q[3]) > 0.2:
            out.append(q)
    return np.array(out)


@pytest.mark.parametrize("N,L", [(32, 16), (64, 24), (64, 32)])
def test_score_grad_high_band_matches_oracle(dev, N, L):
    Bs = basis(N)
    rng = np.random.default_rng(900 + L)
    t, f, q0 = correlated_pair(Bs, rng)
    quats = eval_rotations(rng, q0, 6, 6)
    p = match_plan(N)
    sc, gr = bh.bh_score_grad(p, to_f32(t).to(dev), to_f32(f[None]).to(dev),
                              torch.from_numpy(quats[None].astype(np.float32)).to(dev), L)
    sc, gr = sc.cpu().numpy()[0], gr.cpu().numpy()[0]
    o = Bs.offsets[L + 1]
    bound = np.linalg.norm(t[:o]) * np.linalg.norm(f[:o])
    xi = align.build_xi(Bs, t, f, L)
    relative = 0
    for s, q in enumerate(quats):
        S_ref, g_ref = align.score_grad(xi, q.astype(np.float32).astype(np.float64), L)
        err = abs(sc[s] - S_ref)
        assert err <= 1e-4 * bound, (s, sc[s], S_ref)
        if abs(S_ref) >= 0.1 * bound:
            assert err <= 1e-4 * abs(S_ref), (s, sc[s], S_ref, err / abs(S_ref))
            relative += 1
        assert np.max(np.abs(gr[s] - g_ref)) <= 1e-4 * (L + 1) * bound, (s, gr[s], g_ref)
    assert relative >= 6  # the rotations near the optimum carry the relative check


@pytest.mark.parametrize("N,L", [(32, 16), (64, 32)])
def test_score_hess_high_band_matches_oracle(dev, N, L):
    Bs = basis(N)
    rng = np.random.default_rng(950 + L)
    t, f, q0 = correlated_pair(Bs, rng)
    quats = eval_rotations(rng, q0, 4, 4)
    p = match_plan(N)
    sc, gr, H = bh.bh_score_hess(p, to_f32(t).to(dev), to_f32(f[None]).to(dev),
                                 torch.from_numpy(quats[None].astype(np.float32)).to(dev), L)
    sc, gr, H = sc.cpu().numpy()[0], gr.cpu().numpy()[0], H.cpu().numpy()[0]
    o = Bs.offsets[L + 1]
    bound = np.linalg.norm(t[:o]) * np.linalg.norm(f[:o])
    xi = align.build_xi(Bs, t, f, L)
    for s, q in enumerate(quats):
        S_ref, g_ref, H_ref = align.score_grad_hess(xi, q.astype(np.float32).astype(np.float64), L)
        assert abs(sc[s] - S_ref) <= 1e-4 * bound
        if abs(S_ref) >= 0.1 * bound:
            assert abs(sc[s] - S_ref) <= 1e-4 * abs(S_ref)
        assert np.max(np.abs(gr[s] - g_ref)) <= 1e-4 * (L + 1) * bound
        assert np.max(np.abs(H[s] - H_ref)) <= 1e-4 * (L + 1) ** 2 * bound, (s, H[s], H_ref)


DEGREES = [2, 4, 8, 12, 16, 20, 24, 28, 32]


def test_fp32_recursion_error_by_degree(dev, capsys):
    """The error of the FP32 evaluation (rescaled d-recursion, seeds, phases, sums) for one degree at a time:
    coefficients only at degree l, err_l = max over 24 rotations of |S_gpu - S_ref| / (||t^l|| ||f^l||),
    the error of D^l in the xi-weighted norm.  Measured on a GB300: 2e-8 at l = 2, 1e-7 at l = 16, 3e-7 at
    l = 32 (FP64 re-score 5e-9 to 2e-8), growing about linearly with l and far below the 1e-4 score
    tolerance, which is why the ascent keeps the whole recursion in FP32 and FP64 is used only for the
    final re-score.  The table is printed (pytest -s) with the FP64 re-score's error beside it."""
    N = 64
    Bs = basis(N)
    p = match_plan(N)
    rng = np.random.default_rng(77)
    quats = np.array([q for q in synth.uniform_quaternions(rng, 64)
                      if 2 * math.hypot(q[1], q[2]) * math.hypot(q[0], q[3]) > 0.05][:24])
    rows = []
    for l in DEGREES:
        mask = np.zeros(Bs.Nb)
        mask[Bs.offsets[l]:Bs.offsets[l + 1]] = 1.0
        t = real_symmetric(Bs, rng, decay=0.0) * mask
        f = real_symmetric(Bs, rng, decay=0.0) * mask
        sc, _ = bh.bh_score_grad(p, to_f32(t).to(dev), to_f32(f[None]).to(dev),
                                 torch.from_numpy(quats[None].astype(np.float32)).to(dev), l, with_grad=False)
        # FP64 re-score of the same rotations: each rotation as its own start, K = 1
        sq = torch.from_numpy(quats[:, None, :].astype(np.float32)).to(dev).contiguous()
        ss = torch.zeros((len(quats), 1), device=dev)
        tt = to_f32(t).to(dev)
        ff = to_f32(np.repeat(f[None], len(quats), 0)).to(dev)
        _, _, s64 = bh.bh_refine_fp64(p, tt, ff, sq, ss, l, 1)
        sc, s64 = sc.cpu().numpy()[0], s64.cpu().numpy()
        xi = align.build_xi(Bs, t, f, l)
        scale = np.linalg.norm(t) * np.linalg.norm(f)
        e32 = e64 = 0.0
        for s, q in enumerate(quats):
            ref = align.score(xi, q.astype(np.float32).astype(np.float64), l)
            e32 = max(e32, abs(sc[s] - ref) / scale)
            e64 = max(e64, abs(s64[s] - ref) / scale)
        rows.append((l, e32, e64))
    with capsys.disabled():
        print("\ndegree  FP32 evaluation  FP64 re-score   (max |S_gpu - S_ref| / (||t^l|| ||f^l||), 24 rotations)")
        for l, e32, e64 in rows:
            print(f"{l:6d}  {e32:15.2e}  {e64:13.2e}")
    for l, e32, e64 in rows:
        assert e32 <= 3e-8 * (l + 1), (l, e32)  # measured 2e-8 at l = 2 to 3e-7 at l = 32
        assert e64 <= 5e-8, (l, e64)             # limited by the FP32 rounding of the table


@pytest.mark.slow
def test_align_64_fp32_path_matches_oracle(dev):
    """One 64^3 subtomogram of the precision workload (l <= 32, marching 4-8-16-32 x 30) aligned on the FP32
    path (no FP64 re-score) from 8 of its starts, with the orbits dealt by rows and in flat order: the
    oracle's optimum from the same starts on the same coefficients within 0.1 degree, unless tied."""
    w = synth.make_workload("precision64", count=1)
    Bs = basis(64)
    F = ball.expand(Bs, np.concatenate([w.template[None], w.vols]).astype(np.float64))
    t, f = F[0].astype(np.complex64).astype(np.complex128), F[1].astype(np.complex64).astype(np.complex128)
    starts = w.starts[:, :8]
    p = match_plan(64)
    ref = align.align_particle(Bs, t, f, starts[0].astype(np.float64), w.stages, w.steps)
    srt = np.sort(ref.start_score)[::-1]
    tied = (srt[0] - srt[1]) < 1e-4 * abs(srt[0])
    for kw in (dict(group=8, starts_per_thread=1, dealing=1), dict(group=16, starts_per_thread=1, dealing=2),
               dict(group=8, starts_per_thread=2, dealing=2), dict(group=16, starts_per_thread=2, dealing=2)):
        q, s = bh.bh_align_batch(p, to_f32(t).to(dev), to_f32(f[None]).to(dev),
                                 torch.from_numpy(np.ascontiguousarray(starts)).to(dev), w.stages, w.steps, **kw)
        q = q.cpu().numpy()[0].astype(np.float64)
        ang = math.degrees(wigner.geodesic_angle(q / np.linalg.norm(q), ref.q))
        assert tied or ang < 0.1, (kw, ang)
        assert tied or abs(float(s[0]) - ref.score) < 1e-4 * abs(ref.score), kw
