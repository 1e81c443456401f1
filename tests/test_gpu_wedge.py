"""GPU parity of the missing-wedge constrained correlation (Sec. II-B) against the FP64 oracle.

Tolerances: host-prepared coefficients q, w, |T(0)|^2 agree with the oracle's to 1e-9 relative (both
FP64; a direct DFT against numpy's FFT); the norm Dn(R) to 1e-4 of its value and its gradient to
1e-4 (L+1) Dn (FP32 evaluation, as the score); the constrained ascent's optimum within 0.1 degree of the
oracle's from the same starts.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ball, wedge, wigner  # noqa: E402
from paper_2509_01180_gb300 import bh, synth  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    bh.lib()
    return torch.device("cuda:0")


def to_f32(c):
    return torch.from_numpy(np.stack([c.real, c.imag], -1).astype(np.float32))


def off_pole(rng, n):
    out = []
    while len(out) < n:
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        if 2 * math.hypot(q[1], q[2]) * math.hypot(q[0], q[3]) > 0.2:
            out.append(q)
    return np.array(out)


@pytest.mark.parametrize("N,L,a", [(16, 8, 60.0), (32, 16, 50.0)])
def test_wedge_coefficients_match_oracle(dev, N, L, a):
    w = synth.make_workload("pair16" if N == 16 else "batch32", count=1)
    p = bh.bh_plan_create(N, L, math.pi * N / 2, bh.BH_MODE_FP32)
    wd = bh.bh_wedge_create(p, w.template, a, L)
    q, wl, c0 = wd.coeffs()
    ref = wedge.make_wedge(w.template.astype(np.float64), a, L)
    assert abs(c0 - ref.c0) <= 1e-9 * ref.c0
    qs = max(float(np.abs(x).max()) for x in ref.q)
    for l in range(L + 1):
        assert np.abs(q[l] - ref.q[l]).max() <= 1e-9 * qs, l
        assert np.abs(wl[l] - ref.w[l]).max() <= 1e-12, l
    wd.destroy()
    p.destroy()


@pytest.mark.parametrize("L", [2, 4, 8])
def test_wedge_norm_matches_oracle(dev, L):
    w = synth.make_workload("pair16")
    p = bh.bh_plan_create(16, 8, 8 * math.pi, bh.BH_MODE_FP32)
    wd = bh.bh_wedge_create(p, w.template, 60.0, 8)
    ref = wedge.make_wedge(w.template.astype(np.float64), 60.0, 8)
    qs = off_pole(np.random.default_rng(90 + L), 9)
    dn, g = bh.bh_wedge_norm(p, wd, torch.from_numpy(qs.astype(np.float32)).to(dev), L)
    dn, g = dn.cpu().numpy(), g.cpu().numpy()
    for s in range(len(qs)):
        D, gD = wedge.denominator(ref, qs[s].astype(np.float32).astype(np.float64), L)
        assert abs(dn[s] - D) <= 1e-4 * D
        assert np.abs(g[s] - gD).max() <= 1e-4 * (L + 1) * D
    wd.destroy()
    p.destroy()


def test_constrained_align_matches_oracle(dev):
    """Plain method's pair with a +-60 deg missing wedge and SNR 1: same optimum as the oracle's constrained
    ascent from the same starts."""
    w = synth.make_workload("pair16", count=2, snr=1.0, wedge=60.0)
    Bs = ball.make_basis(8, 8 * math.pi)
    t = ball.expand(Bs, w.template.astype(np.float64))[0]
    F = ball.expand(Bs, w.vols.astype(np.float64))
    ref_w = wedge.make_wedge(w.template.astype(np.float64), 60.0, 8)
    p = bh.bh_plan_create(16, 8, 8 * math.pi, bh.BH_MODE_FP32)
    wd = bh.bh_wedge_create(p, w.template, 60.0, 8)
    q, s = bh.bh_align_batch(p, to_f32(t).to(dev), to_f32(F).to(dev), torch.from_numpy(w.starts).to(dev), w.stages,
                             w.steps, wedge=wd)
    q, s = q.cpu().numpy().astype(np.float64), s.cpu().numpy()
    for b in range(w.B):
        ref = wedge.align_constrained(Bs, t, F[b], ref_w, w.starts[b].astype(np.float64), w.stages, w.steps)
        qb = q[b] / np.linalg.norm(q[b])
        srt = np.sort(ref.start_score)[::-1]
        tied = len(srt) > 1 and (srt[0] - srt[1]) < 1e-4 * abs(srt[0])
        assert tied or math.degrees(wigner.geodesic_angle(qb, ref.q)) < 0.1
        assert abs(float(s[b]) - ref.score) < 1e-4 * abs(ref.score)
    wd.destroy()
    p.destroy()


def test_constrained_align_argument_errors(dev):
    w = synth.make_workload("pair16")
    p = bh.bh_plan_create(16, 8, 8 * math.pi, bh.BH_MODE_FP32)
    wd = bh.bh_wedge_create(p, w.template, 60.0, 4)
    c = torch.zeros((2, p.Nb, 2), device=dev)
    st = torch.from_numpy(w.starts).to(dev)
    with pytest.raises(bh.BHError):
        bh.bh_align_batch(p, c[0], c[1:], st, [2, 4, 8], 5, wedge=wd)  # band 8 above the wedge's 4
    with pytest.raises(bh.BHError):
        bh.bh_align_batch(p, c[0], c[1:], st, [2, 4], 5, wedge=wd, newton=True)
    with pytest.raises(bh.BHError):
        bh.bh_wedge_create(p, w.template, 95.0, 4)
    with pytest.raises(bh.BHError):
        bh.bh_wedge_create(p, w.template, 60.0, 9)
    wd.destroy()
    p.destroy()
