"""Band choice by the energy ratio (Fig. 1; Sec. III picks its L_set with it) and per-subtomogram marching
schedules, through the C ABI, against the FP64 oracle."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import align, ball, wigner  # noqa: E402
from paper_2509_01180_gb300 import bh, synth  # noqa: E402

THR32 = [0.05, 0.01, 0.001]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    bh.lib()
    return torch.device("cuda:0")


def to_f32(c):
    return torch.from_numpy(np.stack([c.real, c.imag], -1).astype(np.float32))


def f32_round(c):
    """The coefficients as the GPU holds them (complex64), back in FP64 for the oracle."""
    return c.astype(np.complex64).astype(np.complex128)


@pytest.fixture(scope="module")
def data32():
    """Six subtomograms of the 1024 x 32^3 workload, expanded by the oracle and rounded to FP32."""
    w = synth.make_workload("batch32", count=6)
    Bs = ball.make_basis(w.Lmax, w.lam_max)
    t = f32_round(ball.expand(Bs, w.template.astype(np.float64))[0])
    F = f32_round(ball.expand(Bs, w.vols.astype(np.float64)))
    return w, Bs, t, F


def robust(r, taus, margin=1e-4):
    """True when no ratio lies within `margin` (relative) of a threshold, so FP32 xi cannot flip a decision."""
    return all(abs(x - tau) > margin * tau for x in r for tau in taus)


def test_choose_bands_matches_oracle(dev, data32):
    w, Bs, t, F = data32
    p = bh.bh_plan_create(w.N, w.Lmax, w.lam_max, bh.BH_MODE_FP32, flags=bh.BH_PLAN_MATCH_ONLY)
    for L, thr, L_min in ((16, THR32, 1), (16, [0.2, 0.02, 0.002, 0.0002], 2), (12, [0.5], 3)):
        tab, e = bh.bh_choose_bands(p, to_f32(t).to(dev), to_f32(F).to(dev), L, thr, L_min=L_min, with_energy=True)
        rows, e = bh.stage_rows(tab), e.cpu().numpy()
        checked = 0
        for b in range(w.B):
            xi = align.build_xi(Bs, t, F[b], L)
            ref_e = np.array([np.sum(np.abs(x) ** 2) for x in xi])
            assert np.allclose(e[b], ref_e, rtol=1e-5, atol=1e-7 * ref_e.sum())
            r = align.energy_ratio(xi)
            ref = align.choose_bands(xi, thr, L_min)
            if robust(r, thr):
                assert rows[b] == ref, (L, thr, b, rows[b], ref)
                checked += 1
            # always: a valid schedule under the rule
            assert rows[b] == sorted(set(rows[b])) and rows[b][0] >= L_min and rows[b][-1] <= L
        assert checked >= w.B - 1
    p.destroy()


def test_choose_bands_arguments(dev, data32):
    w, Bs, t, F = data32
    p = bh.bh_plan_create(w.N, w.Lmax, w.lam_max, bh.BH_MODE_FP32, flags=bh.BH_PLAN_MATCH_ONLY)
    tt, ff = to_f32(t).to(dev), to_f32(F).to(dev)
    for thr, L, L_min in (([0.01, 0.05], 16, 1), ([1.5], 16, 1), ([0.1], 17, 1), ([0.1], 16, 0), ([0.1] * 9, 16, 1)):
        with pytest.raises(bh.BHError):
            bh.bh_choose_bands(p, tt, ff, L, thr, L_min=L_min)
    p.destroy()


def test_uniform_stage_table_is_the_plain_call(dev, data32):
    """A table whose every row is the launch's schedule gives bitwise the launch's results (ascent in each
    kernel variant, Newton, FP64 re-score)."""
    w, Bs, t, F = data32
    p = bh.bh_plan_create(w.N, w.Lmax, w.lam_max, bh.BH_MODE_FP32, flags=bh.BH_PLAN_MATCH_ONLY)
    tt, ff = to_f32(t).to(dev), to_f32(F).to(dev)
    starts = torch.from_numpy(w.starts).to(dev)
    row = [len(w.stages)] + w.stages + [0] * (bh.BH_STAGE_ROW - 1 - len(w.stages))
    tab = torch.tensor([row] * w.B, dtype=torch.int32, device=dev)
    for kw in (dict(group=4, starts_per_thread=2), dict(group=8, starts_per_thread=1), dict(newton=True),
               dict(refine_fp64=3)):
        steps = 10 if kw.get("newton") else w.steps
        a = bh.bh_align_batch(p, tt, ff, starts, w.stages, steps, **kw)
        b = bh.bh_align_batch(p, tt, ff, starts, w.stages, steps, stage_table=tab, **kw)
        torch.cuda.synchronize()
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]), kw
    p.destroy()


def test_per_subtomogram_schedules_match_oracle(dev, data32):
    """Bands chosen per subtomogram, then the marching ascent of each on its own schedule: the oracle's
    optimum on that schedule within 0.1 degree (unless its two best starts are tied), and each subtomogram
    re-scored in FP64 at its own last band."""
    w, Bs, t, F = data32
    p = bh.bh_plan_create(w.N, w.Lmax, w.lam_max, bh.BH_MODE_FP32, flags=bh.BH_PLAN_MATCH_ONLY)
    tt, ff = to_f32(t).to(dev), to_f32(F).to(dev)
    tab, _ = bh.bh_choose_bands(p, tt, ff, 16, THR32)
    # make the schedules differ between subtomograms even when the data choose alike
    tab[1] = torch.tensor([2, 3, 9] + [0] * 6, dtype=torch.int32, device=dev)
    rows = bh.stage_rows(tab)
    starts = torch.from_numpy(w.starts).to(dev)
    q, s = bh.bh_align_batch(p, tt, ff, starts, [4, 8, 16], w.steps, stage_table=tab)
    q64, s64 = bh.bh_align_batch(p, tt, ff, starts, [4, 8, 16], w.steps, stage_table=tab, refine_fp64=4)
    q, q64, s64 = q.cpu().numpy().astype(np.float64), q64.cpu().numpy().astype(np.float64), s64.cpu().numpy()
    for b in range(w.B):
        ref = align.align_particle(Bs, t, F[b], w.starts[b].astype(np.float64), rows[b], w.steps)
        srt = np.sort(ref.start_score)[::-1]
        tied = (srt[0] - srt[1]) < 1e-4 * abs(srt[0])
        ang = math.degrees(wigner.geodesic_angle(q[b] / np.linalg.norm(q[b]), ref.q))
        assert tied or ang < 0.1, (b, rows[b], ang)
        L = rows[b][-1]
        xi = align.build_xi(Bs, t, F[b], L)
        ref64 = align.score(xi, q64[b] / np.linalg.norm(q64[b]), L)
        assert abs(s64[b] - ref64) < 1e-6 * abs(ref64), (b, L, s64[b], ref64)
    p.destroy()
