"""GPU tests of the plan options and the separate FP64 re-score call, through the C ABI."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import align, ball  # noqa: E402
from paper_2509_01180_gb300 import bh, synth  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    bh.lib()
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def batch(dev):
    """Three 32^3 subtomograms of the 1024 x 32^3 workload, expanded on the GPU (BF16-split plan)."""
    w = synth.make_workload("batch32", count=3)
    p = bh.bh_plan_create(w.N, w.Lmax, w.lam_max, bh.BH_MODE_BF16_SPLIT)
    tmpl = bh.bh_expand(p, torch.from_numpy(w.template[None]).to(dev))[0].contiguous()
    coef = bh.bh_expand(p, torch.from_numpy(w.vols).to(dev))
    yield w, p, tmpl, coef
    p.destroy()


def test_refine_call_equals_the_align_option(dev, batch):
    """bh_refine_fp64 after an ascent with per-start outputs gives bitwise what bh_align_batch with
    refine_fp64 = K gives (the same kernel on the same inputs)."""
    w, p, tmpl, coef = batch
    starts = torch.from_numpy(w.starts).to(dev)
    q1, s1 = bh.bh_align_batch(p, tmpl, coef, starts, w.stages, w.steps, refine_fp64=4)
    q0, s0, sq, ss = bh.bh_align_batch(p, tmpl, coef, starts, w.stages, w.steps, per_start=True)
    q2, s2, s64 = bh.bh_refine_fp64(p, tmpl, coef, sq, ss, w.stages[-1], 4)
    torch.cuda.synchronize()
    assert torch.equal(q1, q2) and torch.equal(s1, s2)
    assert torch.equal(s2, s64.float())
    # the re-scored value is the FP64 Eq. 2 at the reported rotation (oracle, on the GPU's coefficients)
    Bs = ball.make_basis(w.Lmax, w.lam_max)
    c = coef.cpu().numpy().astype(np.float64)
    t = tmpl.cpu().numpy().astype(np.float64)
    t = t[..., 0] + 1j * t[..., 1]
    for b in range(w.B):
        xi = align.build_xi(Bs, t, c[b, :, 0] + 1j * c[b, :, 1], w.stages[-1])
        qb = q2[b].cpu().numpy().astype(np.float64)
        ref = align.score(xi, qb / np.linalg.norm(qb), w.stages[-1])
        assert abs(float(s64[b]) - ref) < 1e-6 * abs(ref)


def test_refine_call_arguments(dev, batch):
    w, p, tmpl, coef = batch
    sq = torch.zeros((w.B, w.S, 4), device=dev)
    ss = torch.zeros((w.B, w.S), device=dev)
    with pytest.raises(bh.BHError):
        bh.bh_refine_fp64(p, tmpl, coef, sq, ss, w.stages[-1], w.S + 1)  # K > S
    with pytest.raises(bh.BHError):
        bh.bh_refine_fp64(p, tmpl, coef, sq, ss, w.Lmax + 1, 2)  # band above Lmax


def test_match_only_plan(dev, batch):
    """A plan without the expansion table aligns bitwise like the full plan; expansion calls are refused."""
    w, p, tmpl, coef = batch
    pm = bh.bh_plan_create(w.N, w.Lmax, w.lam_max, bh.BH_MODE_BF16_SPLIT, flags=bh.BH_PLAN_MATCH_ONLY)
    assert pm.flags == bh.BH_PLAN_MATCH_ONLY and pm.Nb == p.Nb and pm.V == p.V
    starts = torch.from_numpy(w.starts).to(dev)
    qa, sa = bh.bh_align_batch(p, tmpl, coef, starts, w.stages, w.steps, group=4, starts_per_thread=2)
    qb, sb = bh.bh_align_batch(pm, tmpl, coef, starts, w.stages, w.steps, group=4, starts_per_thread=2)
    torch.cuda.synchronize()
    assert torch.equal(qa, qb) and torch.equal(sa, sb)
    vols = torch.zeros((1, w.N, w.N, w.N), device=dev)
    for fn in (bh.lib().bh_expand, bh.lib().bh_expand_noalloc):
        out = torch.zeros((1, pm.Nb, 2), device=dev)
        assert fn(pm.handle, vols.data_ptr(), 1, out.data_ptr(), None) == bh.BH_ERR_ARG
        assert b"MATCH_ONLY" in bh.lib().bh_last_error()
    bh.bh_autotune(pm, 8, w.S, w.stages, 2)  # tunes the ascent only
    pm.destroy()


def test_plan_device_is_checked(dev, batch):
    """Calls that read a plan's tables refuse to run on another device (needs two GPUs)."""
    if torch.cuda.device_count() < 2:
        pytest.skip("one GPU: no other device to make current")
    w, p, tmpl, coef = batch
    out = torch.zeros((1, p.Nb, 2), device=dev)
    with torch.cuda.device(1):
        assert bh.lib().bh_expand(p.handle, out.data_ptr(), 1, out.data_ptr(), None) == bh.BH_ERR_ARG
        assert b"device" in bh.lib().bh_last_error()
