"""Bounds checks without a sanitizer: every output buffer of every entry point sits between two guard
regions filled with a sentinel bit pattern; after the call (at odd sizes: B = 1, B not a tile multiple,
S = 1 or odd, L = 0/1) the guards must be intact and every output slot written.  A kernel writing past
its buffer lands in the guard of the same allocation, so a bug shows up as a failed assertion, never as
a fault."""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2509_01180_gb300 import bh, synth  # noqa: E402

GUARD = 2048
SENT = 0x7FC0BAD5  # a NaN payload no kernel produces


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    bh.lib()
    return torch.device("cuda:0")


class Guarded:
    """A device buffer of n 4-byte elements with sentinel guards on both sides."""

    def __init__(self, shape, dev, dtype=torch.float32):
        self.n = int(np.prod(shape))
        self.buf = torch.empty(self.n + 2 * GUARD, dtype=dtype, device=dev)
        self.buf.view(torch.int32).fill_(SENT)
        self.t = self.buf[GUARD:GUARD + self.n].view(*shape)

    @property
    def ptr(self) -> int:
        return self.t.data_ptr()

    def check(self, written: bool = True):
        torch.cuda.synchronize()
        raw = self.buf.view(torch.int32).cpu().numpy()
        assert (raw[:GUARD] == SENT).all(), "write before the buffer"
        assert (raw[GUARD + self.n:] == SENT).all(), "write past the buffer"
        if written:
            assert (raw[GUARD:GUARD + self.n] != SENT).all(), "output slot left unwritten"


def _plan(N=16, L=8, mode=bh.BH_MODE_FP32, max_batch=0):
    return bh.bh_plan_create(N, L, math.pi * N / 2, mode, max_batch)


def _coeffs(p, dev, B, seed=0):
    rng = np.random.default_rng(seed)
    vols = torch.from_numpy(rng.normal(size=(B + 1, p.N, p.N, p.N)).astype(np.float32)).to(dev)
    c = bh.bh_expand(p, vols)
    return c[0].contiguous(), c[1:].contiguous()


@pytest.mark.parametrize("mode", [bh.BH_MODE_FP32, bh.BH_MODE_BF16_SPLIT])
@pytest.mark.parametrize("B,max_batch", [(1, 0), (37, 16), (130, 0)])
def test_expand_guards(dev, mode, B, max_batch):
    p = _plan(mode=mode, max_batch=max_batch)
    vols = torch.randn((B, 16, 16, 16), device=dev)
    out = Guarded((B, p.Nb, 2), dev)
    bh._check(bh.lib().bh_expand(p.handle, vols.data_ptr(), B, out.ptr, bh._stream(None)), "bh_expand")
    out.check()
    p.destroy()


@pytest.mark.parametrize("S,L", [(1, 0), (7, 1), (3, 8)])
def test_score_grad_hess_guards(dev, S, L):
    p = _plan()
    t, sub = _coeffs(p, dev, 3)
    q = torch.from_numpy(synth.uniform_quaternions(np.random.default_rng(1), 3 * S).astype(np.float32)).to(dev)
    sc, gr = Guarded((3, S), dev), Guarded((3, S, 3), dev)
    bh._check(bh.lib().bh_score_grad(p.handle, t.data_ptr(), sub.data_ptr(), 3, q.data_ptr(), S, L, sc.ptr, gr.ptr,
                                     bh._stream(None)), "bh_score_grad")
    sc.check()
    gr.check()
    sc, gr, he = Guarded((3, S), dev), Guarded((3, S, 3), dev), Guarded((3, S, 6), dev)
    bh._check(bh.lib().bh_score_hess(p.handle, t.data_ptr(), sub.data_ptr(), 3, q.data_ptr(), S, L, sc.ptr, gr.ptr,
                                     he.ptr, bh._stream(None)), "bh_score_hess")
    for g in (sc, gr, he):
        g.check()
    p.destroy()


@pytest.mark.parametrize("B,S,group,spt,newton,refine", [
    (1, 1, 0, 0, 0, 0), (5, 3, 1, 1, 0, 0), (37, 16, 4, 2, 0, 0), (37, 6, 8, 1, 0, 2),
    (5, 5, 0, 0, 1, 0), (9, 4, 32, 0, 1, 3)])
def test_align_batch_guards(dev, B, S, group, spt, newton, refine):
    p = _plan()
    t, sub = _coeffs(p, dev, B)
    starts = torch.from_numpy(synth.uniform_quaternions(np.random.default_rng(2), B * S).astype(np.float32)).to(dev)
    quat, score = Guarded((B, 4), dev), Guarded((B,), dev)
    sq, ss = Guarded((B, S, 4), dev), Guarded((B, S), dev)
    o = bh.AlignOpts()
    o.group, o.starts_per_thread, o.newton, o.refine_fp64 = group, spt, newton, refine
    o.start_quat_out, o.start_score_out = sq.ptr, ss.ptr
    st = (ctypes.c_int * 3)(2, 4, 8)
    bh._check(bh.lib().bh_align_batch(p.handle, t.data_ptr(), sub.data_ptr(), B, starts.data_ptr(), S, st, 3, 4,
                                      quat.ptr, score.ptr, ctypes.byref(o), bh._stream(None)), "bh_align_batch")
    for g in (quat, score, sq, ss):
        g.check()
    p.destroy()


@pytest.mark.parametrize("n,S", [(37, 1), (37, 37), (1000, 5), (300, 100)])
def test_candidate_guards(dev, n, S):
    p = _plan()
    t, sub = _coeffs(p, dev, 3)
    grid = bh.bh_grid_create(synth.super_fibonacci(n), math.radians(40.0))
    st, ix, sc = Guarded((3, S, 4), dev), Guarded((3, S), dev, torch.int32), Guarded((3, n), dev)
    bh._check(bh.lib().bh_candidates(p.handle, grid.handle, t.data_ptr(), sub.data_ptr(), 3, 2, None, 0, S, st.ptr,
                                     ix.ptr, sc.ptr, bh._stream(None)), "bh_candidates")
    for g in (st, ix, sc):
        g.check()
    grid.destroy()
    p.destroy()


def test_energy_shift_and_wedge_guards(dev):
    p = _plan()
    t, sub = _coeffs(p, dev, 5)
    en = Guarded((5, 9), dev)
    bh._check(bh.lib().bh_energy(p.handle, t.data_ptr(), sub.data_ptr(), 5, 8, None, 0, en.ptr, bh._stream(None)),
              "bh_energy")
    en.check()

    B, S = 3, 4
    vols = torch.randn((B, 16, 16, 16), device=dev)
    sh = np.array([[0, 0, 0], [1, 0, -1], [-2, 1, 0]], dtype=np.int32)
    starts = torch.from_numpy(synth.uniform_quaternions(np.random.default_rng(3), B * S).astype(np.float32)).to(dev)
    nbytes = int(bh.lib().bh_align_shifts_workspace(p.handle, B, 3, S))
    ws = torch.empty((nbytes + 255) // 256 * 64, dtype=torch.float32, device=dev)
    si, qo, so = Guarded((B,), dev, torch.int32), Guarded((B, 4), dev), Guarded((B,), dev)
    st = (ctypes.c_int * 2)(2, 4)
    bh._check(bh.lib().bh_align_shifts(p.handle, t.data_ptr(), vols.data_ptr(), B, sh.ctypes.data, 3, starts.data_ptr(),
                                       S, st, 2, 3, ws.data_ptr(), ws.numel() * 4, si.ptr, qo.ptr, so.ptr, None,
                                       bh._stream(None)), "bh_align_shifts")
    for g in (si, qo, so):
        g.check()

    w = synth.make_workload("pair16")
    wd = bh.bh_wedge_create(p, w.template, 60.0, 8)
    q = torch.from_numpy(synth.uniform_quaternions(np.random.default_rng(4), 5).astype(np.float32)).to(dev)
    dn, gr = Guarded((5,), dev), Guarded((5, 3), dev)
    bh._check(bh.lib().bh_wedge_norm(p.handle, wd.handle, q.data_ptr(), 5, 4, dn.ptr, gr.ptr, bh._stream(None)),
              "bh_wedge_norm")
    dn.check()
    gr.check()
    wd.destroy()
    p.destroy()


def test_bounded_device_wait_reports_timeout_and_context_survives(dev):
    """A wait of the tensor-core pipeline's kind runs out on a barrier phase that nothing completes: the
    probe kernel returns after the wait's time limit, the plan's status reports BH_ERR_TIMEOUT once, and
    the context keeps working (an expansion right after matches one before)."""
    p = _plan(mode=bh.BH_MODE_BF16_SPLIT)
    vols = torch.randn((3, 16, 16, 16), device=dev)
    before = bh.bh_expand(p, vols).clone()
    bh.bh_plan_status(p)  # clean
    bh.bh_plan_probe_wait(p)
    torch.cuda.synchronize()
    with pytest.raises(bh.BHError) as e:
        bh.bh_plan_status(p)
    assert e.value.status == bh.BH_ERR_TIMEOUT
    bh.bh_plan_status(p)  # cleared
    after = bh.bh_expand(p, vols)
    torch.cuda.synchronize()
    assert torch.equal(before, after)
    bh.bh_plan_status(p)
    p.destroy()
