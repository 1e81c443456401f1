"""GPU parity of the candidate starts (Sec. III: local maxima of the lowest band on a rotation grid).

Compared with the FP64 oracle: the neighbour lists (bit-exact), the band-L grid scores (score tolerance
1e-4 * ||t_<=L|| ||f_<=L||), the candidate indices where the oracle's decisions are not within twice that
tolerance of a tie, and the optimum reached from the candidates (0.1 degree).  Where FP32 rounding may
decide a near-tie, the kernel's selection is checked for validity against its own scores instead.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import align, ball, candidates, wigner  # noqa: E402
from paper_2509_01180_gb300 import bh, synth  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    bh.lib()
    return torch.device("cuda:0")


def to_c(t):
    a = t.detach().cpu().numpy().astype(np.float64)
    return a[..., 0] + 1j * a[..., 1]


def to_f32(c):
    return torch.from_numpy(np.stack([c.real, c.imag], -1).astype(np.float32))


def selection_from(scores, nb, S):
    """The selection the definition gives for these exact scores: rank = (score desc, index asc); local
    maxima (ranked above every neighbour) by rank, then the rest by rank."""
    n = len(scores)
    order = np.lexsort((np.arange(n), -np.asarray(scores, np.float64)))
    rank = np.empty(n, dtype=np.int64)
    rank[order] = np.arange(n)
    is_max = np.array([bool(np.all(rank[i] < rank[nb[i]])) for i in range(n)])
    return np.concatenate([order[is_max[order]], order[~is_max[order]]])[:S]


def robust_prefix(sc64, nb, cand, tau):
    """Length of the prefix of the oracle's candidate list that no score perturbation below tau can change."""
    n = len(sc64)
    margin = np.array([sc64[i] - (sc64[nb[i]].max() if len(nb[i]) else -np.inf) for i in range(n)])
    ambiguous = np.abs(margin) <= tau
    k = 0
    for s, c in enumerate(cand):
        if margin[c] <= tau:  # a point that is not clearly a local maximum ends the robust part
            break
        nxt = cand[s + 1] if s + 1 < len(cand) else None
        if nxt is not None and sc64[c] - sc64[nxt] <= tau:
            break
        if np.any(ambiguous & (sc64 >= sc64[c] - tau)):
            break
        k += 1
    return k


@pytest.mark.parametrize("n,radius_deg", [(37, 0.0), (37, 60.0), (1000, 30.0), (1000, 50.0), (4608, 25.0)])
def test_grid_neighbors_bit_exact(dev, n, radius_deg):
    g = synth.super_fibonacci(n)
    grid = bh.bh_grid_create(g, math.radians(radius_deg))
    got = grid.neighbors()
    ref = candidates.grid_neighbors(g, math.radians(radius_deg))
    assert grid.n == n
    assert all(np.array_equal(a, b) for a, b in zip(got, ref))
    assert grid.max_neighbors == max(len(r) for r in ref)
    grid.destroy()


def _pair16_case(dev, count, L1):
    w = synth.make_workload("pair16", count=count, snr=0.5)
    Bs = ball.make_basis(w.Lmax, w.lam_max)
    p = bh.bh_plan_create(w.N, w.Lmax, w.lam_max, bh.BH_MODE_FP32)
    vols = torch.from_numpy(np.concatenate([w.template[None], w.vols])).to(dev)
    c = bh.bh_expand(p, vols)
    t = ball.expand(Bs, w.template.astype(np.float64))[0]
    F = ball.expand(Bs, w.vols.astype(np.float64))
    return w, Bs, p, c, t, F


@pytest.mark.parametrize("n,S", [(1000, 8), (37, 37), (300, 1), (300, 100)])  # S > 64: the sort path
def test_candidates_match_oracle(dev, n, S):
    L1, radius = 4, math.radians(50.0 if n >= 300 else 80.0)
    w, Bs, p, c, t, F = _pair16_case(dev, 3, L1)
    g = synth.super_fibonacci(n)
    grid = bh.bh_grid_create(g, radius)
    starts, idx, sc = bh.bh_candidates(p, grid, c[0].contiguous(), c[1:].contiguous(), L1, S, with_index=True,
                                       with_scores=True)
    starts, idx, sc = starts.cpu().numpy(), idx.cpu().numpy(), sc.cpu().numpy()
    nb = candidates.grid_neighbors(g, radius)
    for b in range(w.B):
        xi = align.build_xi(Bs, t, F[b], L1)
        ref = candidates.grid_scores(xi, g, L1)
        scale = math.sqrt(sum(np.sum(np.abs(ball.split_by_degree(Bs, t)[l]) ** 2) for l in range(L1 + 1)) *
                          sum(np.sum(np.abs(ball.split_by_degree(Bs, F[b])[l]) ** 2) for l in range(L1 + 1)))
        tol = 1e-4 * scale
        assert np.abs(sc[b].astype(np.float64) - ref).max() <= tol
        # the kernel's selection is the one its own scores define, and its starts are those grid entries
        assert np.array_equal(idx[b], selection_from(sc[b], nb, S))
        assert np.array_equal(starts[b], g[idx[b]])
        # where the oracle's FP64 decisions are robust to the score tolerance, the indices agree
        cand = candidates.candidates(ref, nb, S)
        k = robust_prefix(ref, nb, cand, 2 * tol)
        assert np.array_equal(idx[b][:k], cand[:k]), (b, k, idx[b][:k], cand[:k])
        if S >= 8:
            assert k >= 1
    grid.destroy()
    p.destroy()


def test_grid_factors_cached_per_band(dev):
    """The grid's Wigner factors are built on the first call for a band and reused: repeated calls, calls
    for another band in between, and a second plan sharing the grid give bitwise the same scores and
    candidates; each band's scores match the oracle."""
    w, Bs, p, c, t, F = _pair16_case(dev, 3, 4)
    g = synth.super_fibonacci(500)
    grid = bh.bh_grid_create(g, math.radians(40.0))
    tm, sub = c[0].contiguous(), c[1:].contiguous()
    first = [x.cpu().numpy() for x in bh.bh_candidates(p, grid, tm, sub, 4, 6, with_index=True, with_scores=True)]
    other = [x.cpu().numpy() for x in bh.bh_candidates(p, grid, tm, sub, 2, 6, with_index=True, with_scores=True)]
    again = [x.cpu().numpy() for x in bh.bh_candidates(p, grid, tm, sub, 4, 6, with_index=True, with_scores=True)]
    p2 = bh.bh_plan_create(16, 8, 8 * math.pi, bh.BH_MODE_FP32)
    c2 = bh.bh_expand(p2, torch.from_numpy(np.concatenate([w.template[None], w.vols])).to(dev))
    assert torch.equal(c2, c)  # the same coefficients from a second plan
    third = [x.cpu().numpy() for x in bh.bh_candidates(p2, grid, c2[0].contiguous(), c2[1:].contiguous(), 4, 6,
                                                         with_index=True, with_scores=True)]
    for a, b in zip(first, again):
        assert np.array_equal(a, b)
    for a, b in zip(first, third):
        assert np.array_equal(a, b)
    for L, res in ((4, first), (2, other)):
        for b in range(w.B):
            ref = candidates.grid_scores(align.build_xi(Bs, t, F[b], L), g, L)
            scale = math.sqrt(sum(np.sum(np.abs(ball.split_by_degree(Bs, t)[l]) ** 2) for l in range(L + 1)) *
                              sum(np.sum(np.abs(ball.split_by_degree(Bs, F[b])[l]) ** 2) for l in range(L + 1)))
            assert np.abs(res[2][b].astype(np.float64) - ref).max() <= 1e-4 * scale, (L, b)
    grid.destroy()
    p2.destroy()
    p.destroy()


def test_candidate_pipeline_reaches_oracle_optimum(dev):
    """Sec. III pipeline: band-4 candidates -> marching ascent 4-8 from them; GPU vs oracle end to end."""
    L1, S, n, radius = 4, 8, 1000, math.radians(50.0)
    w, Bs, p, c, t, F = _pair16_case(dev, 3, L1)
    g = synth.super_fibonacci(n)
    grid = bh.bh_grid_create(g, radius)
    starts, idx, _ = bh.bh_candidates(p, grid, c[0].contiguous(), c[1:].contiguous(), L1, S, with_index=True)
    q, s = bh.bh_align_batch(p, c[0].contiguous(), c[1:].contiguous(), starts, [4, 8], 40)
    q, s = q.cpu().numpy().astype(np.float64), s.cpu().numpy()
    for b in range(w.B):
        oidx, ref = candidates.align_from_candidates(Bs, t, F[b], g, radius, S, [4, 8], 40)
        qb = q[b] / np.linalg.norm(q[b])
        assert math.degrees(wigner.geodesic_angle(qb, ref.q)) < 0.1
        assert abs(float(s[b]) - ref.score) < 1e-4 * abs(ref.score)
        assert math.degrees(wigner.geodesic_angle(qb, wigner.quat_conj(w.q_true[b]))) < 5.0
    grid.destroy()
    p.destroy()


def test_candidates_batch32_shape_properties(dev):
    """1024 x 32^3 shape (l <= 16, band 4, 4608-point grid, 16 candidates): every subtomogram's selection is
    the one its own scores define; sampled grid scores agree with the oracle."""
    w = synth.make_workload("batch32", count=1024)
    p = bh.bh_plan_create(w.N, w.Lmax, w.lam_max, bh.BH_MODE_BF16_SPLIT, max_batch=1024)
    c = bh.bh_expand(p, torch.from_numpy(np.concatenate([w.template[None], w.vols])).to(dev))
    g = synth.super_fibonacci(4608)
    radius = math.radians(25.0)
    grid = bh.bh_grid_create(g, radius)
    starts, idx, sc = bh.bh_candidates(p, grid, c[0].contiguous(), c[1:].contiguous(), 4, 16, with_index=True,
                                       with_scores=True)
    idx, sc = idx.cpu().numpy(), sc.cpu().numpy()
    nb = grid.neighbors()
    for b in list(range(0, 1024, 97)) + [1023]:
        assert np.array_equal(idx[b], selection_from(sc[b], nb, 16))
    Bs = ball.make_basis(w.Lmax, w.lam_max)
    t = ball.expand(Bs, w.template.astype(np.float64))[0]
    for b in (0, 511, 1023):
        f = ball.expand(Bs, w.vols[b].astype(np.float64))[0]
        xi = align.build_xi(Bs, t, f, 4)
        T4 = ball.split_by_degree(Bs, t)
        F4 = ball.split_by_degree(Bs, f)
        scale = math.sqrt(sum(np.sum(np.abs(T4[l]) ** 2) for l in range(5)) *
                          sum(np.sum(np.abs(F4[l]) ** 2) for l in range(5)))
        for i in (0, 1234, 4607, int(idx[b][0])):
            assert abs(float(sc[b, i]) - align.score(xi, g[i].astype(np.float64), 4)) <= 1e-4 * scale
    grid.destroy()
    p.destroy()


def test_candidate_argument_errors(dev):
    p = bh.bh_plan_create(16, 8, 8 * math.pi, bh.BH_MODE_FP32)
    g = synth.super_fibonacci(50)
    with pytest.raises(bh.BHError):
        bh.bh_grid_create(g, -0.1)
    with pytest.raises(bh.BHError):
        bh.bh_grid_create(np.zeros((0, 4), np.float32), 0.5)
    grid = bh.bh_grid_create(g, 0.5)
    t = torch.zeros((1, p.Nb, 2), device=dev)
    with pytest.raises(bh.BHError):
        bh.bh_candidates(p, grid, t[0], t, 4, 51)  # S > n
    with pytest.raises(bh.BHError):
        bh.bh_candidates(p, grid, t[0], t, 9, 4)  # band above Lmax
    s0, _, _ = bh.bh_candidates(p, grid, t[0], t[:0], 4, 4)  # empty batch
    assert s0.shape == (0, 4, 4)
    grid.destroy()
    p.destroy()
