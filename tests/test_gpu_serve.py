"""Serving with continuous batching (request loop over the expansion and alignment kernels), on the GPU.

Checks: a request's result alone equals its result in a mix of requests of other sizes, box edges and
templates (per-subtomogram work depends only on its own inputs); the served result equals the batch API
on the same inputs; HBM-budget admission rejects requests that can never fit; a host-injected stall
(paused admission) makes a bounded wait return BH_ERR_TIMEOUT and the request still completes after
resuming; malformed requests get error codes; many requests overlap in several in-flight batches; the
express class (high-priority streams for small requests) and in-place ingestion (the expansion reading
request buffers in host memory) give the same results as bulk batches and device copies."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2509_01180_gb300 import bh, synth  # noqa: E402


@pytest.fixture(scope="module")
def srv():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    s = bh.bh_serve_create(hbm_budget_bytes=2 << 30, max_inflight=4, max_batch=256, steps=20)
    tids = {}
    for N, seeds in ((16, (11, 12)), (24, (13,))):
        for sd in seeds:
            tpl = synth.blob_template(synth.rng_for(9, sd), 20 if N == 16 else 30, 1.2, 0.75 * N / 2)
            tids[(N, sd)] = s.add_template(synth.render(N, tpl).astype(np.float32))
    yield s, tids
    s.destroy()


def vols_for(N, B, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(B, N, N, N)).astype(np.float32)


def test_alone_equals_in_the_mix(srv):
    s, tids = srv
    R = dict(template_id=tids[(16, 11)], vols=vols_for(16, 5, 1), S=8, seed=77)
    q0, s0, _ = s.wait(s.submit(**R), timeout_ms=60000)
    rng = np.random.default_rng(5)
    tickets = []
    for i in range(14):
        N = 16 if i % 3 else 24
        tid = tids[(16, 12)] if (N == 16 and i % 2) else (tids[(16, 11)] if N == 16 else tids[(24, 13)])
        B = int(rng.integers(1, 40))
        tickets.append(s.submit(tid, vols_for(N, B, 100 + i), S=8 if N == 16 else 16, seed=i))
        if i == 6:
            tr = s.submit(**R)
    res = [s.wait(t, timeout_ms=120000) for t in tickets]
    q1, s1, _ = s.wait(tr, timeout_ms=120000)
    assert np.array_equal(q0, q1) and np.array_equal(s0, s1), (np.abs(q0 - q1).max(), np.abs(s0 - s1).max())
    assert all(np.isfinite(r[1]).all() for r in res)
    assert s.stats()["batches"] >= 2


def test_served_result_equals_batch_api(srv):
    s, tids = srv
    N, B, S, seed = 16, 7, 8, 123
    vols = vols_for(N, B, 9)
    q_srv, sc_srv, _ = s.wait(s.submit(tids[(16, 12)], vols, S, seed=seed), timeout_ms=60000)
    tpl = synth.blob_template(synth.rng_for(9, 12), 20, 1.2, 0.75 * N / 2)
    tvol = synth.render(N, tpl).astype(np.float32)
    plan = bh.bh_plan_create(N, N // 2, math.pi * N / 2, bh.BH_MODE_BF16_SPLIT)
    dev = torch.device("cuda:0")
    t = bh.bh_expand(plan, torch.from_numpy(tvol[None]).to(dev))[0].contiguous()
    c = bh.bh_expand(plan, torch.from_numpy(vols).to(dev))
    starts = torch.from_numpy(bh.bh_random_starts(seed, B, S)).to(dev)
    q, sc = bh.bh_align_batch(plan, t, c, starts, [2, 4, 8], 20)
    assert np.array_equal(q.cpu().numpy(), q_srv) and np.array_equal(sc.cpu().numpy(), sc_srv)
    plan.destroy()


def test_budget_admission_rejects_requests_that_never_fit():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    s = bh.bh_serve_create(hbm_budget_bytes=4 << 20, max_batch=4096)
    tpl = synth.blob_template(synth.rng_for(9, 1), 10, 1.2, 6.0)
    tid = s.add_template(synth.render(16, tpl).astype(np.float32))
    with pytest.raises(bh.BHError) as e:  # > 4 MiB of coefficients and scratch even with volumes read in place
        s.submit(tid, vols_for(16, 1000, 0), S=8)
    assert e.value.status == bh.BH_ERR_BUDGET
    q, sc, _ = s.wait(s.submit(tid, vols_for(16, 1, 0), S=8), timeout_ms=60000)  # a small one still fits
    assert np.isfinite(sc).all()
    s.destroy()


def test_paused_admission_times_out_then_completes(srv):
    s, tids = srv
    s.pause(True)
    t = s.submit(tids[(16, 11)], vols_for(16, 3, 2), S=8)
    with pytest.raises(bh.BHError) as e:
        s.wait(t, timeout_ms=300)
    assert e.value.status == bh.BH_ERR_TIMEOUT
    assert s.poll(t) is None
    s.pause(False)
    q, sc, lat = s.wait(t, timeout_ms=60000)
    assert np.isfinite(sc).all() and lat >= 300.0


def test_malformed_requests(srv):
    s, tids = srv
    v = vols_for(16, 2, 3)
    for kw, code in ((dict(template_id=999, vols=v, S=8), bh.BH_ERR_ARG),
                     (dict(template_id=tids[(16, 11)], vols=v, S=0), bh.BH_ERR_ARG),
                     (dict(template_id=tids[(16, 11)], vols=v, S=4096), bh.BH_ERR_ARG)):
        with pytest.raises(bh.BHError) as e:
            s.submit(**kw)
        assert e.value.status == code
    with pytest.raises(bh.BHError):
        s.wait(123456789, timeout_ms=10)


def test_many_requests_overlap_and_report_latency(srv):
    s, tids = srv
    before = s.stats()["batches"]
    tickets = [s.submit(tids[(24, 13)] if i % 2 else tids[(16, 11)], vols_for(24 if i % 2 else 16, 30, 200 + i),
                        S=16 if i % 2 else 8, seed=i) for i in range(24)]
    lat = [s.wait(t, timeout_ms=120000)[2] for t in tickets]
    st = s.stats()
    assert st["completed"] == st["submitted"] and st["queued"] == 0
    assert st["batches"] - before >= 2
    p50, p99 = np.percentile(lat, [50, 99])
    assert 0 < p50 <= p99


def test_newton_server_equals_batch_api():
    """A server built with Newton steps returns what bh_align_batch with newton=True returns on the same inputs."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    s = bh.bh_serve_create(hbm_budget_bytes=1 << 30, max_inflight=2, max_batch=128, steps=8, newton=True)
    N, B, S, seed = 16, 9, 8, 321
    tpl = synth.blob_template(synth.rng_for(9, 12), 20, 1.2, 0.75 * N / 2)
    tvol = synth.render(N, tpl).astype(np.float32)
    tid = s.add_template(tvol)
    vols = vols_for(N, B, 19)
    q_srv, sc_srv, _ = s.wait(s.submit(tid, vols, S, seed=seed), timeout_ms=60000)
    s.destroy()
    plan = bh.bh_plan_create(N, N // 2, math.pi * N / 2, bh.BH_MODE_BF16_SPLIT)
    dev = torch.device("cuda:0")
    t = bh.bh_expand(plan, torch.from_numpy(tvol[None]).to(dev))[0].contiguous()
    c = bh.bh_expand(plan, torch.from_numpy(vols).to(dev))
    starts = torch.from_numpy(bh.bh_random_starts(seed, B, S)).to(dev)
    q, sc = bh.bh_align_batch(plan, t, c, starts, [2, 4, 8], 8, newton=True)
    assert np.array_equal(q.cpu().numpy(), q_srv) and np.array_equal(sc.cpu().numpy(), sc_srv)
    plan.destroy()


def _server_results(reqs, **kw):
    s = bh.bh_serve_create(hbm_budget_bytes=1 << 30, max_inflight=2, max_batch=256, steps=12, **kw)
    tpl = synth.blob_template(synth.rng_for(9, 21), 30, 1.2, 0.75 * 12)
    tid = s.add_template(synth.render(24, tpl).astype(np.float32))
    tickets = [s.submit(tid, v, S=8, seed=sd) for v, sd in reqs]
    out = [s.wait(t, timeout_ms=120000)[:2] for t in tickets]
    st = s.stats()
    s.destroy()
    return out, st


def test_express_and_in_place_give_the_batch_results():
    """The same requests through every server configuration: express streams or bulk only, volumes read in
    place or copied -- bitwise the same rotations and scores, and the counters say which path ran."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    reqs = [(vols_for(24, B, 300 + i), 40 + i) for i, B in enumerate((1, 3, 40, 7, 120, 2))]
    base, st0 = _server_results(reqs, ingest=1)
    assert st0["express_batches"] == 0 and st0["in_place_batches"] == 0
    for kw in (dict(), dict(express_slots=2), dict(express_slots=2, express_ms=1e9), dict(express_slots=1, ingest=1)):
        out, st = _server_results(reqs, **kw)
        for (q0, s0), (q1, s1) in zip(base, out):
            assert np.array_equal(q0, q1) and np.array_equal(s0, s1), kw
        if kw.get("ingest") == 1:
            assert st["in_place_batches"] == 0
        if kw.get("express_ms") == 1e9:
            assert st["express_batches"] == st["batches"]
        if not kw.get("express_slots"):
            assert st["express_batches"] == 0
        assert st["staging_allocs"] >= 2 and st["launch_ms_max"] >= 0.0


def test_pieces_give_the_unsplit_results():
    """A request admitted in pieces (each next piece queued behind later arrivals) returns bitwise what the
    same request returns unsplit: every subtomogram keeps its own random starts."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    tpl = synth.render(16, synth.blob_template(synth.rng_for(9, 11), 20, 1.2, 6.0)).astype(np.float32)
    vols = vols_for(16, 70, 3)
    out = []
    for piece in (16, 1024):
        s = bh.bh_serve_create(hbm_budget_bytes=1 << 30, max_inflight=3, max_batch=256, steps=10, piece=piece)
        tid = s.add_template(tpl)
        small = [s.submit(tid, vols_for(16, 3, 40 + i), S=8, seed=i) for i in range(3)]
        q, sc, _ = s.wait(s.submit(tid, vols, S=8, seed=5), timeout_ms=120000)
        for t in small:
            s.wait(t, timeout_ms=120000)
        st = s.stats()
        out.append((q, sc, st["batches"], st["completed"]))
        s.destroy()
    (q1, s1, b1, c1), (q2, s2, b2, c2) = out
    assert np.array_equal(q1, q2) and np.array_equal(s1, s2)
    assert b1 >= 5 and c1 == c2 == 4  # 70 subtomograms in pieces of 16; completions count requests
