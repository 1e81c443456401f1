"""bh_expand_noalloc: the expansion entry point that allocates nothing, for callers that cannot call
cudaMalloc while they run (for example a thread recording into a stream another component captures into
a CUDA graph, or an application that owns all device memory and only lends pointers).  Its scratch is a
fixed array compiled into the library, so its output must equal bh_expand's, call after call.

Collected last on purpose (file name), so a run that stops at the first failure has run everything else;
it creates its own plans and passes alone in a fresh process as well as after the other tests."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2509_01180_gb300 import bh  # noqa: E402


def _rel_rows(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    a = a[..., 0] + 1j * a[..., 1]
    b = b[..., 0] + 1j * b[..., 1]
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def _noalloc(plan, vols):
    out = torch.full((vols.shape[0], plan.Nb, 2), float("nan"), dtype=torch.float32, device=vols.device)
    st = bh.lib().bh_expand_noalloc(plan.handle, vols.data_ptr(), vols.shape[0], out.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert st == bh.BH_OK, bh.lib().bh_last_error()
    return out


@pytest.mark.parametrize("mode", [bh.BH_MODE_FP32, bh.BH_MODE_BF16_SPLIT])
@pytest.mark.parametrize("N,L,B", [(16, 8, 37), (32, 16, 800)])
def test_noalloc_matches_bh_expand_on_two_calls(mode, N, L, B):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    dev = torch.device("cuda:0")
    plan = bh.bh_plan_create(N, L, math.pi * N / 2, mode, max_batch=256)
    rng = np.random.default_rng(N * 1000 + B + mode)
    for call in range(2):  # two calls in a row: the shared array keeps the previous call's contents
        vols = torch.from_numpy(rng.normal(size=(B, N, N, N)).astype(np.float32)).to(dev)
        ref = bh.bh_expand(plan, vols)
        got = _noalloc(plan, vols)
        torch.cuda.synchronize()
        assert bool(torch.isfinite(got).all())
        rel = _rel_rows(got, ref)
        assert rel.max() < 1e-4, (call, float(rel.max()))
    plan.destroy()


def test_noalloc_rejects_plans_above_its_fixed_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    # a 64^3 box: one 128-row pass needs 128 * (137088 + 256) * 4 bytes > 64 MiB
    plan = bh.bh_plan_create(64, 2, 0.0, bh.BH_MODE_FP32, max_batch=128)
    vols = torch.zeros((1, 64, 64, 64), dtype=torch.float32, device="cuda:0")
    out = torch.zeros((1, plan.Nb, 2), dtype=torch.float32, device="cuda:0")
    st = bh.lib().bh_expand_noalloc(plan.handle, vols.data_ptr(), 1, out.data_ptr(), 0)
    assert st == bh.BH_ERR_ARG
    assert b"scratch" in bh.lib().bh_last_error()
    plan.destroy()
