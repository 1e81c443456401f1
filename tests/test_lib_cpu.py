"""The C-ABI library without a GPU: it loads, exports every symbol include/bh.h declares, and its
host-only FP64 basis data (roots lambda_lk, constants c_lk; Sec. II-A) agree with the oracle."""
import math
import os
import re

import numpy as np
import pytest

from paper_2509_01180_gb300 import bh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    if not os.path.exists(bh.LIB_PATH):
        from paper_2509_01180_gb300 import build
        build.build()
    return bh.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bh.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bh_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(built):
    names = declared_functions()
    assert set(names) == set(bh.EXPORTS)
    for n in names:
        assert hasattr(built, n), n


def test_status_strings(built):
    assert built.bh_status_string(0) == b"BH_OK"
    assert built.bh_status_string(-5) == b"BH_ERR_TIMEOUT"
    assert built.bh_version() >= 10000


@pytest.mark.parametrize("N,L", [(16, 8), (32, 16), (64, 32)])
def test_host_roots_and_constants_match_oracle(built, N, L):
    from oracle import ball
    lam_max = math.pi * N / 2
    K, lam, c = bh.bh_basis_roots(L, lam_max)
    B = ball.make_basis(L, lam_max)
    assert list(K) == B.K
    assert np.allclose(lam, np.concatenate(B.roots), rtol=0, atol=1e-12)
    assert np.allclose(c, np.concatenate(B.consts), rtol=1e-11)


def test_basis_roots_argument_errors(built):
    with pytest.raises(bh.BHError):
        bh.bh_basis_roots(-1, 10.0)
    with pytest.raises(bh.BHError):
        bh.bh_basis_roots(4, -1.0)


def test_plan_create_without_gpu_fails_cleanly(built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(bh.BHError) as e:
        bh.bh_plan_create(16, 8)
    assert e.value.status in (bh.BH_ERR_CUDA, bh.BH_ERR_UNSUPPORTED)


def test_random_starts_are_deterministic_uniform_rotations(built):
    q = bh.bh_random_starts(2509, 400, 50)
    assert q.shape == (400, 50, 4)
    assert np.allclose(np.linalg.norm(q, axis=-1), 1.0, atol=1e-6)
    assert (q[..., 0] >= 0).all()
    assert np.array_equal(q, bh.bh_random_starts(2509, 400, 50))
    # start (b, s) depends only on (seed, b, s): a prefix of a larger batch is the smaller batch
    assert np.array_equal(bh.bh_random_starts(7, 3, 50), bh.bh_random_starts(7, 5, 50)[:3])
    # Haar measure: E[q_i^2] = 1/4 for every component, and E[trace R] = 0 (trace R = 4 w^2 - 1)
    m2 = (q.reshape(-1, 4).astype(np.float64) ** 2).mean(axis=0)
    assert np.allclose(m2, 0.25, atol=0.01)
    assert abs(np.mean(4 * q[..., 0].astype(np.float64) ** 2 - 1)) < 0.02
