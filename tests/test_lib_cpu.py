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
