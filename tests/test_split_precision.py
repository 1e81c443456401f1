"""Why the tensor-core expansion runs three BF16 products (hi*hi + hi*lo + lo*hi) and not two.

Emulated on the CPU with the oracle's basis: the volume and the (conjugated, quadrature-weighted) basis
table are each split into a BF16 high part and a BF16 remainder, the products are summed in FP64, and the
coefficients are compared with the FP64 expansion.  Three products stay two orders of magnitude inside the
1e-4 relative coefficient tolerance; dropping either cross product leaves the error of a single BF16
rounding (about 1e-3), ten times outside it.
"""
import numpy as np
import pytest

from oracle import ball
from paper_2509_01180_gb300 import synth


def _bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as FP64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("name,count", [("pair16", None), ("batch32", 2)])
def test_three_products_needed(name, count):
    w = synth.make_workload(name, count=count)
    basis = ball.make_basis(w.Lmax, w.lam_max)
    flat, pts = ball.voxel_ball(w.N)
    psi = np.conj(ball.psi_at(basis, pts)) * (2.0 / w.N) ** 3
    T = np.concatenate([psi.real, psi.imag], axis=1)
    X = w.vols.reshape(w.vols.shape[0], -1)[:, flat].astype(np.float64)
    exact = X @ T
    Th, Xh = _bf16(T), _bf16(X)
    Tl, Xl = _bf16(T - Th), _bf16(X - Xh)

    def rel(C):
        return float(np.max(np.linalg.norm(C - exact, axis=1) / np.linalg.norm(exact, axis=1)))

    assert rel(Xh @ Th + Xh @ Tl + Xl @ Th) < 1e-5
    assert rel(Xh @ Th + Xh @ Tl) > 1e-4
    assert rel(Xh @ Th + Xl @ Th) > 1e-4
