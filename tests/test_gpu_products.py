"""Kernel-level parity of the x-update's shared-B products (G2: P = X B, G4: BQ = Q B').

The reference restates each product in FP64 numpy with the operands the kernels
are defined on: FP32-rounded X, Q and B for the SIMT path; for the tensor-core
path B rounded to BF16 (round-to-nearest-even) and X, Q split as hi = bf16(v),
lo = bf16(v - hi). What is left is FP32 accumulation, bounded here by
1e-5 x sum |terms| (K or N terms of FP32 rounding, far below it). The tensor-core
P is checked twice: from the separate G2 kernel, and from the fused x-update
kernel's own product (B tile read transposed, X tile from the epilogue, partials
summed over each cluster of asset tiles), which carries G2 inside the iteration.
"""
import numpy as np
import pytest

from paper_2606_23367_gb300 import build, prism
from paper_2606_23367_gb300.workloads import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    prism.load_library()


def bf16(x):
    """Round FP32 values to BF16 (nearest, ties to even), returned as FP64."""
    x = np.asarray(x, np.float32)
    b = x.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def split(x):
    x32 = np.asarray(x, np.float32)
    hi = bf16(x32)
    lo = bf16((x32.astype(np.float64) - hi).astype(np.float32))
    return hi, lo


@pytest.mark.parametrize("N,K,M", [(1200, 64, 130), (700, 32, 5), (10000, 64, 500), (333, 48, 129)])
@pytest.mark.parametrize("precision", [prism.PRISM_BATCHED_BF16, prism.PRISM_BATCHED_BF16 | prism.PRISM_PRODUCTS_FUSED,
                                       prism.PRISM_BATCHED_FP32])
def test_products_match_restatement(N, K, M, precision):
    uni, _ = make_workload(1, N=N, K=K, M=1)
    rng = np.random.default_rng(N + K + M)
    X = rng.normal(0.0, 0.05, size=(M, N))
    Q = rng.normal(0.0, 0.02, size=(M, K))
    h = prism.create_universe(uni)
    try:
        P, BQ = prism.prism_shared_b_products(h, X, Q, precision)
    finally:
        h.close()
    if precision & 0xff == prism.PRISM_BATCHED_BF16:
        Bm = bf16(uni.B.astype(np.float32))
        xh, xl = split(X)
        qh, ql = split(Q)
        Xe, Qe = xh + xl, qh + ql
    else:
        Bm = uni.B.astype(np.float32).astype(np.float64)
        Xe = X.astype(np.float32).astype(np.float64)
        Qe = Q.astype(np.float32).astype(np.float64)
    P_ref = Xe @ Bm
    BQ_ref = Qe @ Bm.T
    P_scale = np.abs(Xe) @ np.abs(Bm)
    BQ_scale = np.abs(Qe) @ np.abs(Bm).T
    assert np.all(np.abs(P - P_ref) <= 1e-5 * P_scale + 1e-12)
    assert np.all(np.abs(BQ - BQ_ref) <= 1e-5 * BQ_scale + 1e-12)
