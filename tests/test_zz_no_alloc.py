"""The allocation-free entry point (prism_polish_noalloc) against prism_solve_batch.

prism_polish_noalloc serves callers that cannot allocate device memory when they
need a result (a process that has reserved the whole GPU for its own pool, a
latency-bound thread, code recording a CUDA graph). It polishes and certifies
weights the caller already holds, with its scratch in a static device array.
Here it is handed prism_solve_batch's own certified weights, twice in a row, and
must return them, with the same statuses, within the parity tolerance. The file
is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2606_23367_gb300 import build, prism
from paper_2606_23367_gb300.workloads import make_workload
from tests.parity_util import W_TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    prism.load_library()


def _noalloc(h, batch, w_in):
    return prism.prism_polish_noalloc(h, batch.offsets, batch.w0, batch.lower, batch.upper, batch.tc,
                                      batch.band_lo, batch.band_hi, w_in, asset_idx=batch.asset_idx,
                                      turnover_cap=batch.turnover_cap)


@pytest.mark.parametrize("workload,kw", [(0, {}), (1, dict(N=1200, K=64, M=4)), (2, dict(N=900, M=5))])
def test_noalloc_matches_solve_batch_twice(workload, kw):
    uni, batch = make_workload(workload, **kw)
    h = prism.create_universe(uni)
    try:
        ref = prism.solve(h, batch, precision=prism.PRISM_BATCHED_FP32)
        assert (ref["status"] == prism.PRISM_CERTIFIED).all()
        for _ in range(2):
            got = _noalloc(h, batch, ref["w"])
            assert np.array_equal(got["status"], ref["status"])
            assert np.max(np.abs(got["w"] - ref["w"])) <= W_TOL
            assert np.max(np.abs(got["diag"][:, 6] - ref["diag"][:, 6])) <= 1e-8 * np.max(np.abs(ref["diag"][:, 6]))
            assert got["diag"][:, 4].max() <= 1e-6 and got["diag"][:, :4].max() <= 1e-6
    finally:
        h.close()


def test_noalloc_rejects_oversized_requests():
    uni, batch = make_workload(1, N=1200, K=16, M=33)
    h = prism.create_universe(uni)
    try:
        with pytest.raises(prism.PrismError) as ei:
            _noalloc(h, batch, batch.w0)
        assert ei.value.code == prism.PRISM_ERR_ARGUMENT
        assert "n_accounts" in str(ei.value)
    finally:
        h.close()
