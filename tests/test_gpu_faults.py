"""Failure vocabulary on the GPU without any device fault: bad inputs are rejected on the
host, infeasible accounts and iteration caps map to the paper's statuses (Table
"Status vocabulary", Sec. 10.2)."""
import dataclasses

import numpy as np
import pytest

from paper_2606_23367_gb300 import build, prism
from paper_2606_23367_gb300.workloads import make_workload
from tests.parity_util import gpu_solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    prism.load_library()


def _expect_arg_error(uni, batch):
    with pytest.raises(prism.PrismError) as ei:
        gpu_solve(uni, batch, precision=prism.PRISM_BATCHED_FP32)
    assert ei.value.code == prism.PRISM_ERR_ARGUMENT


def test_nan_input_rejected():
    uni, batch = make_workload(0)
    batch.w0[3] = np.nan
    _expect_arg_error(uni, batch)


def test_lower_above_upper_rejected():
    uni, batch = make_workload(0)
    batch.lower[5] = batch.upper[5] + 0.1
    _expect_arg_error(uni, batch)


def test_duplicate_asset_rejected():
    uni, batch = make_workload(2, N=300, M=2)
    sl = batch.account_slice(0)
    batch.asset_idx[sl.start + 1] = batch.asset_idx[sl.start]
    _expect_arg_error(uni, batch)


def test_infeasible_account_gets_no_feasible_return():
    uni, batch = make_workload(1, N=600, K=16, M=3)
    sl = batch.account_slice(1)
    batch.upper[sl] = 1e-4            # capacity far below the budget
    res = gpu_solve(uni, batch, precision=prism.PRISM_BATCHED_FP32)
    assert res["status"][1] == prism.PRISM_NO_FEASIBLE_RETURN
    assert res["status"][0] == prism.PRISM_CERTIFIED and res["status"][2] == prism.PRISM_CERTIFIED


def test_iteration_cap_gives_timeout_or_certified():
    uni, batch = make_workload(1, N=600, K=16, M=2)
    res = gpu_solve(uni, batch, precision=prism.PRISM_BATCHED_FP32, max_iter=2, min_iter=1,
                    check_every=1, polish_rounds=1)
    assert set(res["status"].tolist()) <= {prism.PRISM_TIMEOUT, prism.PRISM_CERTIFIED}


@pytest.mark.parametrize("mode", [prism.PRISM_BATCHED_FP32, prism.PRISM_BATCHED_BF16])
def test_empty_account_gets_no_feasible_return(mode):
    # a ragged account with no names cannot meet the budget; its neighbours are unaffected
    uni, batch = make_workload(2, N=300, M=3)
    keep = np.ones(batch.w0.shape[0], bool)
    keep[batch.account_slice(1)] = False
    offsets = batch.offsets.copy()
    n1 = offsets[2] - offsets[1]
    offsets[2:] -= n1
    empty = dataclasses.replace(batch, offsets=offsets, asset_idx=batch.asset_idx[keep], w0=batch.w0[keep],
                                lower=batch.lower[keep], upper=batch.upper[keep], tc=batch.tc[keep])
    res = gpu_solve(uni, empty, precision=mode)
    assert res["status"][1] == prism.PRISM_NO_FEASIBLE_RETURN
    assert res["status"][0] == prism.PRISM_CERTIFIED and res["status"][2] == prism.PRISM_CERTIFIED


@pytest.mark.parametrize("excess", [-1e-7, 1e-7])
def test_capacity_at_the_threshold_is_decided_exactly(excess):
    # total capacity 1 -/+ 1e-7 with no binding band: too close for the FP32 sums, so the
    # closed-form test decides it from FP64 sums (infeasible below 1, attempted above)
    uni, batch = make_workload(1, N=600, K=16, M=2)
    sl = batch.account_slice(1)
    batch.upper[sl] = (1.0 + excess) / 600
    batch.band_hi[1, :] = np.inf
    res = gpu_solve(uni, batch, precision=prism.PRISM_BATCHED_BF16, max_iter=60, polish_rounds=2)
    if excess < 0:
        assert res["status"][1] == prism.PRISM_NO_FEASIBLE_RETURN
    else:
        assert res["status"][1] != prism.PRISM_NO_FEASIBLE_RETURN
    assert res["status"][0] == prism.PRISM_CERTIFIED


def test_time_budget_gives_timeout():
    # a wall-clock budget that runs out during the first graph chunk: the call returns at the
    # chunk's end, the accounts still iterating get TIMEOUT (unless the one polish round already
    # certifies them), and no account ran past that chunk
    uni, batch = make_workload(1, N=600, K=16, M=6)
    res = gpu_solve(uni, batch, precision=prism.PRISM_BATCHED_BF16, time_budget_s=1e-9, check_every=1,
                    stream_after=1, polish_rounds=1)
    st = res["status"]
    assert set(st.tolist()) <= {prism.PRISM_TIMEOUT, prism.PRISM_CERTIFIED}, st
    assert (st == prism.PRISM_TIMEOUT).any(), st
    assert int(res["iters"].max()) <= 2


@pytest.mark.parametrize("mode", [prism.PRISM_BATCHED_FP32, prism.PRISM_BATCHED_BF16])
def test_fp32_overflow_gives_numerical_failure(mode):
    # mu_7 = 1e39 is finite in FP64 (accepted at the boundary) but overflows the FP32 iterates:
    # every account meets Inf/NaN in its iterations and returns NUMERICAL_FAILURE, the call
    # itself succeeds, and the context stays usable for the next solve
    uni, batch = make_workload(1, N=600, K=16, M=3)
    mu = uni.mu.copy()
    mu[7] = 1e39
    bad = dataclasses.replace(uni, mu=mu)
    res = gpu_solve(bad, batch, precision=mode, max_iter=200)
    assert np.all(res["status"] == prism.PRISM_NUMERICAL_FAILURE), res["status"]
    ok = gpu_solve(uni, batch, precision=mode)
    assert np.all(ok["status"] == prism.PRISM_CERTIFIED), ok["status"]


def test_bounded_tensor_core_wait_runs_out_and_reports(monkeypatch):
    # the library's failure-path hook makes the tensor-core G2 wait on a barrier that nothing
    # completes (no load is issued, so nothing is in flight); the wait gives up after 1 ms, the
    # kernel sets its error flag and returns, and the call reports PRISM_ERR_CUDA; the next call,
    # without the hook, solves normally on the same context
    uni, batch = make_workload(1, N=600, K=16, M=3)
    monkeypatch.setenv("PRISM_TEST_STALLED_WAIT_NS", "1000000")
    with pytest.raises(prism.PrismError) as ei:
        gpu_solve(uni, batch, precision=prism.PRISM_BATCHED_BF16)
    assert ei.value.code == prism.PRISM_ERR_CUDA
    assert "timed out" in str(ei.value)
    monkeypatch.delenv("PRISM_TEST_STALLED_WAIT_NS")
    res = gpu_solve(uni, batch, precision=prism.PRISM_BATCHED_BF16)
    assert np.all(res["status"] == prism.PRISM_CERTIFIED), res["status"]
