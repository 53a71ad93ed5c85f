"""Failure vocabulary on the GPU without any device fault: bad inputs are rejected on the
host, infeasible accounts and iteration caps map to the paper's statuses (Table
"Status vocabulary", Sec. 10.2)."""
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
