"""GPU parity for the further families of Eq. 1 (Sec. 4.2): bounds on the factor exposures B'w
(general rows a_lo <= A w <= a_hi with A = B' of the account's names, the constraint-burden
table's bundle B3), a per-account tilt of the return input, and a benchmark in the risk term.

Each book is solved through the C-ABI and every account compared with the FP64 oracle, which
takes the same families as general rows, a shift of mu, and the benchmark's linear term
(tolerances in tests/parity_util.py: 1e-6 max-abs on weights, 1e-8 relative objective, primal
and stationarity residuals <= 1e-6 from the oracle's checker, which also takes the library's
factor multipliers kappa).
"""
import numpy as np
import pytest

from paper_2606_23367_gb300 import build, prism
from paper_2606_23367_gb300.workloads import make_workload
from tests.parity_util import assert_parity, gpu_solve

pytestmark = pytest.mark.gpu

MODES = [prism.PRISM_BATCHED_FP32, prism.PRISM_BATCHED_BF16, prism.PRISM_PLAIN_FP64]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    prism.load_library()


@pytest.mark.parametrize("mode", MODES)
def test_factor_exposure_bounds(mode):
    # the first three factor exposures of every account held to [-0.02, 0.02]
    uni, batch = make_workload(1, N=1200, K=16, M=5, factor_bound=(3, 0.02))
    res = gpu_solve(uni, batch, precision=mode)
    assert_parity(uni, batch, res)
    ex = []
    for a in range(batch.n_accounts):
        w = res["w"][batch.account_slice(a)]
        ex.append(uni.B[batch.account_assets(a, uni.n_assets)].T @ w)
    ex = np.array(ex)
    # some bound binds (else the test would not exercise the rows), and every one holds
    assert np.any(np.abs(np.abs(ex[:, :3]) - 0.02) <= 1e-9)
    assert np.all(np.abs(ex[:, :3]) <= 0.02 + 1e-9)
    assert np.any(res["kappa"][:, :3] != 0.0) and np.all(res["kappa"][:, 3:] == 0.0)


@pytest.mark.parametrize("mode", MODES)
def test_factor_exposure_bounds_with_cap_and_ragged_accounts(mode):
    uni, batch = make_workload(2, N=900, K=12, M=4, factor_bound=(2, 0.03))
    res = gpu_solve(uni, batch, precision=mode)
    assert_parity(uni, batch, res)


@pytest.mark.parametrize("mode", MODES)
def test_return_tilt(mode):
    uni, batch = make_workload(1, N=900, K=16, M=4, tilt=0.01)
    res = gpu_solve(uni, batch, precision=mode)
    assert_parity(uni, batch, res)


@pytest.mark.parametrize("mode", MODES)
def test_benchmark_in_the_risk_term(mode):
    uni, batch = make_workload(1, N=900, K=16, M=4, bench=True)
    res = gpu_solve(uni, batch, precision=mode)
    assert_parity(uni, batch, res)


def test_factor_bounds_at_the_headline_width():
    # 32 accounts x 10,000 assets, K = 64 (the headline universe), four factor exposures bounded,
    # in the launch configuration of the benchmark (batched BF16)
    uni, batch = make_workload(1, M=32, factor_bound=(4, 0.02))
    res = gpu_solve(uni, batch, precision=prism.PRISM_BATCHED_BF16)
    from tests.oracle_pool import compare_all
    from tests.parity_util import check_account
    rows = compare_all(1, res, M=32, factor_bound=(4, 0.02))
    for e in rows:
        e["status"] = int(res["status"][e["account"]])
        check_account(e, e["account"])


def test_backward_rejects_the_factor_block():
    uni, batch = make_workload(1, N=600, K=8, M=2, factor_bound=(2, 0.05))
    with pytest.raises(prism.PrismError) as ei:
        gpu_solve(uni, batch, precision=prism.PRISM_BATCHED_FP32, keep_for_backward=1)
    assert ei.value.code == prism.PRISM_ERR_UNSUPPORTED
