"""The autotuner (prism_autotune) picks a schedule from its grids, and a solve with that schedule
certifies every account and matches the oracle."""
import numpy as np
import pytest

from paper_2606_23367_gb300 import build, prism
from paper_2606_23367_gb300.workloads import make_workload
from tests.parity_util import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    prism.load_library()


def test_autotune_schedule_is_valid_and_certifies():
    uni, batch = make_workload(4, N=400, K=16, M=16)
    h = prism.create_universe(uni)
    try:
        tuned = prism.autotune(h, batch, precision=prism.PRISM_BATCHED_BF16)
        assert tuned["rho0"] in (0.5, 1.0, 2.0, 3.0, 5.0, 8.0)
        assert tuned["alpha"] in (1.4, 1.5, 1.6, 1.7, 1.8)
        assert tuned["check_every"] in (5, 10, 20)
        assert tuned["stream_after"] in (2, 4, 6, 8, 10)
        assert tuned["eps_admm"] in (1e-4, 2e-4, 3e-4, 5e-4, 7e-4)
        assert tuned["chains"] in (0, 1, 2, 4)
        assert tuned["g2_sets"] in (0, 1, 2, 3, 4)
        assert tuned["ragged_layout"] in (0, 1, 2)
        assert tuned["fold_products"] in (0, 1)
        assert tuned["adapt_every"] in (10, 15, 25, 50)
        assert tuned["precision"] == prism.PRISM_BATCHED_BF16
        opts = {k: tuned[k] for k in ("rho0", "alpha", "check_every", "stream_after", "chains", "eps_admm",
                                      "precision", "g2_sets", "fold_products", "adapt_every")}
        res = prism.solve(h, batch, **opts)
        assert np.all(res["status"] == prism.PRISM_CERTIFIED)
        assert_parity(uni, batch, res, accounts=[0, 7, 15])
    finally:
        h.close()


def test_autotune_plain_mode_is_returned_unchanged():
    uni, batch = make_workload(0)
    h = prism.create_universe(uni)
    try:
        tuned = prism.autotune(h, batch, precision=prism.PRISM_PLAIN_FP32, rho0=0.7)
        assert tuned["rho0"] == 0.7 and tuned["precision"] == prism.PRISM_PLAIN_FP32
    finally:
        h.close()
