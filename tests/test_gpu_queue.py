"""The queue harness through the C-ABI: every account accepted inside the window, one audit
record each, and the same weights as one call over the whole book; the burden bundles solve
and certify."""
import numpy as np
import pytest

from paper_2606_23367_gb300 import build, prism
from paper_2606_23367_gb300.queue import burden_books, library_solver, run_queue
from paper_2606_23367_gb300.workloads import make_workload
from tests.parity_util import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    prism.load_library()


def test_queue_of_micro_batches_matches_one_call():
    uni, batch = make_workload(1, N=700, K=32, M=40)
    h = prism.create_universe(uni)
    try:
        r = run_queue(uni, batch, library_solver(h, precision=prism.PRISM_BATCHED_BF16), window_s=60.0,
                      micro_batch=10, keep_outputs=True)
        whole = prism.solve(h, batch, precision=prism.PRISM_BATCHED_BF16)
    finally:
        h.close()
    assert r.completed == 40 and r.missed_rate == 0.0 and r.audit_coverage == 1.0 and r.calls == 4
    assert r.status_counts == {"CERTIFIED": 40}
    assert 0 < r.p50_ms <= r.p99_ms <= r.t_queue_s * 1e3
    assert np.all(whole["status"] == prism.PRISM_CERTIFIED)
    # the same accounts in other batch compositions: the same polished weights, up to rounding
    assert float(np.max(np.abs(r.w - whole["w"]))) <= 1e-9
    assert sorted(rec["account"] for rec in r.records) == list(range(40))
    assert len({rec["input_sha256"] for rec in r.records}) == 40
    assert all(rec["status"] == "CERTIFIED" and len(rec["output_sha256"]) == 64 for rec in r.records)
    assert_parity(uni, batch, whole, accounts=[0, 17, 39])


def test_burden_bundles_certify():
    for name, family, uni, batch in burden_books(N=600, K=16, M=8):
        if batch is None:
            continue
        h = prism.create_universe(uni)
        try:
            res = prism.solve(h, batch, precision=prism.PRISM_BATCHED_BF16)
        finally:
            h.close()
        assert np.all(res["status"] == prism.PRISM_CERTIFIED), (name, res["status"])
        assert_parity(uni, batch, res, accounts=[0, 7])
