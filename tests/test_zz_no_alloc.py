"""The allocation-free entry point (prism_polish_noalloc) against prism_solve_batch and the oracle.

prism_polish_noalloc serves callers that cannot allocate device memory when they
need a result (a process that has reserved the whole GPU for its own pool, or a
latency-bound thread that must not wait on the allocator). It polishes and certifies
weights the caller already holds, with its scratch in a static device array shared by
every call. Here it is handed prism_solve_batch's own certified weights and points
near them that are not optimal (host and device buffers), twice in a row each, and
must return the same answer within the parity tolerances; its limits are checked. The
file is named so that pytest collects it last.
"""
import dataclasses

import numpy as np
import pytest

from paper_2606_23367_gb300 import build, prism
from paper_2606_23367_gb300.workloads import make_workload
from tests.parity_util import W_TOL, check_account, compare_account

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    prism.load_library()


def _noalloc(h, batch, w_in, **kw):
    return prism.prism_polish_noalloc(h, batch.offsets, batch.w0, batch.lower, batch.upper, batch.tc,
                                      batch.band_lo, batch.band_hi, w_in, asset_idx=batch.asset_idx,
                                      turnover_cap=batch.turnover_cap, **kw)


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


def _perturbed_start(batch, w, seed):
    """w moved off the optimum: every weight strictly inside a linear piece of its cost (not on
    a bound, not at its current holding) gets a relative change of up to 1e-4, the result
    clipped to the box. The budget, sector sums and turnover move off their edges (by less
    than the entry point's 1e-4 warm-start margin), and the free weights off their values."""
    r = np.random.default_rng(seed)
    inside = (w > batch.lower + 1e-12) & (w < batch.upper - 1e-12) & (np.abs(w - batch.w0) > 1e-12)
    w2 = w * (1.0 + 1e-4 * r.uniform(-1.0, 1.0, size=w.shape) * inside)
    return np.clip(w2, batch.lower, batch.upper)


# (workload, sizes): a shared-universe book and a capped book without lots, whose cap binds
CASES = [(1, dict(N=1200, K=64, M=4)), (3, dict(N=400, K=12, M=4, lots=False))]


@pytest.mark.parametrize("on_device", [False, True])
@pytest.mark.parametrize("workload,kw", CASES)
def test_noalloc_from_a_perturbed_start_against_the_oracle(workload, kw, on_device):
    uni, batch = make_workload(workload, **kw)
    if workload == 3:
        assert np.isfinite(batch.turnover_cap).all()
    h = prism.create_universe(uni)
    try:
        ref = prism.solve(h, batch, precision=prism.PRISM_BATCHED_FP32)
        assert (ref["status"] == prism.PRISM_CERTIFIED).all()
        w_in = _perturbed_start(batch, ref["w"], seed=workload)
        assert np.max(np.abs(w_in - ref["w"])) > 1e-7
        src = batch
        if on_device:
            torch = pytest.importorskip("torch")
            dev = lambda x: None if x is None else torch.as_tensor(np.ascontiguousarray(x)).cuda()
            src = dataclasses.replace(batch, offsets=dev(batch.offsets), w0=dev(batch.w0), lower=dev(batch.lower),
                                      upper=dev(batch.upper), tc=dev(batch.tc), band_lo=dev(batch.band_lo),
                                      band_hi=dev(batch.band_hi), turnover_cap=dev(batch.turnover_cap),
                                      asset_idx=dev(batch.asset_idx))
            w_in = dev(w_in)
        for _ in range(2):
            got = _noalloc(h, src, w_in, polish_rounds=16)
            got = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in got.items()}
            for a in range(batch.n_accounts):
                check_account(compare_account(uni, batch, got, a), a)
            if workload == 3:
                # the cap binds for at least one account, so its row was rebuilt from the start
                assert np.any(got["theta"] > 0)
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
    # 14 accounts x 10,048 padded positions = 140,672 entries > 131,072
    uni, batch = make_workload(1, N=10000, K=8, M=14)
    h = prism.create_universe(uni)
    try:
        with pytest.raises(prism.PrismError) as ei:
            _noalloc(h, batch, batch.w0)
        assert ei.value.code == prism.PRISM_ERR_ARGUMENT
        assert "131072" in str(ei.value)
    finally:
        h.close()


def test_noalloc_more_free_weights_than_its_limit_fall_back():
    # a budget-only long-only book with mu = 0 and no transition cost: every one of the 1,200
    # weights is free at the optimum, beyond the entry point's 512; the allocating solve
    # certifies it, the allocation-free one returns the given weights uncertified
    uni, batch = make_workload(4, N=1200, K=4, M=1, upper=(1.0, 1.0), tc=(0.0, 0.0), band_hi=1.0, held=None,
                               excl=(0.0, 0.0))
    uni = dataclasses.replace(uni, mu=np.zeros(uni.n_assets))
    h = prism.create_universe(uni)
    try:
        ref = prism.solve(h, batch, precision=prism.PRISM_BATCHED_FP32)
        assert ref["status"][0] == prism.PRISM_CERTIFIED
        n_free = int(((ref["w"] > 1e-12) & (ref["w"] < 1.0 - 1e-12)).sum())
        assert n_free > 512
        got = _noalloc(h, batch, ref["w"])
        assert got["status"][0] in (prism.PRISM_FEASIBLE_NONCERTIFIED, prism.PRISM_NO_FEASIBLE_RETURN)
        assert not np.isfinite(got["diag"][0, prism.PRISM_DIAG_ERR_EST])
    finally:
        h.close()
