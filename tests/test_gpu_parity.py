"""GPU parity: the library's certified weights equal the FP64 oracle's (through the C-ABI).

Tolerances (written here, from the workload targets): 1e-6 max-abs on weights,
1e-8 relative objective (guard max(|f*|, 1e-4)), primal and stationarity
residuals <= 1e-6, all after the FP64 polish.
"""
import dataclasses

import numpy as np
import pytest

from paper_2606_23367_gb300 import build, prism
from paper_2606_23367_gb300.workloads import make_workload
from tests.oracle_pool import compare_all
from tests.parity_util import assert_parity, check_account, gpu_solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    prism.load_library()


MODES = [prism.PRISM_BATCHED_FP32, prism.PRISM_BATCHED_BF16, prism.PRISM_PLAIN_FP32, prism.PRISM_PLAIN_FP64]
BATCHED = [prism.PRISM_BATCHED_FP32, prism.PRISM_BATCHED_BF16]


@pytest.mark.parametrize("mode", MODES)
def test_single_account_n100(mode):
    uni, batch = make_workload(0)
    res = gpu_solve(uni, batch, precision=mode)
    assert_parity(uni, batch, res)


@pytest.mark.parametrize("workload,kw", [(1, dict(N=700, K=32, M=2)), (2, dict(N=900, M=3)),
                                         (3, dict(N=400, K=12, M=2))])
def test_plain_fp64_small_books(workload, kw):
    # the FP64 iterations on a shared-universe book, ragged accounts, and tax lots with a cap
    uni, batch = make_workload(workload, **kw)
    res = gpu_solve(uni, batch, precision=prism.PRISM_PLAIN_FP64)
    assert_parity(uni, batch, res)


@pytest.mark.parametrize("mode", BATCHED)
def test_batch_shared_universe_small(mode):
    # 1,200 assets: several 64-wide tiles plus a ragged tail; K = 64 as at full size
    uni, batch = make_workload(1, N=1200, K=64, M=6)
    res = gpu_solve(uni, batch, precision=mode)
    assert_parity(uni, batch, res)


@pytest.mark.parametrize("layout", [1, 2])
@pytest.mark.parametrize("mode", BATCHED)
def test_ragged_accounts_small(mode, layout):
    # ragged accounts dense-masked over the universe (1) and packed, one persistent launch of
    # per-account blocks over each account's own names (2)
    uni, batch = make_workload(2, N=900, M=6)
    res = gpu_solve(uni, batch, precision=mode, ragged_layout=layout)
    assert_parity(uni, batch, res)


@pytest.mark.parametrize("kw", [dict(N=900, M=40), dict(N=10000, K=16, M=16, ragged=(100, 10000))])
def test_packed_and_dense_masked_ragged_layouts_agree(kw):
    # the two layouts run different iterations (the packed one with each account's own
    # capacitance) to the same minimiser: after the FP64 polish the weights agree; the second
    # book has two accounts (7,378 and 9,286 names) too large for shared memory, whose packed
    # state stays in global memory, next to accounts of 123 .. 3,888 names
    uni, batch = make_workload(2, **kw)
    rd = gpu_solve(uni, batch, precision=prism.PRISM_BATCHED_FP32, ragged_layout=1)
    rp = gpu_solve(uni, batch, precision=prism.PRISM_BATCHED_FP32, ragged_layout=2)
    assert np.all(rd["status"] == prism.PRISM_CERTIFIED) and np.all(rp["status"] == prism.PRISM_CERTIFIED)
    assert float(np.max(np.abs(rd["w"] - rp["w"]))) <= 1e-9
    assert_parity(uni, batch, rp, accounts=[0, batch.n_accounts - 1])


def test_packed_ragged_layout_with_lots_cap_and_factor_bounds():
    # the packed layout with tax lots, a turnover cap and factor-exposure bounds together
    uni, batch = make_workload(3, N=600, K=12, M=4, ragged=(100, 600), factor_bound=(2, 0.03))
    res = gpu_solve(uni, batch, precision=prism.PRISM_BATCHED_FP32, ragged_layout=2)
    assert_parity(uni, batch, res)


@pytest.mark.parametrize("mode", BATCHED)
def test_tax_lots_and_turnover_cap_small(mode):
    uni, batch = make_workload(3, N=400, K=12, M=4)
    res = gpu_solve(uni, batch, precision=mode)
    assert_parity(uni, batch, res)


@pytest.mark.parametrize("mode", BATCHED)
def test_differentiation_workload_forward_small(mode):
    uni, batch = make_workload(4, N=500, M=4)
    res = gpu_solve(uni, batch, precision=mode)
    assert_parity(uni, batch, res)


def test_batch_order_does_not_change_results():
    uni, batch = make_workload(1, N=700, K=32, M=5)
    res = gpu_solve(uni, batch, precision=prism.PRISM_BATCHED_FP32)
    order = [3, 1, 4, 0, 2]
    res2 = gpu_solve(uni, batch.subset(order), precision=prism.PRISM_BATCHED_FP32)
    sub = batch.subset(order)
    for k, a in enumerate(order):
        w1 = res["w"][batch.account_slice(a)]
        w2 = res2["w"][sub.account_slice(k)]
        assert np.max(np.abs(w1 - w2)) <= 1e-12


FULL_WORKLOADS = (1, 2, 3, 4)


@pytest.mark.parametrize("workload", FULL_WORKLOADS)
def test_full_size_workloads_every_account_against_the_oracle(workload):
    # each workload at its full size, in the launch configuration the benchmark times (batched
    # BF16, default schedule); the FP64 oracle solves every account in a host process pool and
    # each is held to the parity bar: weights, objective, the oracle checker's residuals of the
    # library's weights and multipliers, and the library's stated error bound
    uni, batch = make_workload(workload)
    res = gpu_solve(uni, batch, precision=prism.PRISM_BATCHED_BF16)
    st = res["status"]
    for s in (prism.PRISM_DIAG_BUDGET, prism.PRISM_DIAG_BOX, prism.PRISM_DIAG_EXPOSURE,
              prism.PRISM_DIAG_TURNOVER, prism.PRISM_DIAG_STAT):
        assert float(res["diag"][:, s].max()) <= 1e-6, s
    rows = compare_all(workload, res)
    assert len(rows) == batch.n_accounts
    for e in rows:
        e["status"] = int(st[e["account"]])
        check_account(e, e["account"])
    worst = max(e["w_err"] for e in rows)
    print(f"workload {workload}: {len(rows)} accounts, max |w - w*| {worst:.2e}, "
          f"max stated bound {max(e['bound'] for e in rows):.2e}")


def _varied_costs_and_floors(batch, seed=7):
    """The same book with a transition cost drawn per entry and a lower bound of 0.001 on
    about 5% of the eligible names: l and c then differ over every account's positions."""
    r = np.random.default_rng(seed)
    tc = r.uniform(5e-4, 5e-3, size=batch.tc.shape)
    lower = np.where((batch.upper > 0.002) & (r.random(batch.lower.shape) < 0.05), 0.001, 0.0)
    return dataclasses.replace(batch, tc=tc, lower=lower)


@pytest.mark.parametrize("varied", [False, True])
def test_fused_prox_matches_separate_kernels(varied):
    # the prox's streaming pass inside the tensor-core x-update against the separate x-update
    # and prox kernels: the same method, so after the FP64 polish the same weights; the varied
    # book takes the fused kernel's per-entry l and c path
    uni, batch = make_workload(1, N=700, K=32, M=20)
    if varied:
        batch = _varied_costs_and_floors(batch)
    rf = gpu_solve(uni, batch, precision=prism.PRISM_BATCHED_BF16, fuse_prox=1)
    ru = gpu_solve(uni, batch, precision=prism.PRISM_BATCHED_BF16, fuse_prox=0)
    assert np.all(rf["status"] == prism.PRISM_CERTIFIED), rf["status"]
    assert np.all(ru["status"] == prism.PRISM_CERTIFIED), ru["status"]
    assert float(np.max(np.abs(rf["w"] - ru["w"]))) <= 1e-9
    assert_parity(uni, batch, rf, accounts=[0, 7, 19])


def test_account_chains_do_not_change_results():
    # the fused iterations cut into 1, 2 or 4 independent account ranges on their own streams:
    # the same arithmetic for every account, so the same weights bit for bit
    uni, batch = make_workload(1, N=600, K=16, M=520)
    res = {ch: gpu_solve(uni, batch, precision=prism.PRISM_BATCHED_BF16, chains=ch) for ch in (1, 2, 4)}
    for ch in (1, 2, 4):
        assert np.all(res[ch]["status"] == prism.PRISM_CERTIFIED), ch
    assert np.array_equal(res[1]["w"], res[2]["w"]) and np.array_equal(res[1]["w"], res[4]["w"])
    assert np.array_equal(res[1]["iters"], res[4]["iters"])
    assert_parity(uni, batch, res[4], accounts=[0, 200, 519])


@pytest.mark.parametrize("sets", [1, 2, 4, 8])
def test_g2_tile_shapes_keep_parity(sets):
    # the tile shape the autotuner searches (asset chunk per CTA of the tensor-core B'X): every
    # shape is the same product summed in another order, so the polished weights agree
    uni, batch = make_workload(1, N=1200, K=64, M=130)
    ref = gpu_solve(uni, batch, precision=prism.PRISM_BATCHED_BF16)
    res = gpu_solve(uni, batch, precision=prism.PRISM_BATCHED_BF16, g2_sets=sets)
    assert np.all(res["status"] == prism.PRISM_CERTIFIED)
    assert float(np.max(np.abs(res["w"] - ref["w"]))) <= 1e-9
    assert_parity(uni, batch, res, accounts=[0, 129])


@pytest.mark.parametrize("varied", [False, True])
@pytest.mark.parametrize("chains", [1, 4])
def test_folded_products_keep_parity(varied, chains):
    # B'X of the pinned entries inside the fused x-update and the rest plus the K x K solve in the
    # roots kernel: the same products in another order (and split), so after the FP64 polish the
    # same weights; the book's penalties change during the iterations, which takes the accounts
    # concerned through the product kernels for one iteration
    uni, batch = make_workload(1, N=1200, K=64, M=520)
    if varied:
        batch = _varied_costs_and_floors(batch)
    ref = gpu_solve(uni, batch, precision=prism.PRISM_BATCHED_BF16, chains=chains)
    res = gpu_solve(uni, batch, precision=prism.PRISM_BATCHED_BF16, chains=chains, fold_products=1)
    assert np.all(res["status"] == prism.PRISM_CERTIFIED), res["status"]
    assert float(np.max(np.abs(res["w"] - ref["w"]))) <= 1e-9
    assert_parity(uni, batch, res, accounts=[0, 255, 519])


@pytest.mark.parametrize("varied", [False, True])
@pytest.mark.parametrize("chains", [1, 4])
def test_persistent_xupdate_matches_one_cta_per_tile(varied, chains):
    # the fused x-update as persistent CTAs claiming tiles from a counter against one CTA per
    # tile: the same arithmetic on every entry and the same per-tile outputs, so the same
    # iterations and weights bit for bit; accounts stop iterating at different iterations, so
    # the tile list of the persistent form shrinks along the way
    uni, batch = make_workload(1, N=1200, K=64, M=520)
    if varied:
        batch = _varied_costs_and_floors(batch)
    one = gpu_solve(uni, batch, precision=prism.PRISM_BATCHED_BF16, chains=chains, xupdate_form=1)
    per = gpu_solve(uni, batch, precision=prism.PRISM_BATCHED_BF16, chains=chains, xupdate_form=0)
    assert np.all(per["status"] == prism.PRISM_CERTIFIED), per["status"]
    assert np.array_equal(per["iters"], one["iters"])
    assert np.array_equal(per["w"], one["w"])
    assert len(set(per["iters"].tolist())) > 1
    assert_parity(uni, batch, per, accounts=[0, 255, 519])
