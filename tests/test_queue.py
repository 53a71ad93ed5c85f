"""Queue and burden harness logic (host only): the Sec. 5.1 aggregates from per-account
times, deadline handling, audit identities, and the burden bundles' rule families."""
import numpy as np

from paper_2606_23367_gb300 import prism
from paper_2606_23367_gb300.queue import (account_identity, burden_books, output_identity, quantile_ms,
                                          run_queue, universe_identity)
from paper_2606_23367_gb300.workloads import make_workload


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


def fake_solver(clock, call_s, status_of=lambda a: prism.PRISM_CERTIFIED):
    """Each call takes call_s seconds of the fake clock and returns the given statuses."""
    def solve(sub, budget_s):
        clock.t += call_s
        M = sub.n_accounts
        return {"w": sub.w0.copy(), "status": np.array([status_of(k) for k in range(M)], np.int32),
                "diag": np.zeros((M, prism.PRISM_NDIAG)), "t_call_ms": call_s * 1e3, "t_device_ms": 0.0}
    return solve


def test_quantiles_are_order_statistics():
    t = np.arange(1, 101) / 1000.0           # 1 .. 100 ms
    assert quantile_ms(t, 0.50) == 50.0
    assert quantile_ms(t, 0.99) == 99.0
    assert quantile_ms(np.array([0.25]), 0.99) == 250.0


def test_queue_inside_the_window():
    uni, batch = make_workload(0, M=1)
    batch = batch.subset([0] * 40)
    clk = FakeClock()
    r = run_queue(uni, batch, fake_solver(clk, 0.3), window_s=1500.0, micro_batch=10, clock=clk)
    assert r.calls == 4 and r.completed == 40 and r.missed_rate == 0.0
    assert abs(r.t_queue_s - 1.2) < 1e-12 and abs(r.throughput - 40 / 1.2) < 1e-9
    # per-account times: the return of the carrying call (0.3, 0.6, 0.9, 1.2 s, ten each)
    assert r.p50_ms == 600.0 and r.p99_ms == 1200.0
    assert r.audit_coverage == 1.0 and len(r.records) == 40
    assert r.capacity_bound() == int(1500 / 1.2)
    assert r.batched_capacity_bound() == int(1500 / 0.3) * 10


def test_queue_deadline_misses_and_undispatched_accounts():
    uni, batch = make_workload(0, M=1)
    batch = batch.subset([0] * 50)
    clk = FakeClock()
    r = run_queue(uni, batch, fake_solver(clk, 0.3), window_s=1.0, micro_batch=10, clock=clk)
    # calls start at 0, 0.3, 0.6, 0.9 (the fourth returns at 1.2 > 1.0: missed); the fifth
    # would start at 1.2, after the window, so its accounts are never dispatched
    assert r.calls == 4
    assert r.completed == 30
    assert abs(r.missed_rate - 20 / 50) < 1e-12
    assert r.status_counts.get("DEADLINE_EXCEEDED") == 10
    assert r.audit_coverage == 40 / 50


def test_only_accepted_statuses_complete():
    uni, batch = make_workload(0, M=1)
    batch = batch.subset([0] * 10)
    clk = FakeClock()
    st = lambda k: (prism.PRISM_CERTIFIED, prism.PRISM_FEASIBLE_NONCERTIFIED, prism.PRISM_TIMEOUT,
                    prism.PRISM_NO_FEASIBLE_RETURN, prism.PRISM_NUMERICAL_FAILURE)[k % 5]
    r = run_queue(uni, batch, fake_solver(clk, 0.01, st), micro_batch=10, clock=clk)
    assert r.completed == 4 and r.missed_rate == 0.0


def test_audit_identities_bind_inputs_and_outputs():
    uni, batch = make_workload(1, N=300, K=8, M=3)
    uid = universe_identity(uni)
    ids = [account_identity(uid, batch, a) for a in range(3)]
    assert len(set(ids)) == 3
    assert account_identity(uid, batch, 1) == ids[1]
    b2 = batch.subset([0, 1, 2])
    b2.upper[b2.account_slice(1)][5] += 1e-12      # one input changes by one step
    assert account_identity(uid, b2, 1) != ids[1] and account_identity(uid, b2, 0) == ids[0]
    uni2 = make_workload(1, N=300, K=8, M=3)[0]
    uni2.mu[0] += 1e-15
    assert account_identity(universe_identity(uni2), batch, 1) != ids[1]
    w = np.linspace(0, 1, 7)
    h = output_identity(w, 0, np.zeros(prism.PRISM_NDIAG))
    assert h == output_identity(w.copy(), 0, np.zeros(prism.PRISM_NDIAG))
    assert h != output_identity(w, 1, np.zeros(prism.PRISM_NDIAG))
    w2 = w.copy(); w2[3] = np.nextafter(w2[3], 2.0)
    assert h != output_identity(w2, 0, np.zeros(prism.PRISM_NDIAG))


def test_burden_bundles_add_one_rule_family_each():
    books = {name: (uni, b) for name, _, uni, b in burden_books(N=400, K=8, M=6)}
    def per_account(b, f):
        return [f(b, a) for a in range(b.n_accounts)]
    b0, b1, b2, b3, b4, b5 = (books[k][1] for k in ("B0", "B1", "B2", "B3", "B4", "B5"))
    # factor exposure bounds from B3 on, on the first factors only
    for b in (b0, b1, b2):
        assert b.factor_lo is None and b.factor_hi is None
    for b in (b3, b4, b5):
        assert np.all(np.isfinite(b.factor_hi[:, :4])) and np.all(np.isinf(b.factor_hi[:, 4:]))
    assert all(per_account(b3, lambda b, a: np.ptp(b.upper[b.account_slice(a)]) == 0))   # no exclusions yet
    assert np.all(b0.tc == 0) and np.all(np.isinf(b0.band_hi))
    assert all(per_account(b0, lambda b, a: np.ptp(b.upper[b.account_slice(a)]) == 0))   # no exclusions
    assert np.all(b1.tc > 0) and np.all(np.isinf(b1.band_hi))
    assert np.all(b2.band_hi == 0.15)
    assert all(per_account(b2, lambda b, a: np.ptp(b.upper[b.account_slice(a)]) == 0))
    assert any(per_account(b4, lambda b, a: np.any(b.upper[b.account_slice(a)] == 0)))
    assert b4.lot_offsets is None and b5.lot_offsets is not None
    assert np.allclose(np.add.reduceat(b5.lot_size, b5.lot_offsets[:-1][np.diff(b5.lot_offsets) > 0]),
                       b5.w0[np.diff(b5.lot_offsets) > 0])
