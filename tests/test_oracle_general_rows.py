"""Pins for the oracle's further constraint families of Eq. 1 (Sec. 4.2): general rows
a_lo <= A w <= a_hi (factor exposure bounds B'w in [a, b]; policy halfspaces G w <= h), a
per-account tilt of the expected returns and a benchmark w_b in the risk term.

Each is checked against something other than the oracle itself: exhaustive enumeration of
active sets on tiny accounts, the band path (general rows that restate the sector bands
must give the band solution and multipliers), the budget-only closed form of the benchmark
problem (a dense library solve), and the KKT conditions of Sec. 4.4 evaluated independently.
"""
import numpy as np
import pytest

from oracle import brute, closed_form, kkt
from oracle.active_set import AccountProblem, account_problem
from paper_2606_23367_gb300.workloads import make_workload

INF = np.inf


def _tiny(seed, n=5, k=2, S=2, cap=False):
    rng = np.random.default_rng(3000 + seed)
    B = rng.normal(0.0, 0.3, size=(n, k))
    f = rng.uniform(0.01, 0.04, size=k)
    d = 4.0 * rng.uniform(0.005, 0.05, size=n)
    mu = rng.normal(0.05, 0.03, size=n)
    w0 = rng.dirichlet(np.ones(n))
    lower = np.zeros(n)
    upper = rng.uniform(0.3, 0.5, size=n)
    tc = rng.uniform(0.005, 0.03, size=n)
    sector = np.arange(n) % S
    band_lo = np.zeros(S)
    band_hi = np.full(S, 0.65)
    return rng, (B, f, d, mu, sector, S, w0, lower, upper, tc, band_lo, band_hi), INF


def _diag(P, r):
    return kkt.diagnostics(P.B, P.f, P.d, P.mu, P.sector, P.S, r.w, P.w0, P.lower, P.upper, P.tc,
                           P.band_lo, P.band_hi, P.tau, r.nu, r.lam, r.theta, P.lots,
                           rows=P.A, rows_lo=P.a_lo, rows_hi=P.a_hi, kappa=r.kappa)


@pytest.mark.parametrize("seed,cap", [(0, False), (1, False), (3, True)])
def test_binding_rows_match_brute_force(seed, cap):
    """A factor exposure bound and a policy halfspace, each placed so that it binds."""
    rng, args, tau = _tiny(seed, cap=cap)
    B = args[0]
    free = AccountProblem(*args).solve()
    e = B.T @ free.w
    rows = np.vstack([B.T[0], np.r_[1.0, 1.0, 0.0, 0.0, 0.0]])
    lo = np.array([-INF, -INF])
    # tightened below the free solution's values (halved until the account stays feasible)
    cut = np.array([0.02 * max(1.0, abs(e[0])), 0.05])
    for _ in range(8):
        hi = np.array([e[0], float(free.w[0] + free.w[1])]) - cut
        try:
            AccountProblem(*args, rows=rows, rows_lo=lo, rows_hi=hi).feasible_start()
            break
        except RuntimeError:
            cut = 0.5 * cut
    if cap:
        # a cap just above the least turnover the constraints force, so that it can bind
        start = AccountProblem(*args, rows=rows, rows_lo=lo, rows_hi=hi).feasible_start()
        tau = float(np.abs(start - args[6]).sum()) + rng.uniform(0.01, 0.15)
    P = AccountProblem(*args, tau=tau, rows=rows, rows_lo=lo, rows_hi=hi)
    r = P.solve()
    w_bf, obj_bf = brute.solve_brute(*args, tau=tau, rows=rows, rows_lo=lo, rows_hi=hi)
    assert np.max(np.abs(r.w - w_bf)) <= 1e-10
    assert np.any(r.wgen != 0)                      # the pin exercises a held row
    dg = _diag(P, r)
    assert dg["r_primal"] <= 1e-12 and dg["r_stat"] <= 1e-10 and dg["r_comp"] <= 1e-12


@pytest.mark.parametrize("seed", [0, 1])
def test_two_sided_exposure_band_matches_brute_force(seed):
    """B'w held inside a two-sided band [a, b] around an exposure the free solution misses."""
    rng, args, tau = _tiny(10 + seed, n=4, k=2)
    B = args[0]
    free = AccountProblem(*args).solve()
    e = B.T @ free.w
    lo = e - np.array([-0.03, 0.5])                   # row 0: a above the free exposure
    hi = e + np.array([0.5, INF])
    P = AccountProblem(*args, rows=B.T, rows_lo=lo, rows_hi=hi)
    r = P.solve()
    w_bf, _ = brute.solve_brute(*args, rows=B.T, rows_lo=lo, rows_hi=hi)
    assert np.max(np.abs(r.w - w_bf)) <= 1e-10
    assert r.wgen[0] == -1
    assert r.kappa[0] <= 0.0                          # held at its lower edge


def test_slack_rows_leave_the_solution_unchanged():
    uni, batch = make_workload(1, N=600, K=16, M=1)
    base = account_problem(uni, batch, 0)
    r0 = base.solve()
    rng = np.random.default_rng(5)
    rows = rng.normal(size=(3, base.n))
    P = AccountProblem(base.B, base.f, base.d, base.mu, base.sector, base.S, base.w0, base.lower,
                       base.upper, base.tc, base.band_lo, base.band_hi, base.tau, base.lots,
                       rows=rows, rows_lo=np.full(3, -1e3), rows_hi=np.full(3, 1e3))
    r = P.solve()
    assert np.max(np.abs(r.w - r0.w)) <= 1e-12
    assert np.all(r.kappa == 0.0) and np.all(r.wgen == 0)


def test_rows_restating_the_bands_reproduce_the_band_path():
    """Sector bands moved into general rows: the same solution, kappa equal to lambda."""
    uni, batch = make_workload(1, N=300, K=12, M=3)
    held = 0
    for a in range(batch.n_accounts):
        b0 = account_problem(uni, batch, a)
        # the two largest sectors capped below their free sums, so that their bands bind
        ssum = np.bincount(b0.sector, weights=b0.solve().w, minlength=b0.S)
        band_hi = b0.band_hi.copy()
        top = np.argsort(ssum)[-2:]
        band_hi[top] = 0.8 * ssum[top]
        base = AccountProblem(b0.B, b0.f, b0.d, b0.mu, b0.sector, b0.S, b0.w0, b0.lower, b0.upper,
                              b0.tc, b0.band_lo, band_hi, b0.tau, b0.lots)
        r0 = base.solve()
        inc = np.stack([(base.sector == s).astype(np.float64) for s in range(base.S)])
        P = AccountProblem(base.B, base.f, base.d, base.mu, base.sector, base.S, base.w0, base.lower,
                           base.upper, base.tc, np.full(base.S, -INF), np.full(base.S, INF), base.tau,
                           base.lots, rows=inc, rows_lo=base.band_lo, rows_hi=base.band_hi)
        r = P.solve()
        assert np.max(np.abs(r.w - r0.w)) <= 1e-10
        np.testing.assert_allclose(r.kappa, r0.lam, rtol=1e-7, atol=1e-10)
        held += int(np.count_nonzero(r0.wband))
    assert held > 0                                   # some band binds, so the pin has teeth


@pytest.mark.parametrize("n,k", [(60, 4), (400, 16)])
def test_benchmark_budget_only_closed_form(n, k):
    """min (w - w_b)' Sigma (w - w_b) - mu'w, 1'w = 1: with x = w - w_b it is the budget-only
    problem in x with budget 1 - 1'w_b, whose closed form is a dense library solve."""
    rng = np.random.default_rng(40 + n)
    B = rng.normal(0.0, 0.3, size=(n, k))
    f = rng.uniform(0.01, 0.04, size=k)
    d = rng.uniform(0.005, 0.05, size=n)
    mu = rng.normal(0.05, 0.02, size=n)
    wb = rng.dirichlet(np.ones(n)) * 0.7
    P = AccountProblem(B, f, d, mu, np.zeros(n, np.int64), 1, np.full(n, 1.0 / n), np.full(n, -INF),
                       np.full(n, INF), np.zeros(n), np.array([-INF]), np.array([INF]), w_bench=wb)
    r = P.solve()
    Sigma = B @ np.diag(f) @ B.T + np.diag(d)
    c = 1.0 - wb.sum()
    Si1 = np.linalg.solve(Sigma, np.ones(n))
    Simu = np.linalg.solve(Sigma, mu)
    nu = (Simu.sum() - 2.0 * c) / Si1.sum()
    w_cf = wb + 0.5 * (Simu - nu * Si1)
    assert np.max(np.abs(r.w - w_cf)) <= 1e-11
    # the constant the fold drops: the tracking objective at w equals the folded one plus it
    track = float((r.w - wb) @ Sigma @ (r.w - wb)) - float(mu @ r.w)
    folded = float(r.w @ Sigma @ r.w) - float(P.mu @ r.w) + P.obj_const
    assert abs(track - folded) <= 1e-12 * max(1.0, abs(track))


def test_tilt_is_a_shift_of_mu():
    uni, batch = make_workload(4, N=300, M=1)
    base = account_problem(uni, batch, 0)
    t = np.random.default_rng(9).normal(0.0, 0.01, size=base.n)
    P = AccountProblem(base.B, base.f, base.d, base.mu, base.sector, base.S, base.w0, base.lower,
                       base.upper, base.tc, base.band_lo, base.band_hi, base.tau, base.lots, mu_tilt=t)
    Q = AccountProblem(base.B, base.f, base.d, base.mu + t, base.sector, base.S, base.w0, base.lower,
                       base.upper, base.tc, base.band_lo, base.band_hi, base.tau, base.lots)
    assert np.array_equal(P.solve().w, Q.solve().w)
    w_cf, _ = closed_form.budget_only(base.B, base.f, base.d, base.mu + t)   # an unconstrained check
    assert np.isfinite(w_cf).all()


def test_factor_exposure_bounds_certified_at_workload_size():
    """Two factor exposures bounded on one side each, just past the free solution's, so that
    both bind: KKT certificate of the result."""
    uni, batch = make_workload(1, N=800, K=16, M=2)
    for a in range(batch.n_accounts):
        base = account_problem(uni, batch, a)
        e = base.B.T @ base.solve().w
        lo, hi = np.full(2, -INF), np.full(2, INF)
        hi[0] = e[0] - 0.01
        lo[1] = e[1] + 0.01
        P = AccountProblem(base.B, base.f, base.d, base.mu, base.sector, base.S, base.w0, base.lower,
                           base.upper, base.tc, base.band_lo, base.band_hi, base.tau, base.lots,
                           rows=base.B.T[:2], rows_lo=lo, rows_hi=hi)
        r = P.solve()
        dg = _diag(P, r)
        assert dg["r_primal"] <= 1e-12
        assert dg["r_stat"] <= 1e-10
        assert dg["r_comp"] <= 1e-12
        assert r.wgen[0] == 1 and r.wgen[1] == -1


class _NoRowRatioTest(AccountProblem):
    """A planted mistake: the ratio test ignores the general rows."""

    def _take_step(self, w, F, step, fixed, pos, wband, wcap, wgen=None):
        R, self.R = self.R, 0
        try:
            return super()._take_step(w, F, step, fixed, pos, wband, wcap, wgen)
        finally:
            self.R = R


def test_planted_ratio_test_mistake_is_caught():
    rng, args, tau = _tiny(0)
    B = args[0]
    free = AccountProblem(*args).solve()
    e = B.T @ free.w
    rows = B.T[:1]
    lo, hi = np.array([-INF]), np.array([e[0] - 0.02 * max(1.0, abs(e[0]))])
    w_bf, _ = brute.solve_brute(*args, rows=rows, rows_lo=lo, rows_hi=hi)
    P = _NoRowRatioTest(*args, rows=rows, rows_lo=lo, rows_hi=hi)
    try:
        r = P.solve()
    except RuntimeError:
        return                                        # the broken method does not finish: caught
    caught = np.max(np.abs(r.w - w_bf)) > 1e-8 or _diag(P, r)["r_primal"] > 1e-9
    assert caught
