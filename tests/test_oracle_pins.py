"""Pins for the FP64 oracle: closed forms, water-filling, brute force, KKT, invariants.

Each test checks the oracle against something other than itself: the
budget-only closed forms (dense library solve), the exact breakpoint
search for diagonal risk, exhaustive enumeration of active sets on tiny
accounts, and the KKT conditions of Sec. 4.4 evaluated independently.
"""
import numpy as np
import pytest

from oracle import brute, closed_form, kkt, pwl, waterfill
from oracle.active_set import AccountProblem, account_problem
from paper_2606_23367_gb300.workloads import make_workload

INF = np.inf


def _random_factor(rng, n, k):
    B = rng.normal(0.0, 0.3, size=(n, k))
    f = rng.uniform(0.01, 0.04, size=k)
    d = rng.uniform(0.005, 0.05, size=n)
    return B, f, d


def _free_problem(rng, n, k, mu_zero):
    B, f, d = _random_factor(rng, n, k)
    mu = np.zeros(n) if mu_zero else rng.normal(0.05, 0.02, size=n)
    return AccountProblem(B, f, d, mu, np.zeros(n, np.int64), 1, np.full(n, 1.0 / n),
                          np.full(n, -INF), np.full(n, INF), np.zeros(n),
                          np.array([-INF]), np.array([INF]))


@pytest.mark.parametrize("n,k", [(50, 5), (400, 16), (2000, 32)])
def test_min_variance_closed_form(n, k):
    rng = np.random.default_rng(n)
    P = _free_problem(rng, n, k, mu_zero=True)
    r = P.solve()
    w_cf = closed_form.min_variance(P.B, P.f, P.d)
    assert np.max(np.abs(r.w - w_cf)) <= 1e-12


@pytest.mark.parametrize("n,k", [(60, 4), (500, 24)])
def test_budget_only_with_mu_closed_form(n, k):
    rng = np.random.default_rng(7 + n)
    P = _free_problem(rng, n, k, mu_zero=False)
    r = P.solve()
    w_cf, nu_cf = closed_form.budget_only(P.B, P.f, P.d, P.mu)
    assert np.max(np.abs(r.w - w_cf)) <= 1e-12
    assert abs(r.nu - nu_cf) <= 1e-10 * max(1.0, abs(nu_cf))


def _diag_instance(rng, n, S):
    d = rng.uniform(0.005, 0.05, size=n)
    mu = rng.normal(0.05, 0.02, size=n)
    w0 = rng.dirichlet(np.full(n, 0.7))
    upper = rng.uniform(0.03, 0.09, size=n)
    upper[rng.choice(n, size=n // 10, replace=False)] = 0.0      # exclusions
    lower = np.zeros(n)
    tc = rng.uniform(1e-3, 1e-2, size=n)
    sector = rng.integers(0, S, size=n)
    band_lo = np.zeros(S)
    band_hi = np.full(S, 1.3 / S)
    return d, mu, w0, lower, upper, tc, sector, band_lo, band_hi


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_diagonal_waterfilling(seed):
    rng = np.random.default_rng(100 + seed)
    n, S = 80, 4
    d, mu, w0, lower, upper, tc, sector, band_lo, band_hi = _diag_instance(rng, n, S)
    B, f = np.zeros((n, 0)), np.zeros(0)
    P = AccountProblem(B, f, d, mu, sector, S, w0, lower, upper, tc, band_lo, band_hi)
    r = P.solve()
    pieces = [pwl.restricted_pieces(lower[i], upper[i], w0[i], tc[i]) for i in range(n)]
    w_wf, nu_wf, lam_wf = waterfill.solve_diagonal(d, mu, pieces, sector, band_lo, band_hi)
    assert np.max(np.abs(r.w - w_wf)) <= 1e-12
    assert abs(r.nu - nu_wf) <= 1e-10


def test_diagonal_waterfilling_with_lots():
    rng = np.random.default_rng(5)
    n, S = 40, 3
    d, mu, w0, lower, upper, tc, sector, band_lo, band_hi = _diag_instance(rng, n, S)
    lots = []
    for i in range(n):
        L = int(rng.integers(1, 5))
        lots.append((rng.dirichlet(np.ones(L)) * w0[i], rng.uniform(-0.2, 0.2, size=L)))
    P = AccountProblem(np.zeros((n, 0)), np.zeros(0), d, mu, sector, S, w0, lower, upper, tc,
                       band_lo, band_hi, lots=lots)
    r = P.solve()
    pieces = [pwl.restricted_pieces(lower[i], upper[i], w0[i], tc[i], *lots[i]) for i in range(n)]
    w_wf, _, _ = waterfill.solve_diagonal(d, mu, pieces, sector, band_lo, band_hi)
    assert np.max(np.abs(r.w - w_wf)) <= 1e-12


def _tiny(rng, n, k, S, cap, with_lots):
    B, f, d = _random_factor(rng, n, k)
    d = d * 4.0
    mu = rng.normal(0.05, 0.03, size=n)
    w0 = rng.dirichlet(np.ones(n))
    upper = rng.uniform(0.3, 0.5, size=n)
    lower = np.zeros(n)
    tc = rng.uniform(0.005, 0.03, size=n)
    sector = np.arange(n) % S
    band_lo = np.zeros(S)
    band_hi = np.full(S, 0.65)
    tau = rng.uniform(0.3, 0.6) if cap else INF
    lots = None
    if with_lots:
        lots = []
        for i in range(n):
            L = int(rng.integers(1, 4))
            lots.append((rng.dirichlet(np.ones(L)) * w0[i], rng.uniform(-0.08, 0.08, size=L)))
    return B, f, d, mu, sector, S, w0, lower, upper, tc, band_lo, band_hi, tau, lots


@pytest.mark.parametrize("seed,n,cap,with_lots", [
    (0, 5, False, False), (1, 5, False, False), (2, 5, False, False),
    (3, 4, True, False), (4, 4, True, False), (5, 3, True, True), (6, 3, False, True),
])
def test_brute_force_tiny(seed, n, cap, with_lots):
    rng = np.random.default_rng(1000 + seed)
    args = _tiny(rng, n, 2, 2, cap, with_lots)
    B, f, d, mu, sector, S, w0, lower, upper, tc, band_lo, band_hi, tau, lots = args
    if np.isfinite(tau):
        # a cap just above the least turnover the box and bands force, so it can bind
        start = AccountProblem(*args[:12], lots=lots).feasible_start()
        tau = float(np.abs(start - w0).sum()) + rng.uniform(0.01, 0.15)
    r = AccountProblem(*args[:12], tau=tau, lots=lots).solve()
    w_bf, obj_bf = brute.solve_brute(*args[:12], tau=tau, lots=lots)
    assert np.max(np.abs(r.w - w_bf)) <= 1e-10
    obj = kkt.objective(B, f, d, mu, r.w, w0, tc, lots)
    assert abs(obj - obj_bf) <= 1e-12 * max(1.0, abs(obj_bf))


@pytest.mark.parametrize("seed,upper_range,band_hi0,tilt,binding", [
    (21, (0.2, 0.35), 0.4, 0.05, "band"),      # sector 0's band held at its upper edge
    (22, (0.13, 0.16), 1.0, 0.0, "box"),       # four weights held at their upper bounds
])
def test_brute_force_n8_fresh_accounts(seed, upper_range, band_hi0, tilt, binding):
    """Enumeration of every active set at N = 8 (budget, box, two sector bands, transition cost)
    for accounts without holdings: with w0 = 0 = l the cost's kink sits on the lower bound, so
    each weight has three states and the 3^8 x 9 assignments run in seconds."""
    rng = np.random.default_rng(seed)
    n, k, S = 8, 2, 2
    B, f, d = rng.normal(0, 0.3, size=(n, k)), rng.uniform(0.01, 0.04, size=k), rng.uniform(0.005, 0.05, size=n) * 4
    mu = rng.normal(0.05, 0.03, size=n)
    w0, lower = np.zeros(n), np.zeros(n)
    upper = rng.uniform(*upper_range, size=n)
    tc = rng.uniform(0.005, 0.03, size=n)
    sector = np.arange(n) % S
    band_lo, band_hi = np.zeros(S), np.array([band_hi0, 1.0])
    mu[sector == 0] += tilt
    args = (B, f, d, mu, sector, S, w0, lower, upper, tc, band_lo, band_hi)
    r = AccountProblem(*args).solve()
    w_bf, obj_bf = brute.solve_brute(*args)
    assert np.max(np.abs(r.w - w_bf)) <= 1e-10
    obj = kkt.objective(B, f, d, mu, r.w, w0, tc, None)
    assert abs(obj - obj_bf) <= 1e-12 * max(1.0, abs(obj_bf))
    if binding == "band":
        assert abs(w_bf[sector == 0].sum() - band_hi0) <= 1e-12 and r.lam[0] > 0
    else:
        assert int(np.sum(np.abs(w_bf - upper) <= 1e-12)) >= 3


def _diag_of(P, r):
    return kkt.diagnostics(P.B, P.f, P.d, P.mu, P.sector, P.S, r.w, P.w0, P.lower, P.upper,
                           P.tc, P.band_lo, P.band_hi, P.tau, r.nu, r.lam, r.theta, P.lots)


@pytest.mark.parametrize("workload,kw", [
    (0, {}), (1, dict(N=1200, K=64, M=2)), (2, dict(N=900, M=3)),
    (3, dict(N=400, K=12, M=3)), (4, dict(N=500, M=2)),
])
def test_kkt_certificate(workload, kw):
    uni, batch = make_workload(workload, **kw)
    for a in range(batch.n_accounts):
        P = account_problem(uni, batch, a)
        r = P.solve()
        dg = _diag_of(P, r)
        assert dg["r_primal"] <= 1e-12
        assert dg["r_stat"] <= 1e-10
        assert dg["r_comp"] <= 1e-12


def test_asset_permutation_invariance():
    uni, batch = make_workload(1, N=700, K=16, M=1)
    P = account_problem(uni, batch, 0)
    r = P.solve()
    perm = np.random.default_rng(3).permutation(P.n)
    Q = AccountProblem(P.B[perm], P.f, P.d[perm], P.mu[perm], P.sector[perm], P.S, P.w0[perm],
                       P.lower[perm], P.upper[perm], P.tc[perm], P.band_lo, P.band_hi, P.tau)
    rq = Q.solve()
    assert np.max(np.abs(rq.w - r.w[perm])) <= 1e-12


def test_scaling_invariance():
    """Scaling Sigma, mu, c and kappa by alpha > 0 scales f and leaves w* unchanged."""
    uni, batch = make_workload(3, N=300, K=8, M=1)
    P = account_problem(uni, batch, 0)
    r = P.solve()
    alpha = 3.7
    lots = [(s, alpha * k) for s, k in P.lots]
    Q = AccountProblem(P.B * np.sqrt(alpha), P.f, P.d * alpha, P.mu * alpha, P.sector, P.S,
                       P.w0, P.lower, P.upper, P.tc * alpha, P.band_lo, P.band_hi, P.tau, lots)
    rq = Q.solve()
    assert np.max(np.abs(rq.w - r.w)) <= 1e-12


def test_checker_detects_known_violations():
    """The external diagnostics report exactly the planted violation."""
    uni, batch = make_workload(0)
    P = account_problem(uni, batch, 0)
    r = P.solve()
    base = _diag_of(P, r)
    w = r.w.copy()
    j = int(np.argmax(w))
    w[j] += 0.01                                   # budget +0.01, box maybe, band maybe
    dg = kkt.diagnostics(P.B, P.f, P.d, P.mu, P.sector, P.S, w, P.w0, P.lower, P.upper, P.tc,
                         P.band_lo, P.band_hi, P.tau)
    assert abs(dg["r_budget"] - 0.01) <= 1e-15
    assert abs(dg["r_box"] - max(w[j] - P.upper[j], 0.0)) <= 1e-15
    # a wrong budget multiplier shows up in stationarity
    dg2 = kkt.diagnostics(P.B, P.f, P.d, P.mu, P.sector, P.S, r.w, P.w0, P.lower, P.upper, P.tc,
                          P.band_lo, P.band_hi, P.tau, r.nu + 1e-3, r.lam, r.theta)
    assert dg2["r_stat"] >= 1e-3 - 1e-12 or base["r_stat"] > 0
    free = (r.w > 1e-9) & (r.w < P.upper - 1e-9) & (np.abs(r.w - P.w0) > 1e-9)
    if free.any():
        assert dg2["r_stat"] >= 1e-3 - 1e-12


def test_phi_matches_l1_without_lots():
    for x in np.linspace(-0.2, 0.4, 31):
        assert pwl.phi_value(x, 0.1, 0.003) == pytest.approx(0.003 * abs(x - 0.1), abs=1e-18)


def test_phi_kinks_consistent_with_values():
    """Slopes from phi_kinks equal finite differences of phi_value; slopes increase."""
    rng = np.random.default_rng(9)
    for _ in range(20):
        w0 = rng.uniform(0.01, 0.05)
        c = rng.uniform(5e-4, 5e-3)
        L = int(rng.integers(1, 5))
        sizes = rng.dirichlet(np.ones(L)) * w0
        kappas = rng.uniform(-0.2, 0.2, size=L)
        kinks, slopes = pwl.phi_kinks(w0, c, sizes, kappas)
        assert np.all(np.diff(slopes) > -1e-15)
        pts = np.concatenate([[0.0], kinks[(kinks > 0) & (kinks < 0.1)], [0.1]])
        for a, b in zip(pts[:-1], pts[1:]):
            if b - a < 1e-9:
                continue
            x1, x2 = a + 0.25 * (b - a), a + 0.75 * (b - a)
            fd = (pwl.phi_value(x2, w0, c, sizes, kappas) - pwl.phi_value(x1, w0, c, sizes, kappas)) / (x2 - x1)
            mid = 0.5 * (x1 + x2)
            assert fd == pytest.approx(slopes[int(np.searchsorted(kinks, mid))], abs=1e-9)


def test_phi_is_lot_lp_partial_minimum():
    """phi(w) equals the lot LP's optimum, found by enumerating the LP's vertices.

    LP: sell s_j in [0, h_j] of each lot and buy b >= 0 with w = w0 - sum s + b,
    cost c (sum s + b) + sum kappa_j s_j. A vertex has every variable but one
    at a bound; the remaining one is fixed by the equality.
    """
    import itertools
    rng = np.random.default_rng(11)
    for _ in range(10):
        L = int(rng.integers(1, 5))
        w0 = 0.04
        c = float(rng.uniform(5e-4, 5e-3))
        sizes = rng.dirichlet(np.ones(L)) * w0
        kappas = rng.uniform(-0.1, 0.1, size=L)
        for w in np.linspace(0.0, 0.08, 17):
            best = np.inf
            for basic in range(L + 1):                      # index L is b
                others = [j for j in range(L) if j != basic]
                for bits in itertools.product((0, 1), repeat=len(others)):
                    s_ = np.zeros(L)
                    for j, bit in zip(others, bits):
                        s_[j] = sizes[j] * bit
                    if basic == L:
                        b = w - w0 + s_.sum()
                        if b < -1e-15:
                            continue
                    else:
                        b = 0.0
                        val = w0 - w + b - (s_.sum() - s_[basic])
                        if val < -1e-15 or val > sizes[basic] + 1e-15:
                            continue
                        s_[basic] = val
                    best = min(best, c * (s_.sum() + max(b, 0.0)) + kappas @ s_)
            assert pwl.phi_value(w, w0, c, sizes, kappas) == pytest.approx(best, abs=1e-15)


# ---- planted mistakes: each pin above must catch a plausible oracle bug ----

def test_planted_dropped_factor_term_is_caught(monkeypatch):
    """Dropping F^{-1} from the Woodbury capacitance breaks the closed-form pin."""
    rng = np.random.default_rng(50)
    P = _free_problem(rng, 80, 6, mu_zero=True)

    def bad(F, X):
        dinv = 1.0 / P.d[F]
        Y = dinv[:, None] * X
        BF = P.B[F]
        C = BF.T @ (dinv[:, None] * BF)                 # F^{-1} missing
        T = np.linalg.solve(C, BF.T @ Y)
        return Y - dinv[:, None] * (BF @ T)
    monkeypatch.setattr(P, "solve_sigma_ff", bad)
    try:
        r = P.solve()
    except (RuntimeError, np.linalg.LinAlgError):
        return                                           # the bug also shows as a failure
    assert np.max(np.abs(r.w - closed_form.min_variance(P.B, P.f, P.d))) > 1e-6


def test_planted_cap_sign_is_caught():
    """Flipping the cap's segment signs breaks the brute-force pin on a capped account."""
    rng = np.random.default_rng(1003)
    args = _tiny(rng, 4, 2, 2, True, False)
    start = AccountProblem(*args[:12]).feasible_start()
    tau = float(np.abs(start - args[6]).sum()) + 0.02
    w_bf, _ = brute.solve_brute(*args[:12], tau=tau)
    P = AccountProblem(*args[:12], tau=tau)
    P.sg = -P.sg
    try:
        w_bad = P.solve().w
    except (RuntimeError, np.linalg.LinAlgError):
        return
    good = AccountProblem(*args[:12], tau=tau).solve().w
    assert np.max(np.abs(good - w_bf)) <= 1e-10
    assert np.max(np.abs(w_bad - w_bf)) > 1e-8


def test_planted_slope_error_is_caught():
    """Using the right-hand slope on every segment breaks the water-filling pin."""
    rng = np.random.default_rng(100)
    n, S = 80, 4
    d, mu, w0, lower, upper, tc, sector, band_lo, band_hi = _diag_instance(rng, n, S)
    P = AccountProblem(np.zeros((n, 0)), np.zeros(0), d, mu, sector, S, w0, lower, upper, tc,
                       band_lo, band_hi)
    P.sl = np.abs(P.sl)                                  # sells priced like buys
    r = P.solve()
    pieces = [pwl.restricted_pieces(lower[i], upper[i], w0[i], tc[i]) for i in range(n)]
    w_wf, _, _ = waterfill.solve_diagonal(d, mu, pieces, sector, band_lo, band_hi)
    assert np.max(np.abs(r.w - w_wf)) > 1e-6
