"""Pins of the oracle-side adjoint (gradients of L = g'w* through the KKT system of Sec. 4.4):
the closed-form budget-only Jacobian, FP64 central finite differences of the oracle's own
solution on seeded directions, and planted mistakes that those checks must catch."""
import numpy as np
import pytest

from oracle import adjoint
from oracle.active_set import AccountProblem, account_problem
from paper_2606_23367_gb300.workloads import make_workload

# small instances with binding bands, a binding cap and tax-lot kinks (sizes shrunk from the
# differentiation workload so that the oracle solves each in milliseconds)
FAMILIES = {
    "bands": dict(N=40, K=5, M=4, S=4, band_hi=0.3, upper=(0.1, 0.2), held=(10, 20)),
    "held_at_w0": dict(N=40, K=5, M=4, S=4, band_hi=0.3, upper=(0.1, 0.2), held=(15, 25), tc=(5e-3, 1e-2)),
    "cap": dict(N=40, K=5, M=4, S=4, band_hi=0.35, upper=(0.1, 0.2), held=(10, 20), tau=0.6),
    "lots_cap": dict(N=40, K=5, M=4, S=4, band_hi=0.35, upper=(0.1, 0.2), held=(10, 20), tau=0.8,
                     lots=True, restrict=0.05),
}


def _problem(prob, mu=None, B=None, d=None, w0=None):
    return AccountProblem(prob.B if B is None else B, prob.f, prob.d if d is None else d,
                          prob.mu if mu is None else mu, prob.sector, prob.S,
                          prob.w0 if w0 is None else w0, prob.lower, prob.upper, prob.tc,
                          prob.band_lo, prob.band_hi, prob.tau, prob.lots)


def _same_active_set(r0, r1):
    return (np.array_equal(r0.fixed, r1.fixed) and np.array_equal(r0.pos, r1.pos)
            and np.array_equal(r0.wband, r1.wband) and r0.wcap == r1.wcap)


def _fd_check(prob, res, g, grads, n_dir, seed, h=1e-6):
    """Central differences of L = g'w* along seeded directions in (mu, B, d, w0).
    Returns (kept, worst relative error, list of (fd, ad))."""
    dmu, dB, dd, dw0 = grads
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_dir):
        vmu = rng.normal(size=prob.n) * 0.02
        vB = rng.normal(size=prob.B.shape) * 0.3
        vd = rng.normal(size=prob.n) * 0.01
        vw0 = rng.normal(size=prob.n) * 0.01 * (prob.w0 > 0)
        ad = float(dmu @ vmu + np.sum(dB * vB) + dd @ vd + dw0 @ vw0)
        rs = []
        for sgn in (1.0, -1.0):
            p = _problem(prob, mu=prob.mu + sgn * h * vmu, B=prob.B + sgn * h * vB,
                         d=prob.d + sgn * h * vd, w0=prob.w0 + sgn * h * vw0)
            rs.append(p.solve())
        if not (_same_active_set(res, rs[0]) and _same_active_set(res, rs[1])):
            continue
        fd = float(g @ (rs[0].w - rs[1].w)) / (2 * h)
        out.append((fd, ad))
    errs = [abs(fd - ad) / max(abs(ad), 1e-3) for fd, ad in out]
    return len(out), (max(errs) if errs else 0.0), out


def test_budget_only_closed_form_jacobian():
    rng = np.random.default_rng(7)
    n, K = 12, 3
    B = rng.normal(0, 0.3, (n, K)); f = rng.uniform(0.01, 0.04, K); d = rng.uniform(0.005, 0.05, n)
    mu = rng.normal(0.05, 0.02, n)
    inf = np.full(n, np.inf)
    prob = AccountProblem(B, f, d, mu, np.zeros(n, np.int64), 1, np.zeros(n), -inf, inf, np.zeros(n),
                          np.array([-np.inf]), np.array([np.inf]))
    res = prob.solve()
    assert res.n_free == n
    g = rng.normal(size=n)
    dmu, dB, dd, dw0 = adjoint.account_gradients(prob, res, g)
    J = adjoint.budget_only_dw_dmu(B, f, d)
    assert np.allclose(dmu, J.T @ g, rtol=1e-9, atol=1e-9)
    # d and B against central differences of the closed form w = 1/2 Sigma^{-1} (mu - nu 1)
    def closed(Bx, dx):
        Sig = Bx @ (f[:, None] * Bx.T) + np.diag(dx)
        Si = np.linalg.inv(Sig); one = np.ones(n)
        nu = (one @ Si @ mu - 2.0) / (one @ Si @ one)
        return 0.5 * Si @ (mu - nu * one)
    h = 1e-6
    for i in (0, 5, 11):
        e = np.zeros(n); e[i] = h
        fd = g @ (closed(B, d + e) - closed(B, d - e)) / (2 * h)
        assert abs(fd - dd[i]) <= 1e-7 * max(1.0, abs(dd[i]))
        for k in range(K):
            E = np.zeros((n, K)); E[i, k] = h
            fd = g @ (closed(B + E, d) - closed(B - E, d)) / (2 * h)
            assert abs(fd - dB[i, k]) <= 1e-7 * max(1.0, abs(dB[i, k]))
    assert np.all(dw0 == 0.0)


@pytest.mark.parametrize("family", sorted(FAMILIES))
def test_adjoint_matches_central_differences(family):
    uni, batch = make_workload(4, **FAMILIES[family])
    kept_total, worst = 0, 0.0
    for a in range(batch.n_accounts):
        prob = account_problem(uni, batch, a)
        res = prob.solve()
        g = np.random.default_rng(100 + a).normal(size=prob.n)
        grads = adjoint.account_gradients(prob, res, g)
        kept, err, _ = _fd_check(prob, res, g, grads, n_dir=5, seed=1000 + a)
        kept_total += kept
        worst = max(worst, err)
    assert kept_total >= 10, f"only {kept_total} of 20 directions kept the active set"
    assert worst <= 1e-6, worst


def test_planted_adjoint_mistakes_are_caught():
    """Two plausible mistakes (dropping the w_i F t term of dL/dB; taking dL/dw0 = g_i for a
    weight held at its kink, i.e. ignoring how the free weights respond) must fail the
    finite-difference check."""
    uni, batch = make_workload(4, **FAMILIES["held_at_w0"])
    caught_B = caught_w0 = False
    for a in range(batch.n_accounts):
        prob = account_problem(uni, batch, a)
        res = prob.solve()
        g = np.random.default_rng(100 + a).normal(size=prob.n)
        dmu, dB, dd, dw0 = adjoint.account_gradients(prob, res, g)
        F = np.nonzero(~res.fixed)[0]
        t = prob.B[F].T @ dmu[F]
        dB_wrong = dB + 2.0 * np.outer(res.w, prob.f * t)
        interior = np.array([res.fixed[i] and 0 < res.pos[i] < prob.nbp[i] - 1 for i in range(prob.n)])
        dw0_wrong = np.where(interior, g, dw0)
        _, err_B, _ = _fd_check(prob, res, g, (dmu, dB_wrong, dd, dw0), n_dir=5, seed=1000 + a)
        _, err_w0, _ = _fd_check(prob, res, g, (dmu, dB, dd, dw0_wrong), n_dir=5, seed=1000 + a)
        caught_B |= err_B > 1e-6
        caught_w0 |= err_w0 > 1e-6
    assert caught_B and caught_w0
