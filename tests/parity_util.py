"""Shared helpers for the GPU parity tests: solve through the C-ABI, compare with the oracle."""
import numpy as np

from oracle import kkt
from oracle.active_set import account_problem
from paper_2606_23367_gb300 import prism

W_TOL = 1e-6          # max-abs on weights
OBJ_TOL = 1e-8        # relative objective, guarded by max(|f*|, 1e-4)
KKT_TOL = 1e-6        # primal and stationarity residuals


def gpu_solve(uni, batch, **opts):
    h = prism.create_universe(uni)
    try:
        return prism.solve(h, batch, **opts)
    finally:
        h.close()


def compare_account(uni, batch, res, a, ref=None):
    """Oracle vs library for account a; returns a dict of errors."""
    P = account_problem(uni, batch, a)
    r = P.solve() if ref is None else ref
    sl = batch.account_slice(a)
    w = res["w"][sl]
    f_star = kkt.objective(P.B, P.f, P.d, P.mu, r.w, P.w0, P.tc, P.lots)
    rows = {}
    if P.R:
        # the factor rows of the oracle's problem are the factors with a finite bound
        flo, fhi = batch.factor_lo, batch.factor_hi
        J = np.flatnonzero(np.isfinite(flo[a]) | np.isfinite(fhi[a]))
        rows = dict(rows=P.A, rows_lo=P.a_lo, rows_hi=P.a_hi, kappa=np.asarray(res["kappa"][a])[J])
    dg = kkt.diagnostics(P.B, P.f, P.d, P.mu, P.sector, P.S, w, P.w0, P.lower, P.upper, P.tc,
                         P.band_lo, P.band_hi, P.tau, res["nu"][a], res["lambda_band"][a],
                         res["theta"][a], P.lots, **rows)
    return dict(w_err=float(np.max(np.abs(w - r.w))),
                obj_rel=abs(dg["obj"] - f_star) / max(abs(f_star), 1e-4),
                r_primal=dg["r_primal"], r_stat=dg["r_stat"], r_comp=dg["r_comp"],
                status=int(res["status"][a]), lib_obj=float(res["diag"][a][6]), obj=dg["obj"],
                bound=float(res["diag"][a][prism.PRISM_DIAG_ERR_EST]))


# the oracle's own distance from the exact minimiser (its KKT residuals are ~1e-16, divided
# by the strong-convexity modulus ~1e-2 and a sqrt(N) <= 100 norm change)
ORACLE_ERR = 1e-10


def check_account(e, a=None):
    """The parity bar for one account's comparison dict (see compare_account)."""
    assert e["status"] == prism.PRISM_CERTIFIED, (a, e)
    assert e["w_err"] <= W_TOL, (a, e)
    assert e["obj_rel"] <= OBJ_TOL, (a, e)
    assert e["r_primal"] <= KKT_TOL and e["r_stat"] <= KKT_TOL, (a, e)
    # the library's own FP64 objective agrees with the checker's
    assert abs(e["lib_obj"] - e["obj"]) <= 1e-12 * max(1.0, abs(e["obj"])), (a, e)
    # the error the library states for the result bounds the measured one, and meets the target
    assert e["w_err"] <= e["bound"] + ORACLE_ERR, (a, e)
    assert e["bound"] <= W_TOL, (a, e)


def assert_parity(uni, batch, res, accounts=None):
    accounts = range(batch.n_accounts) if accounts is None else accounts
    worst = []
    for a in accounts:
        e = compare_account(uni, batch, res, a)
        worst.append(e)
        check_account(e, a)
    return worst
