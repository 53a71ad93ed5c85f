"""Test-side process pool that runs the FP64 oracle on every account of a seeded workload.

Each worker regenerates the workload from its seed (the generator is deterministic, so
both sides see the same bytes) and compares one account of the library's result with the
oracle: the oracle's minimiser, the objective gap and the oracle checker's residuals of
the library's weights and multipliers. The pool uses the ``spawn`` start method, so it is
safe to create after the GPU has been used, and each worker runs single-threaded BLAS.
"""
from __future__ import annotations

import multiprocessing as mp
import os

_CACHE = {}


def _cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _init():
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"


def _workload(key):
    if key not in _CACHE:
        from paper_2606_23367_gb300.workloads import make_workload
        workload, kw = key[0], dict(key[1])
        _CACHE.clear()
        _CACHE[key] = make_workload(workload, **kw)
    return _CACHE[key]


def _compare(job):
    key, a, w, nu, lam, theta, lib_obj, bound, kappa = job
    import numpy as np
    from oracle import kkt
    from oracle.active_set import account_problem
    uni, batch = _workload(key)
    P = account_problem(uni, batch, a)
    r = P.solve()
    f_star = kkt.objective(P.B, P.f, P.d, P.mu, r.w, P.w0, P.tc, P.lots)
    rows = {}
    if P.R:
        # the factor rows of the oracle's problem are the factors with a finite bound
        J = np.flatnonzero(np.isfinite(batch.factor_lo[a]) | np.isfinite(batch.factor_hi[a]))
        rows = dict(rows=P.A, rows_lo=P.a_lo, rows_hi=P.a_hi, kappa=np.asarray(kappa)[J])
    dg = kkt.diagnostics(P.B, P.f, P.d, P.mu, P.sector, P.S, w, P.w0, P.lower, P.upper, P.tc,
                         P.band_lo, P.band_hi, P.tau, nu, lam, theta, P.lots, **rows)
    return dict(account=a, w_err=float(np.max(np.abs(w - r.w))) if len(w) else 0.0,
                obj_rel=abs(dg["obj"] - f_star) / max(abs(f_star), 1e-4),
                r_primal=float(dg["r_primal"]), r_stat=float(dg["r_stat"]), r_comp=float(dg["r_comp"]),
                obj=float(dg["obj"]), lib_obj=float(lib_obj), bound=float(bound))


def compare_all(workload, res, accounts=None, processes=None, **overrides):
    """Oracle comparison of every account (or the given ones) of ``res``, the library's
    result on ``make_workload(workload, **overrides)``. Returns one dict per account."""
    from paper_2606_23367_gb300.workloads import make_workload
    uni, batch = make_workload(workload, **overrides)
    key = (workload, tuple(sorted(overrides.items())))
    accounts = list(range(batch.n_accounts)) if accounts is None else list(accounts)
    jobs = []
    for a in accounts:
        sl = batch.account_slice(a)
        kap = res["kappa"][a].copy() if res.get("kappa") is not None else None
        jobs.append((key, a, res["w"][sl].copy(), float(res["nu"][a]), res["lambda_band"][a].copy(),
                     float(res["theta"][a]), float(res["diag"][a][6]), float(res["diag"][a][7]), kap))
    n = max(1, min(processes or _cores(), len(jobs)))
    ctx = mp.get_context("spawn")
    with ctx.Pool(n, initializer=_init) as pool:
        return pool.map(_compare, jobs, chunksize=1)


def _adjoint(job):
    key, a, g = job
    from oracle import adjoint
    from oracle.active_set import account_problem
    uni, batch = _workload(key)
    prob = account_problem(uni, batch, a)
    res = prob.solve()
    m, b, d_, w0g = adjoint.account_gradients(prob, res, g)
    return a, m, b, d_, w0g


def adjoint_all(workload, g, accounts=None, processes=None, **overrides):
    """Oracle-side gradients of L = sum_a g_a'w_a (g ragged) in (mu, B, d, w0), summed over
    the given accounts (all by default), each account's share from a pool worker."""
    import numpy as np
    from paper_2606_23367_gb300.workloads import make_workload
    uni, batch = make_workload(workload, **overrides)
    key = (workload, tuple(sorted(overrides.items())))
    accounts = list(range(batch.n_accounts)) if accounts is None else list(accounts)
    jobs = [(key, a, g[batch.account_slice(a)].copy()) for a in accounts]
    n = max(1, min(processes or _cores(), len(jobs)))
    N, K = uni.B.shape
    out = dict(dmu=np.zeros(N), dB=np.zeros((N, K)), dd=np.zeros(N), dw0=np.zeros(int(batch.offsets[-1])))
    with mp.get_context("spawn").Pool(n, initializer=_init) as pool:
        parts = pool.map(_adjoint, jobs, chunksize=1)
    for a, m, b, d_, w0g in sorted(parts, key=lambda t: t[0]):
        idx = batch.account_assets(a, N)
        out["dmu"][idx] += m
        out["dB"][idx] += b
        out["dd"][idx] += d_
        out["dw0"][batch.account_slice(a)] = w0g
    return out
