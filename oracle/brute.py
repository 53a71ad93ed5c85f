"""Brute-force enumeration of active sets for tiny accounts (a pin for the oracle).

At the minimiser of a strictly convex program with a piecewise-linear
transition cost, every weight either sits on a breakpoint of phi_i (a kink
or a box bound) or lies strictly inside one linear segment, and every band
and the cap is either slack or held at an edge. Fixing such an assignment
turns the problem into an equality-constrained QP whose solution, when it
satisfies every dropped constraint, is a feasible point; the minimiser is
the feasible candidate of least objective. Enumerating all assignments is
exponential, so this is only used with a handful of assets.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import kkt, pwl


def solve_brute(B, f, d, mu, sector, n_sectors, w0, lower, upper, tc, band_lo, band_hi,
                tau=np.inf, lots=None, tol=1e-11, rows=None, rows_lo=None, rows_hi=None):
    """The minimiser by enumeration; ``rows``: optional general rows rows_lo <= A w <= rows_hi,
    each slack or held at one of its edges."""
    n = d.shape[0]
    Sigma = B @ np.diag(f) @ B.T + np.diag(d)
    pieces = []
    for i in range(n):
        sizes, kappas = lots[i] if lots is not None else ((), ())
        pieces.append(pwl.restricted_pieces(lower[i], upper[i], w0[i], tc[i], sizes, kappas))
    # per-variable options: ('fix', value) or ('free', lo, hi, slope, sign-vs-w0)
    opts = []
    for i in range(n):
        bp, sl = pieces[i]
        o = [("fix", float(b)) for b in bp if np.isfinite(b)]
        for j in range(bp.shape[0] - 1):
            a, b = bp[j], bp[j + 1]
            mid = 0.5 * (a + b) if np.isfinite(a) and np.isfinite(b) else (b - 1 if np.isfinite(b) else a + 1)
            if not (np.isfinite(a) or np.isfinite(b)):
                mid = w0[i] + 1.0
            o.append(("free", a, b, float(sl[j]), 1.0 if mid > w0[i] else -1.0))
        opts.append(o)
    band_states = [(0,) if not (np.isfinite(band_lo[s]) or np.isfinite(band_hi[s])) else (0, -1, 1)
                   for s in range(n_sectors)]
    cap_states = (0, 1) if np.isfinite(tau) else (0,)
    Ag = np.zeros((0, n)) if rows is None else np.atleast_2d(np.asarray(rows, np.float64))
    glo = np.full(Ag.shape[0], -np.inf) if rows_lo is None else np.asarray(rows_lo, np.float64)
    ghi = np.full(Ag.shape[0], np.inf) if rows_hi is None else np.asarray(rows_hi, np.float64)
    gen_states = [tuple([0] + ([-1] if np.isfinite(glo[r]) else []) + ([1] if np.isfinite(ghi[r]) else []))
                  for r in range(Ag.shape[0])]
    best = None
    for assign in itertools.product(*opts):
        F = [i for i in range(n) if assign[i][0] == "free"]
        A = [i for i in range(n) if assign[i][0] == "fix"]
        wA = np.zeros(n)
        for i in A:
            wA[i] = assign[i][1]
        for bst in itertools.product(*band_states):
            for cst, gst in itertools.product(cap_states, itertools.product(*gen_states)):
                rows, rhs = [], []
                r = np.zeros(n); r[F] = 1.0
                rows.append(r); rhs.append(1.0 - wA.sum())
                for s in range(n_sectors):
                    if bst[s] == 0:
                        continue
                    r = np.zeros(n)
                    memb = [i for i in F if sector[i] == s]
                    r[memb] = 1.0
                    edge = band_hi[s] if bst[s] > 0 else band_lo[s]
                    rows.append(r); rhs.append(edge - wA[sector == s].sum())
                if cst:
                    r = np.zeros(n)
                    const = 0.0
                    for i in F:
                        r[i] = assign[i][4]
                        const -= assign[i][4] * w0[i]
                    for i in A:
                        const += abs(wA[i] - w0[i])
                    rows.append(r); rhs.append(tau - const)
                for rg in range(Ag.shape[0]):
                    if gst[rg] == 0:
                        continue
                    r = np.zeros(n); r[F] = Ag[rg, F]
                    edge = ghi[rg] if gst[rg] > 0 else glo[rg]
                    rows.append(r); rhs.append(edge - float(Ag[rg] @ wA))
                E = np.asarray(rows)[:, F] if F else np.zeros((len(rows), 0))
                e = np.asarray(rhs)
                w = wA.copy()
                if F:
                    sF = np.array([assign[i][3] for i in F])
                    g0 = mu[F] - sF - 2.0 * Sigma[np.ix_(F, A)] @ wA[A] if A else mu[F] - sF
                    m = E.shape[0]
                    KKT = np.block([[2.0 * Sigma[np.ix_(F, F)], E.T], [E, np.zeros((m, m))]])
                    rhs_full = np.concatenate([g0, e])
                    sol, *_ = np.linalg.lstsq(KKT, rhs_full, rcond=None)
                    if np.max(np.abs(KKT @ sol - rhs_full)) > 1e-9:
                        continue
                    w[F] = sol[:len(F)]
                    ok = all(assign[i][1] - tol <= w[i] <= assign[i][2] + tol for i in F)
                    if not ok:
                        continue
                else:
                    if np.max(np.abs(e)) > tol:
                        continue
                diag = kkt.diagnostics(B, f, d, mu, sector, n_sectors, w, w0, lower, upper, tc,
                                       band_lo, band_hi, tau, lots=lots,
                                       rows=Ag if Ag.shape[0] else None, rows_lo=glo, rows_hi=ghi)
                if diag["r_primal"] > tol:
                    continue
                if best is None or diag["obj"] < best[0]:
                    best = (diag["obj"], w.copy())
    if best is None:
        raise RuntimeError("no feasible assignment")
    return best[1], best[0]
