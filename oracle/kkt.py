"""External diagnostics (Sec. 4.4) and the objective, in FP64.

Residuals computed from public inputs and a returned portfolio w (Sec. 4.4):

    r_budget   = |1'w - 1|
    r_box      = max(||(l - w)_+||_inf, ||(w - u)_+||_inf)
    r_exposure = max(||(b_min - A w)_+||_inf, ||(A w - b_max)_+||_inf)
    r_turnover = (||w - w0||_1 - tau)_+

and, with multipliers (nu for the budget, lambda_s for the sector bands,
theta for the turnover cap), the stationarity and complementarity checks.
Sec. 4.4 states r_stat for smooth constraint functions; the objective here
has the nonsmooth transition cost phi_i and the cap's |w - w0| terms, so
r_stat is read as the subgradient distance

    r_stat = max_i dist( -[(2 Sigma w - mu)_i + nu + lambda_{s(i)}],
                         d phi_i(w_i) + theta d|w_i - w0_i| + N_[l_i,u_i](w_i) )

with the bound multipliers implicit in the normal cone N. A weight within
``kink_tol`` of a kink or bound is taken to sit on it.

    r_comp = max over bands and the cap of |multiplier| * |slack|, plus any
             multiplier of the wrong sign.

General rows a_lo <= A w <= a_hi (Eq. 1's exposure matrix and policy rows), when
given, enter r_exposure, add A' kappa to the stationarity and their kappa to the
complementarity check, like the bands.

Objective (Sec. 9 display, Eq. 1 with Q = 2 Sigma): f(w) = w'Sigma w - mu'w + sum_i phi_i(w_i).
Quality gates (Sec. 5.5): budget <= 1e-4 and bound <= 1e-6 in the paper; the
workloads here hold every residual to 1e-6.
"""
from __future__ import annotations

import numpy as np

from . import pwl

KINK_TOL = 1e-10


def sigma_times(B, f, d, w):
    """Sigma w with Sigma = B diag(f) B' + diag(d), without forming Sigma (O(N K))."""
    return B @ (f * (B.T @ w)) + d * w


def objective(B, f, d, mu, w, w0, tc, lots=None):
    """f(w) = w' Sigma w - mu' w + sum_i phi_i(w_i) (FP64)."""
    quad = float(w @ sigma_times(B, f, d, w))
    lin = float(mu @ w)
    trans = 0.0
    for i in range(w.shape[0]):
        if lots is not None and len(lots[i][0]) > 0:
            trans += pwl.phi_value(w[i], w0[i], tc[i], lots[i][0], lots[i][1])
        else:
            trans += tc[i] * abs(w[i] - w0[i])
    return quad - lin + trans


def _one_sided_slopes(x, lower, upper, w0, c, sizes, kappas, theta, tol):
    """Left/right slopes of phi + theta|.-w0| at x, with -inf/+inf at the box bounds."""
    kinks, slopes = pwl.phi_kinks(w0, c, sizes, kappas)
    # phi part
    j_left = int(np.searchsorted(kinks, x - tol, side="left"))   # first kink >= x - tol
    j_right = int(np.searchsorted(kinks, x + tol, side="right"))  # first kink > x + tol
    left = slopes[j_left]
    right = slopes[j_right]
    # cap part
    if theta != 0.0:
        if abs(x - w0) <= tol:
            left += -theta
            right += theta
        else:
            sgn = 1.0 if x > w0 else -1.0
            left += theta * sgn
            right += theta * sgn
    if x <= lower + tol:
        left = -np.inf
    if x >= upper - tol:
        right = np.inf
    return left, right


def diagnostics(B, f, d, mu, sector, n_sectors, w, w0, lower, upper, tc,
                band_lo, band_hi, tau, nu=None, lam=None, theta=None, lots=None,
                kink_tol=KINK_TOL, rows=None, rows_lo=None, rows_hi=None, kappa=None):
    """All residuals of Sec. 4.4 plus the objective for one account (FP64 dict)."""
    w = np.asarray(w, np.float64)
    out = {}
    out["r_budget"] = abs(float(w.sum()) - 1.0)
    out["r_box"] = float(max(np.max(np.maximum(lower - w, 0.0), initial=0.0),
                             np.max(np.maximum(w - upper, 0.0), initial=0.0)))
    sec_sum = np.bincount(sector, weights=w, minlength=n_sectors)
    out["r_exposure"] = float(max(np.max(np.maximum(band_lo - sec_sum, 0.0), initial=0.0),
                                  np.max(np.maximum(sec_sum - band_hi, 0.0), initial=0.0)))
    if rows is not None:
        A = np.atleast_2d(np.asarray(rows, np.float64))
        av = A @ w
        out["r_exposure"] = float(max(out["r_exposure"],
                                      np.max(np.maximum(np.asarray(rows_lo) - av, 0.0), initial=0.0),
                                      np.max(np.maximum(av - np.asarray(rows_hi), 0.0), initial=0.0)))
    turn = float(np.abs(w - w0).sum())
    out["r_turnover"] = max(turn - tau, 0.0) if np.isfinite(tau) else 0.0
    out["r_primal"] = max(out["r_budget"], out["r_box"], out["r_exposure"], out["r_turnover"])
    out["obj"] = objective(B, f, d, mu, w, w0, tc, lots)
    if nu is None:
        return out
    lam = np.zeros(n_sectors) if lam is None else np.asarray(lam, np.float64)
    theta = 0.0 if theta is None else float(theta)
    g = 2.0 * sigma_times(B, f, d, w) - mu + nu + lam[sector]
    if rows is not None and kappa is not None:
        g = g + A.T @ np.asarray(kappa, np.float64)
    r_stat = 0.0
    for i in range(w.shape[0]):
        sizes, kappas = (lots[i] if lots is not None else ((), ()))
        lft, rgt = _one_sided_slopes(w[i], lower[i], upper[i], w0[i], tc[i], sizes, kappas,
                                     theta, kink_tol)
        x = -g[i]
        r_stat = max(r_stat, lft - x, x - rgt)
    out["r_stat"] = float(r_stat)
    comp = 0.0
    for s in range(n_sectors):
        ls = lam[s]
        if ls > 0:
            comp = max(comp, ls * abs(band_hi[s] - sec_sum[s]))
        elif ls < 0:
            comp = max(comp, -ls * abs(sec_sum[s] - band_lo[s]))
    if theta > 0:
        comp = max(comp, theta * abs(tau - turn) if np.isfinite(tau) else theta)
    elif theta < 0:
        comp = max(comp, -theta)
    if rows is not None and kappa is not None:
        for r, kr in enumerate(np.asarray(kappa, np.float64)):
            if kr > 0:
                comp = max(comp, kr * abs(rows_hi[r] - av[r]) if np.isfinite(rows_hi[r]) else kr)
            elif kr < 0:
                comp = max(comp, -kr * abs(av[r] - rows_lo[r]) if np.isfinite(rows_lo[r]) else -kr)
    out["r_comp"] = float(comp)
    out["r_kkt"] = max(out["r_primal"], out["r_stat"])
    return out
