"""Exact solution for diagonal risk by breakpoint search (water-filling).

With Sigma = diag(d) (B = 0) the account problem

    min sum_i [ d_i w_i^2 - mu_i w_i + phi_i(w_i) ]
    s.t. 1'w = 1, l <= w <= u, lo_s <= sum_{i in s} w_i <= hi_s

separates once the budget multiplier nu and the band multipliers lambda_s
are fixed: w_i(eta) = argmin_{l<=w<=u} d_i w^2 + (eta - mu_i) w + phi_i(w)
with eta = nu + lambda_{s(i)}. Each w_i(eta) is nonincreasing and piecewise
linear in eta, so the sector sums S_s(eta) are too. A sector whose band is
slack has lambda_s = 0; a sector pushed past a band edge is held on it, so
the budget reads T(nu) = sum_s clamp(S_s(nu), lo_s, hi_s) = 1. Sorting the
breakpoints gives the piece of T (and then of each held sector's S_s) that
holds the root, which is then solved exactly as a linear equation.

This is the textbook breakpoint search for a separable quadratic knapsack
problem. It pins the active-set oracle on diagonal risk, and, because one
prox/projection step of a splitting method is exactly such a problem (with
d_i = rho/2 and mu_i = rho v_i), it is also the exact answer of that step.
"""
from __future__ import annotations

import numpy as np


def _w_of_eta(eta, d, mu, bp, sl):
    """w_i(eta) for one variable: minimiser of d w^2 + (eta - mu) w + phi(w) on [b_0, b_J].

    With t_j = (mu - eta - s_j) / (2 d) the stationary point on segment j
    (t_j decreasing in j because the slopes increase), the minimiser is
    clip(t_0, b_0, b_1) + sum_{j>=1} (clip(t_j, b_j, b_{j+1}) - b_j): the
    segments below the answer contribute their full width, those above nothing.
    """
    J = bp.shape[0] - 1
    if J == 0:
        return bp[0]
    t = (mu - eta - sl) / (2.0 * d)
    w = min(max(t[0], bp[0]), bp[1])
    for j in range(1, J):
        w += min(max(t[j], bp[j]), bp[j + 1]) - bp[j]
    return w


def _eta_breaks(d, mu, bp, sl):
    """Values of eta where w_i(eta) changes slope."""
    J = bp.shape[0] - 1
    out = []
    for j in range(J + 1):
        if j > 0:
            out.append(mu - 2.0 * d * bp[j] - sl[j - 1])
        if j < J:
            out.append(mu - 2.0 * d * bp[j] - sl[j])
    return [e for e in out if np.isfinite(e)]


def _root_pwl(fun, breaks, target):
    """eta with fun(eta) = target for a nonincreasing continuous PWL fun with kinks ``breaks``."""
    br = np.unique(np.asarray(breaks, np.float64))
    if br.size == 0:
        br = np.array([0.0])
    vals = np.array([fun(e) for e in br])
    # extend by one unit step on each side so the root is bracketed on a linear piece
    step = max(1.0, float(np.max(np.abs(br))))
    lo_e, hi_e = br[0] - step, br[-1] + step
    for _ in range(200):
        if fun(lo_e) >= target:
            break
        lo_e -= step
        step *= 2
    else:
        raise RuntimeError("target above the function's range")
    step = max(1.0, float(np.max(np.abs(br))))
    for _ in range(200):
        if fun(hi_e) <= target:
            break
        hi_e += step
        step *= 2
    else:
        raise RuntimeError("target below the function's range")
    xs = np.concatenate([[lo_e], br, [hi_e]])
    ys = np.concatenate([[fun(lo_e)], vals, [fun(hi_e)]])
    # find consecutive xs[k] <= root <= xs[k+1] with ys[k] >= target >= ys[k+1]
    for k in range(xs.shape[0] - 1):
        if ys[k] >= target >= ys[k + 1]:
            if ys[k] == ys[k + 1]:
                return xs[k]
            t = (ys[k] - target) / (ys[k] - ys[k + 1])
            return xs[k] + t * (xs[k + 1] - xs[k])
    raise RuntimeError("root not bracketed")


def solve_diagonal(d, mu, pieces, sector, band_lo, band_hi):
    """Exact minimiser for diagonal risk. ``pieces`` = list of (bp, slope) per variable.

    Returns (w, nu, lam) with lam_s = eta_s - nu for sectors held on a band edge.
    """
    n = d.shape[0]
    S = band_lo.shape[0]
    members = [np.nonzero(sector == s)[0] for s in range(S)]

    def S_s(s, eta):
        return sum(_w_of_eta(eta, d[i], mu[i], *pieces[i]) for i in members[s])

    breaks_s = []
    for s in range(S):
        br = []
        for i in members[s]:
            br.extend(_eta_breaks(d[i], mu[i], *pieces[i]))
        breaks_s.append(br)

    def T(nu):
        return sum(min(max(S_s(s, nu), band_lo[s]), band_hi[s]) for s in range(S))

    # T is PWL with kinks at the S_s kinks and where some S_s crosses a band edge;
    # both kinds of kink go into the sorted list, so T is linear between neighbours.
    all_breaks = sorted(set(b for br in breaks_s for b in br))
    extra = []
    for s in range(S):
        for edge in (band_lo[s], band_hi[s]):
            if np.isfinite(edge) and members[s].size:
                try:
                    extra.append(_root_pwl(lambda e, s=s: S_s(s, e), breaks_s[s], edge))
                except RuntimeError:
                    pass
    nu = _root_pwl(T, all_breaks + extra, 1.0)
    eta = np.full(S, nu)
    for s in range(S):
        if not members[s].size:
            continue
        val = S_s(s, nu)
        if val > band_hi[s]:
            eta[s] = _root_pwl(lambda e, s=s: S_s(s, e), breaks_s[s], band_hi[s])
        elif val < band_lo[s]:
            eta[s] = _root_pwl(lambda e, s=s: S_s(s, e), breaks_s[s], band_lo[s])
    w = np.array([_w_of_eta(eta[sector[i]], d[i], mu[i], *pieces[i]) for i in range(n)])
    return w, nu, eta - nu
