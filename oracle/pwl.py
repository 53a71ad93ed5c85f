"""Convex piecewise-linear transition cost phi_i (Eq. 1 terms C and T_tax).

Eq. 1 (Sec. 4.2) charges a transaction-cost term C(dw) and a tax-aware
transition term T_tax(dw; D_a). The workloads use

  * an L1 cost c_i |w - w0_i| (Sec. 9 display, gamma ||w - w0||_1), and
  * for tax-aware accounts a convex lot model. The paper leaves discrete lot
    logic out of its benchmark (Sec. 4.2 scope notes, Sec. 9); the convex
    reading used here is the partial minimum of the lot LP: selling S units
    cheapest-first costs K(S) = sum of kappa over the units sold, every unit
    traded costs c, and the sale may exceed the net reduction (sell and buy
    back) when that lowers the total. With G(S) = 2 c S + K(S) and
    S* = total size of lots whose 2c + kappa < 0,

        phi(w) = c (w - w0) + G(max(S*, w0 - w)),      w >= 0.

    It is convex and piecewise linear, equals c|w - w0| without lots, and
    equals "cost of selling cheapest lots first plus c|dw|" when every lot
    has 2c + kappa >= 0.

The oracle works with phi restricted to [l, u]: breakpoints l = b_0 < ... <
b_J = u (the kinks of phi inside (l, u), plus w0 itself so that the turnover
cap's kink is a breakpoint) and the slope of phi on each segment.
"""
from __future__ import annotations

import numpy as np


def _sorted_lots(sizes, kappas):
    sizes = np.asarray(sizes, np.float64)
    kappas = np.asarray(kappas, np.float64)
    order = np.argsort(kappas, kind="stable")  # cheapest first; ties: smallest lot index
    return sizes[order], kappas[order]


def phi_value(x, w0, c, sizes=(), kappas=()):
    """phi(x) from its definition: c (x - w0) + min over S >= max(0, w0 - x) of G(S)."""
    x = float(x)
    if len(sizes) == 0:
        return c * abs(x - w0)
    h, k = _sorted_lots(sizes, kappas)
    H = np.concatenate([[0.0], np.cumsum(h)])

    def G(S):
        # selling S cheapest-first; beyond the held amount the last lot's rate continues
        val = 2.0 * c * S
        rem = S
        for j in range(h.shape[0]):
            take = min(rem, h[j]) if j < h.shape[0] - 1 else rem
            val += k[j] * take
            rem -= take
            if rem <= 0:
                break
        return val

    s_star = float(np.sum(h[(2.0 * c + k) < 0.0]))
    return c * (x - w0) + G(max(s_star, w0 - x))


def phi_kinks(w0, c, sizes=(), kappas=()):
    """Kinks x_1 < ... < x_m of phi over the real line and slopes s_0 < ... < s_m.

    s_0 is the slope left of x_1, s_m the slope right of x_m.
    """
    if len(sizes) == 0:
        return np.array([w0], np.float64), np.array([-c, c], np.float64)
    h, k = _sorted_lots(sizes, kappas)
    L = h.shape[0]
    marg = 2.0 * c + k
    jstar = int(np.sum(marg < 0.0))   # lots worth selling even without a net sale
    H = np.cumsum(h)
    if jstar == L:
        # every lot is harvested: phi is linear with slope c over w >= 0
        return np.zeros(0), np.array([c], np.float64)
    s_star = H[jstar - 1] if jstar > 0 else 0.0
    kinks = [w0 - s_star]
    slopes_left_to_right = [c]
    # going left from w0 - S*, the next unit sold comes from lot jstar, then jstar+1, ...
    for j in range(jstar, L):
        slopes_left_to_right.insert(0, -c - k[j])
        if j < L - 1:
            kinks.insert(0, w0 - H[j])
    return np.asarray(kinks, np.float64), np.asarray(slopes_left_to_right, np.float64)


def restricted_pieces(lower, upper, w0, c, sizes=(), kappas=(), merge_tol=0.0):
    """Breakpoints b_0 = l < ... < b_J = u of phi on [l, u] and the slope of each segment.

    w0 is always a breakpoint when it lies strictly inside (l, u) (the turnover
    cap's kink). Kinks within ``merge_tol`` of another breakpoint are merged.
    Returns (bp, slope); when l == u, bp = [l] and slope is empty.
    """
    if upper < lower:
        raise ValueError("upper < lower")
    if upper == lower:
        return np.array([lower], np.float64), np.zeros(0)
    kinks, slopes = phi_kinks(w0, c, sizes, kappas)
    inner = [x for x in kinks if lower < x < upper]
    if lower < w0 < upper and not any(x == w0 for x in inner):
        inner.append(w0)
    inner = sorted(inner)
    pts = [lower]
    for x in inner:
        if x - pts[-1] > merge_tol:
            pts.append(x)
    if upper - pts[-1] <= merge_tol and len(pts) > 1:
        pts[-1] = upper
    else:
        pts.append(upper)
    bp = np.asarray(pts, np.float64)
    slope = np.empty(bp.shape[0] - 1)
    for j in range(bp.shape[0] - 1):
        a, b = bp[j], bp[j + 1]
        if np.isinf(a) and np.isinf(b):
            mid = w0
        elif np.isinf(a):
            mid = b - 1.0
        elif np.isinf(b):
            mid = a + 1.0
        else:
            mid = 0.5 * (a + b)
        slope[j] = slopes[int(np.searchsorted(kinks, mid))]
    return bp, slope
