"""Budget-only closed forms (pins for the oracle).

With only the budget row (no box, no bands, no transition cost) the problem
min w'Sigma w - mu'w s.t. 1'w = 1 has the stationarity condition
2 Sigma w - mu + nu 1 = 0, so w = 1/2 Sigma^{-1}(mu - nu 1) and the budget
fixes nu = (1'Sigma^{-1}mu - 2) / (1'Sigma^{-1}1). With mu = 0 this is the
minimum-variance portfolio Sigma^{-1}1 / (1'Sigma^{-1}1). Computed with a
dense FP64 Sigma and a library linear solve.
"""
from __future__ import annotations

import numpy as np


def dense_sigma(B, f, d):
    return B @ np.diag(f) @ B.T + np.diag(d)


def min_variance(B, f, d):
    S = dense_sigma(B, f, d)
    x = np.linalg.solve(S, np.ones(S.shape[0]))
    return x / x.sum()


def budget_only(B, f, d, mu):
    """(w, nu) of min w'Sigma w - mu'w s.t. 1'w = 1."""
    S = dense_sigma(B, f, d)
    a = np.linalg.solve(S, np.ones(S.shape[0]))
    b = np.linalg.solve(S, mu)
    nu = (b.sum() - 2.0) / a.sum()
    return 0.5 * (b - nu * a), nu
