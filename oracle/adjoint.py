"""Oracle-side adjoint: gradients of L = g'w* with respect to (mu, B, d, w0) for one account.

Test infrastructure (see the package docstring). FP64, numpy.

At the solution w* of the account's problem (Eq. 1 as instantiated in the
package docstring), let F be the free weights (strictly inside a linear piece
of phi_i on [l_i, u_i]), A the fixed ones (at a breakpoint), and E_F the
working rows (budget, bands held at an edge, the cap) restricted to F. The
KKT conditions of Sec. 4.4 on that active set are the linear system

    2 Sigma_FF w_F + E_F' lambda = mu_F - s_F - 2 Sigma_FA w_A
    E_F w_F                      = e - E_A w_A,

s_F the slopes of the free weights' pieces. Where the active set is locally
constant (strict complementarity), the implicit-function theorem gives the
derivatives of w_F from this system; w_A is constant, except that a weight
fixed at an interior breakpoint (a kink of phi_i: w0 itself or a tax-lot
kink at w0 minus a cumulative lot size) moves one-for-one with w0_i. With the
adjoint solve

    [2 Sigma_FF  E_F'] [u    ]   [g_F]
    [E_F         0   ] [kappa] = [0  ],

and h = B'w*, t = B_F' u, the chain rule gives, with u_i = 0 outside F:

    dL/dmu_i = u_i
    dL/dd_i  = -2 u_i w_i
    dL/dB_i  = -2 (u_i F h + w_i F t)                       (row i of B)
    dL/dw0_i = g_i - 2 B_i . (F t) - kappa_budget - kappa_band(s(i))
                                         for i fixed at an interior breakpoint,
               kappa_cap sg_i            otherwise, sg_i the sign of w_i - w0_i
                                         (the cap row's coefficient; 0 at w0),

where kappa_band(s) is taken only when the band of sector s is a working row
(the cap row does not move for a weight that moves with w0, since |w_i - w0_i|
is unchanged). Every product here is a plain dense FP64 solve of the system
above; nothing is blocked or reordered.
"""
from __future__ import annotations

import numpy as np


def account_gradients(prob, res, g):
    """(dmu, dB, dd, dw0) of L = g'w* for one account, in the account's own asset order.

    ``prob`` is the oracle's AccountProblem, ``res`` its OracleResult (with the active
    set), ``g`` the loss gradient dL/dw (length n).
    """
    g = np.asarray(g, np.float64)
    n, S = prob.n, prob.S
    w = res.w
    fixed, pos = res.fixed, res.pos
    F = np.nonzero(~fixed)[0]
    # working rows on F, in the oracle's order: budget, bands, cap
    rows = [np.ones(F.shape[0])]
    band_rows = []
    for s in range(S):
        if res.wband[s] != 0:
            rows.append((prob.sector[F] == s).astype(np.float64))
            band_rows.append(s)
    if res.wcap:
        rows.append(prob.sg[F, pos[F]])
    E = np.asarray(rows)
    m = E.shape[0]
    BF = prob.B[F]
    SigFF = BF @ (prob.f[:, None] * BF.T) + np.diag(prob.d[F])
    KKT = np.zeros((F.shape[0] + m, F.shape[0] + m))
    KKT[:F.shape[0], :F.shape[0]] = 2.0 * SigFF
    KKT[:F.shape[0], F.shape[0]:] = E.T
    KKT[F.shape[0]:, :F.shape[0]] = E
    rhs = np.concatenate([g[F], np.zeros(m)])
    sol = np.linalg.lstsq(KKT, rhs, rcond=None)[0]   # dependent rows get the minimum-norm kappa
    uF, kappa = sol[:F.shape[0]], sol[F.shape[0]:]
    u = np.zeros(n)
    u[F] = uF
    h = prob.B.T @ w
    t = BF.T @ uF
    dmu = u.copy()
    dd = -2.0 * u * w
    dB = -2.0 * (np.outer(u, prob.f * h) + np.outer(w, prob.f * t))
    k_budget = kappa[0]
    k_band = np.zeros(S)
    for k, s in enumerate(band_rows):
        k_band[s] = kappa[1 + k]
    k_cap = kappa[1 + len(band_rows)] if res.wcap else 0.0
    dw0 = np.zeros(n)
    Ft = prob.f * t
    for i in range(n):
        interior = fixed[i] and 0 < pos[i] < prob.nbp[i] - 1
        if interior:
            dw0[i] = g[i] - 2.0 * float(prob.B[i] @ Ft) - k_budget - k_band[prob.sector[i]]
        elif res.wcap:
            if fixed[i]:
                sgn = float(np.sign(w[i] - prob.w0[i]))
            else:
                sgn = float(prob.sg[i, pos[i]])
            dw0[i] = k_cap * sgn
    return dmu, dB, dd, dw0


def budget_only_dw_dmu(B, f, d):
    """Closed form dw*/dmu for the budget-only problem (no bounds, bands, costs):
    w* = 1/2 Sigma^{-1} (mu - nu 1) with nu fixed by 1'w* = 1, so
    dw*/dmu = 1/2 (Sigma^{-1} - Sigma^{-1} 1 1' Sigma^{-1} / (1' Sigma^{-1} 1)). Dense FP64."""
    Sig = B @ (f[:, None] * B.T) + np.diag(d)
    Si = np.linalg.inv(Sig)
    one = np.ones(d.shape[0])
    s1 = Si @ one
    return 0.5 * (Si - np.outer(s1, s1) / float(one @ s1))
