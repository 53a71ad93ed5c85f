"""FP64 CPU oracle for batched account rebalancing (test infrastructure).

This package is test infrastructure, not part of the product: only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it. It shares no code with the CUDA path.

Contents
  pwl          the convex transition cost phi_i (L1 turnover and the tax-lot
               partial minimum), from its definition
  kkt          external diagnostics of Sec. 4.4 (feasibility residuals,
               stationarity and complementarity) and the objective
  closed_form  budget-only minimum-variance solutions (pins)
  waterfill    exact breakpoint search for diagonal risk (pins; also the
               exact answer of one prox/projection step)
  brute        brute-force enumeration of active sets for tiny accounts (pins)
  active_set   the oracle proper: a primal active-set method in FP64 that
               returns the unique minimiser of each account's problem

Problem (Eq. 1, Sec. 4.2, with Q = 2 Sigma, w_b = 0, eta = 1, R = 0, no G rows,
D_a = I, A = sector incidence; objective scaling as in the Sec. 9 display):

    minimise   w' Sigma w - mu' w + sum_i phi_i(w_i)
    subject to 1'w = 1,  l <= w <= u,  lo_s <= sum_{i in s} w_i <= hi_s,
               ||w - w0||_1 <= tau,
    Sigma = B F B' + D.

The active-set oracle also takes, optionally, the further families of Eq. 1: general rows
a_lo <= A w <= a_hi (factor exposure bounds with A = B', policy halfspaces G w <= h), a
per-account tilt of mu and a benchmark w_b in the risk term (pinned in
tests/test_oracle_general_rows.py). The CUDA path does not take them yet.
"""
