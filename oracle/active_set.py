"""The FP64 oracle: a primal active-set method for one account (CPU, numpy).

Each account of a book is the convex program of Eq. 1 (Sec. 4.2) as the
workloads instantiate it (objective scaled as in the Sec. 9 display):

    minimise   f(w) = w' Sigma w - mu' w + sum_i phi_i(w_i)
    subject to 1'w = 1,  l <= w <= u,  lo_s <= sum_{i in s} w_i <= hi_s,
               ||w - w0||_1 <= tau,      Sigma = B F B' + D,

and, optionally, the further constraint families of Eq. 1: general linear rows
a_lo <= A w <= a_hi (factor exposure bounds B'w in [a, b] are the rows A = B';
policy halfspaces G w <= h are rows with a_lo = -inf), a per-account tilt t of
the expected returns (mu -> mu + t) and a benchmark w_b, whose tracking risk
(w - w_b)' Sigma (w - w_b) replaces w' Sigma w: it differs from it by the
linear term -2 (Sigma w_b)' w and a constant, so mu -> mu + t + 2 Sigma w_b.

D > 0 makes f strictly convex, so the minimiser is unique, and the strict
feasibility the generator enforces (Slater, Sec. 4.2) makes the KKT
conditions (Sec. 4.4) necessary and sufficient. The oracle computes that
minimiser exactly up to FP64 rounding by a primal active-set method, the
classical algorithm for convex QPs (start feasible, solve the equality
QP on the current working set, step to the first blocking constraint,
drop a constraint whose multiplier has the wrong sign), extended to the
piecewise-linear phi_i by "segment states":

  * phi_i restricted to [l_i, u_i] has breakpoints b_0 = l_i < ... < b_J = u_i
    (its kinks and w0_i) and is linear on each segment;
  * a weight is FIXED at a breakpoint, or FREE in one segment, where its
    cost is linear with that segment's slope and its cap coefficient is the
    sign of the segment relative to w0_i;
  * the working rows are the budget, any band held at an edge and the cap.

The equality QP on the free set F is solved through the Woodbury identity
Sigma_FF^{-1} = D_F^{-1} - D_F^{-1} B_F (F^{-1} + B_F' D_F^{-1} B_F)^{-1} B_F' D_F^{-1}
and a Schur complement over the working rows. At a zero step the
multipliers are checked: a fixed weight must have -(2 Sigma w - mu)_i - nu
- lambda_{s(i)} inside [left slope, right slope] of phi_i + theta|.-w0_i|
(with -inf / +inf at the box bounds); a band at its upper edge needs
lambda_s >= 0, at its lower edge lambda_s <= 0, the cap theta >= 0. The
most violated condition is released (ties: smallest index), and the method
stops when none is violated by more than ``dual_tol``.

This module is test infrastructure, used only by the tests, the smoke check
and the CPU-baseline leg of the benchmark.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import pwl


@dataclasses.dataclass
class OracleResult:
    w: np.ndarray
    nu: float
    lam: np.ndarray      # (S,) band multipliers, 0 for slack bands
    theta: float         # cap multiplier, 0 when the cap is slack
    iters: int
    n_free: int
    # the identified active set at the solution
    fixed: np.ndarray = None   # (n,) bool: weight at a breakpoint
    pos: np.ndarray = None     # (n,) breakpoint index (fixed) or segment index (free)
    wband: np.ndarray = None   # (S,) +1 band held at hi, -1 at lo, 0 not a working row
    wcap: bool = False         # cap a working row
    kappa: np.ndarray = None   # (R,) multipliers of the general rows (0 when slack)
    wgen: np.ndarray = None    # (R,) +1 row held at a_hi, -1 at a_lo, 0 not a working row


class AccountProblem:
    """One account's data in its own (local) asset order."""

    def __init__(self, B, f, d, mu, sector, n_sectors, w0, lower, upper, tc,
                 band_lo, band_hi, tau=np.inf, lots=None, rows=None, rows_lo=None, rows_hi=None,
                 mu_tilt=None, w_bench=None):
        self.B = np.ascontiguousarray(B, np.float64)
        self.f = np.asarray(f, np.float64)
        self.d = np.asarray(d, np.float64)
        self.mu = np.asarray(mu, np.float64)
        # general rows a_lo <= A w <= a_hi (none by default)
        n0 = self.d.shape[0]
        self.A = np.zeros((0, n0)) if rows is None else np.atleast_2d(np.asarray(rows, np.float64))
        self.R = self.A.shape[0]
        self.a_lo = np.full(self.R, -np.inf) if rows_lo is None else np.asarray(rows_lo, np.float64)
        self.a_hi = np.full(self.R, np.inf) if rows_hi is None else np.asarray(rows_hi, np.float64)
        # tilt and benchmark fold into the linear term (the constant is kept for the objective)
        self.obj_const = 0.0
        if mu_tilt is not None:
            self.mu = self.mu + np.asarray(mu_tilt, np.float64)
        if w_bench is not None:
            wb = np.asarray(w_bench, np.float64)
            sb = self.B @ (self.f * (self.B.T @ wb)) + self.d * wb
            self.mu = self.mu + 2.0 * sb
            self.obj_const = float(wb @ sb)
        self.sector = np.asarray(sector, np.int64)
        self.S = int(n_sectors)
        self.w0 = np.asarray(w0, np.float64)
        self.lower = np.asarray(lower, np.float64)
        self.upper = np.asarray(upper, np.float64)
        self.tc = np.asarray(tc, np.float64)
        self.band_lo = np.asarray(band_lo, np.float64)
        self.band_hi = np.asarray(band_hi, np.float64)
        self.tau = float(tau)
        self.lots = lots
        n = self.d.shape[0]
        self.n = n
        pieces = []
        for i in range(n):
            sizes, kappas = lots[i] if lots is not None else ((), ())
            pieces.append(pwl.restricted_pieces(self.lower[i], self.upper[i], self.w0[i],
                                                self.tc[i], sizes, kappas))
        P = max(p[0].shape[0] for p in pieces)
        self.nbp = np.array([p[0].shape[0] for p in pieces], np.int64)
        self.bp = np.full((n, P), np.nan)
        self.sl = np.full((n, max(P - 1, 1)), np.nan)
        self.sg = np.zeros((n, max(P - 1, 1)))   # sign of each segment relative to w0
        for i, (bp, sl) in enumerate(pieces):
            self.bp[i, :bp.shape[0]] = bp
            self.sl[i, :sl.shape[0]] = sl
            for j in range(sl.shape[0]):
                a, b = bp[j], bp[j + 1]
                if np.isfinite(a) and np.isfinite(b):
                    mid = 0.5 * (a + b)
                elif np.isfinite(a):
                    mid = a + 1.0
                elif np.isfinite(b):
                    mid = b - 1.0
                else:
                    mid = self.w0[i] + 1.0
                self.sg[i, j] = 1.0 if mid > self.w0[i] else -1.0

    # ---- Sigma products -------------------------------------------------
    def sigma_w(self, w):
        return self.B @ (self.f * (self.B.T @ w)) + self.d * w

    def solve_sigma_ff(self, F, X):
        """Sigma_FF^{-1} X by the Woodbury identity (FP64)."""
        dinv = 1.0 / self.d[F]
        Y = dinv[:, None] * X
        if self.B.shape[1] == 0:
            return Y
        BF = self.B[F]
        C = np.diag(1.0 / self.f) + BF.T @ (dinv[:, None] * BF)
        L = np.linalg.cholesky(C)
        T = np.linalg.solve(L.T, np.linalg.solve(L, BF.T @ Y))
        return Y - dinv[:, None] * (BF @ T)

    # ---- feasible start -----------------------------------------------
    def feasible_start(self):
        """Greedy least-turnover feasible point: clip to the box, trim sectors above
        their bands, then sell or buy pro rata to room until the budget holds. With
        general rows, the least-turnover point of a linear program instead."""
        if self.R:
            return self._feasible_start_lp()
        w = np.clip(self.w0, self.lower, self.upper)
        S, sec = self.S, self.sector

        def move(mask, amount, up):
            # move ``amount`` (>0) up or down inside ``mask`` pro rata to the room left
            room = (self.upper - w) if up else (w - self.lower)
            room = np.where(mask, room, 0.0)
            inf = np.nonzero(np.isinf(room))[0]
            if inf.size:
                w[inf[0]] += amount if up else -amount
                return amount
            tot = room.sum()
            take = min(amount, tot)
            if take > 0:
                w[:] = np.where(mask, w + (1 if up else -1) * room * (take / tot), w)
            return take

        for s in range(S):
            m = sec == s
            tot = w[m].sum()
            if tot > self.band_hi[s]:
                move(m, tot - self.band_hi[s], up=False)
            elif tot < self.band_lo[s]:
                move(m, self.band_lo[s] - tot, up=True)
        need = 1.0 - w.sum()
        for s in range(S):
            if abs(need) <= 0:
                break
            m = sec == s
            tot = w[m].sum()
            if need > 0:
                room = self.band_hi[s] - tot
                need -= move(m, min(need, room), up=True) if room > 0 else 0.0
            else:
                room = tot - self.band_lo[s]
                need += move(m, min(-need, room), up=False) if room > 0 else 0.0
        w = np.clip(w, self.lower, self.upper)
        if abs(w.sum() - 1.0) > 1e-12:
            raise RuntimeError("greedy start could not meet the budget (infeasible account?)")
        if np.isfinite(self.tau) and np.abs(w - self.w0).sum() > self.tau:
            raise RuntimeError("greedy start violates the turnover cap (infeasible account?)")
        return w

    def _feasible_start_lp(self):
        """min sum_i t_i over (w, t) with t_i >= |w_i - w0_i| and every constraint (a
        library LP solve, HiGHS); the cap is sum_i t_i <= tau. The constraint matrix is
        stored sparse (its identity blocks would take gigabytes dense at n = 10,000)."""
        import scipy.sparse as sp
        from scipy.optimize import linprog
        n, S = self.n, self.S
        c = np.concatenate([np.zeros(n), np.ones(n)])
        I = sp.identity(n, format="csr")
        A_ub = [sp.hstack([I, -I]), sp.hstack([-I, -I])]
        b_ub = [self.w0, -self.w0]
        zn = sp.csr_matrix((1, n))

        def row(vec_w):
            return sp.hstack([sp.csr_matrix(vec_w[None, :]), zn])

        for s in range(S):
            m = (self.sector == s).astype(np.float64)
            if np.isfinite(self.band_hi[s]):
                A_ub.append(row(m)); b_ub.append([self.band_hi[s]])
            if np.isfinite(self.band_lo[s]):
                A_ub.append(row(-m)); b_ub.append([-self.band_lo[s]])
        for r in range(self.R):
            if np.isfinite(self.a_hi[r]):
                A_ub.append(row(self.A[r])); b_ub.append([self.a_hi[r]])
            if np.isfinite(self.a_lo[r]):
                A_ub.append(row(-self.A[r])); b_ub.append([-self.a_lo[r]])
        if np.isfinite(self.tau):
            A_ub.append(sp.hstack([zn, sp.csr_matrix(np.ones((1, n)))])); b_ub.append([self.tau])
        A_eq = sp.hstack([sp.csr_matrix(np.ones((1, n))), zn])
        bounds = [(self.lower[i], self.upper[i]) for i in range(n)] + [(0, None)] * n
        res = linprog(c, A_ub=sp.vstack(A_ub, format="csr"), b_ub=np.concatenate(b_ub), A_eq=A_eq, b_eq=[1.0],
                      bounds=bounds, method="highs")
        if res.status != 0:
            raise RuntimeError("no feasible point (infeasible account?)")
        w = np.clip(res.x[:n], self.lower, self.upper)
        return w

    def _gen_values(self, w):
        return self.A @ w if self.R else np.zeros(0)

    # ---- the method -----------------------------------------------------
    def _classify(self, w):
        """Segment state of each weight: fixed at breakpoint p, or free in segment p."""
        n = self.n
        fixed = np.zeros(n, bool)
        pos = np.zeros(n, np.int64)
        for i in range(n):
            bp = self.bp[i, :self.nbp[i]]
            hit = np.nonzero(bp == w[i])[0]
            if hit.size or self.nbp[i] == 1:
                fixed[i] = True
                pos[i] = hit[0] if hit.size else 0
                w[i] = bp[pos[i]]
            else:
                pos[i] = int(np.searchsorted(bp, w[i])) - 1
        return fixed, pos

    def _rows(self, F, wband, wcap, pos, wgen=None):
        """Working rows restricted to the free set, in order: budget, bands, cap, general rows."""
        rows = [np.ones(F.shape[0])]
        for s in range(self.S):
            if wband[s] != 0:
                rows.append((self.sector[F] == s).astype(np.float64))
        if wcap:
            rows.append(self.sg[F, pos[F]])
        if wgen is not None:
            for r in range(self.R):
                if wgen[r] != 0:
                    rows.append(self.A[r, F])
        return np.asarray(rows)

    def solve(self, dual_tol=1e-12, max_iter=None, w_start=None):
        n, S = self.n, self.S
        w = self.feasible_start() if w_start is None else np.array(w_start, np.float64)
        fixed, pos = self._classify(w)
        wband = np.zeros(S, np.int64)      # +1 held at hi, -1 held at lo, 0 not in W
        wcap = False
        # the same for the general rows: they enter only through the ratio test, which keeps
        # the working rows independent (a blocking row has a nonzero rate along a step that
        # the working rows annihilate)
        wgen = np.zeros(self.R, np.int64)
        if fixed.all():
            # the budget row needs a free weight; free one with room to move
            cand = np.nonzero(self.nbp > 1)[0]
            i = int(cand[0])
            fixed[i] = False
            pos[i] = min(pos[i], self.nbp[i] - 2)
        max_iter = max_iter or (20 * n + 2000)
        lam_full = np.zeros(1)
        it = 0
        # after a full (unblocked) step the point is the minimiser of the equality problem of
        # the working set, so the next iteration goes to the multiplier check: the step a new
        # solve would give is zero up to rounding, which an ill-conditioned working set (more
        # working rows than the free weights can meet independently) can keep above the
        # zero-step threshold
        at_eqp_min = False
        for it in range(1, max_iter + 1):
            F = np.nonzero(~fixed)[0]
            h = self.B.T @ w
            gF = 2.0 * (self.B[F] @ (self.f * h) + self.d[F] * w[F]) - self.mu[F]
            q = gF + self.sl[F, pos[F]]
            E = self._rows(F, wband, wcap, pos, wgen if self.R else None)
            Y = self.solve_sigma_ff(F, np.column_stack([q, E.T]))
            Yq, YE = Y[:, 0], Y[:, 1:]
            lam_full = np.linalg.solve(E @ YE, -(E @ Yq))
            step = -0.5 * (Yq + YE @ lam_full)
            scale = max(1.0, float(np.max(np.abs(w[np.isfinite(w)]), initial=0.0)))
            if not at_eqp_min and np.max(np.abs(step), initial=0.0) > 1e-14 * scale:
                wcap, blocked = self._take_step(w, F, step, fixed, pos, wband, wcap, wgen)
                at_eqp_min = not blocked
                continue
            at_eqp_min = False
            # zero step: check the multipliers
            nu = lam_full[0]
            lam = np.zeros(S)
            k = 1
            for s in range(S):
                if wband[s] != 0:
                    lam[s] = lam_full[k]
                    k += 1
            theta = lam_full[k] if wcap else 0.0
            kappa = np.zeros(self.R)
            k += 1 if wcap else 0
            for rr in range(self.R):
                if wgen[rr] != 0:
                    kappa[rr] = lam_full[k]
                    k += 1
            g = 2.0 * self.sigma_w(w) - self.mu
            r = g + nu + lam[self.sector]
            if self.R:
                r = r + self.A.T @ kappa
            best, what = dual_tol, None
            A = np.nonzero(fixed)[0]
            if A.size:
                p = pos[A]
                has_l = p > 0
                has_r = p < self.nbp[A] - 1
                pl = np.where(has_l, p - 1, 0)
                pr = np.where(has_r, p, 0)
                left = np.where(has_l, self.sl[A, pl] + theta * self.sg[A, pl], -np.inf)
                right = np.where(has_r, self.sl[A, pr] + theta * self.sg[A, pr], np.inf)
                up = -r[A] - right
                dn = left + r[A]
                viol = np.maximum(up, dn)
                k_best = int(np.argmax(viol))          # first maximum: smallest index on ties
                if viol[k_best] > best:
                    best = viol[k_best]
                    what = ("up" if up[k_best] >= dn[k_best] else "dn", int(A[k_best]))
            for s in range(S):
                v = -lam[s] if wband[s] > 0 else (lam[s] if wband[s] < 0 else -np.inf)
                if v > best:
                    best, what = v, ("band", s)
            if wcap and -theta > best:
                best, what = -theta, ("cap", 0)
            for rr in range(self.R):
                v = -kappa[rr] if wgen[rr] > 0 else (kappa[rr] if wgen[rr] < 0 else -np.inf)
                if v > best:
                    best, what = v, ("gen", rr)
            if what is None:
                return OracleResult(w=w, nu=float(nu), lam=lam, theta=float(theta),
                                    iters=it, n_free=int(F.shape[0]), fixed=fixed.copy(),
                                    pos=pos.copy(), wband=wband.copy(), wcap=bool(wcap),
                                    kappa=kappa, wgen=wgen.copy())
            kind, j = what
            if kind == "up":
                fixed[j] = False            # pos stays: segment p lies right of breakpoint p
            elif kind == "dn":
                fixed[j] = False
                pos[j] -= 1
            elif kind == "band":
                wband[j] = 0
            elif kind == "gen":
                wgen[j] = 0
            else:
                wcap = False
        raise RuntimeError(f"active-set method did not finish in {max_iter} iterations")

    def _take_step(self, w, F, step, fixed, pos, wband, wcap, wgen=None):
        """Ratio test: largest alpha <= 1 keeping every free weight in its segment and
        every row outside the working set feasible; the first blocker joins W.
        Returns whether the cap is in the working set afterwards, and whether a blocker
        stopped the step short of the full one."""
        alpha, block = 1.0, None
        a = self.bp[F, pos[F]]
        b = self.bp[F, pos[F] + 1]
        for k, i in enumerate(F):
            dk = step[k]
            if dk > 0 and np.isfinite(b[k]):
                t = max((b[k] - w[i]) / dk, 0.0)
                if t < alpha:
                    alpha, block = t, ("hi", i)
            elif dk < 0 and np.isfinite(a[k]):
                t = max((a[k] - w[i]) / dk, 0.0)
                if t < alpha:
                    alpha, block = t, ("lo", i)
        full = np.zeros(self.n)
        full[F] = step
        sec_w = np.bincount(self.sector, weights=w, minlength=self.S)
        sec_d = np.bincount(self.sector, weights=full, minlength=self.S)
        for s in range(self.S):
            if wband[s] != 0:
                continue
            if sec_d[s] > 0 and np.isfinite(self.band_hi[s]):
                t = max((self.band_hi[s] - sec_w[s]) / sec_d[s], 0.0)
                if t < alpha:
                    alpha, block = t, ("bhi", s)
            elif sec_d[s] < 0 and np.isfinite(self.band_lo[s]):
                t = max((self.band_lo[s] - sec_w[s]) / sec_d[s], 0.0)
                if t < alpha:
                    alpha, block = t, ("blo", s)
        if self.R:
            gv = self.A @ w
            gd = self.A[:, F] @ step
            for r in range(self.R):
                if wgen[r] != 0:
                    continue
                if gd[r] > 0 and np.isfinite(self.a_hi[r]):
                    t = max((self.a_hi[r] - gv[r]) / gd[r], 0.0)
                    if t < alpha:
                        alpha, block = t, ("ghi", r)
                elif gd[r] < 0 and np.isfinite(self.a_lo[r]):
                    t = max((self.a_lo[r] - gv[r]) / gd[r], 0.0)
                    if t < alpha:
                        alpha, block = t, ("glo", r)
        if np.isfinite(self.tau) and not wcap:
            rate = float(self.sg[F, pos[F]] @ step)
            if rate > 0:
                turn = float(np.abs(w - self.w0).sum())
                t = max((self.tau - turn) / rate, 0.0)
                if t < alpha:
                    alpha, block = t, ("cap", 0)
        w[F] = np.clip(w[F] + alpha * step, a, b)
        if block is None:
            return wcap, False
        kind, j = block
        if kind == "hi":
            fixed[j] = True
            pos[j] = pos[j] + 1
            w[j] = self.bp[j, pos[j]]
        elif kind == "lo":
            fixed[j] = True
            w[j] = self.bp[j, pos[j]]
        elif kind == "bhi":
            wband[j] = 1
        elif kind == "blo":
            wband[j] = -1
        elif kind == "ghi":
            wgen[j] = 1
        elif kind == "glo":
            wgen[j] = -1
        else:
            wcap = True
        return wcap, True


def account_problem(uni, batch, a) -> AccountProblem:
    """AccountProblem for account ``a`` of a (Universe, Batch) pair. The batch's optional
    families become the general rows of Eq. 1 (factor-exposure bounds: A = the rows of B'
    with a finite bound), the tilt and the benchmark."""
    idx = batch.account_assets(a, uni.n_assets)
    sl = batch.account_slice(a)
    lots = batch.account_lots(a) if batch.lot_offsets is not None else None
    B = uni.B[idx]
    rows = rows_lo = rows_hi = None
    flo, fhi = getattr(batch, "factor_lo", None), getattr(batch, "factor_hi", None)
    if flo is not None or fhi is not None:
        K = B.shape[1]
        lo = np.full(K, -np.inf) if flo is None else np.asarray(flo[a], np.float64)
        hi = np.full(K, np.inf) if fhi is None else np.asarray(fhi[a], np.float64)
        J = np.flatnonzero(np.isfinite(lo) | np.isfinite(hi))
        if J.size:
            rows, rows_lo, rows_hi = B[:, J].T, lo[J], hi[J]
    tilt = getattr(batch, "mu_tilt", None)
    bench = getattr(batch, "w_bench", None)
    return AccountProblem(B, uni.f, uni.d[idx], uni.mu[idx], uni.sector[idx],
                          uni.n_sectors, batch.w0[sl], batch.lower[sl], batch.upper[sl],
                          batch.tc[sl], batch.band_lo[a], batch.band_hi[a],
                          batch.turnover_cap[a], lots, rows=rows, rows_lo=rows_lo, rows_hi=rows_hi,
                          mu_tilt=None if tilt is None else tilt[sl],
                          w_bench=None if bench is None else bench[sl])


def solve_account(uni, batch, a, **kw) -> OracleResult:
    return account_problem(uni, batch, a).solve(**kw)
