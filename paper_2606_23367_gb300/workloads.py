"""Seeded synthetic workloads for batched account rebalancing.

This module only draws instance data. It holds none of the solver's
arithmetic and is shared, unchanged, by the FP64 CPU oracle, the tests and
the benchmark, so both sides of every comparison see the same bytes.

The problem class is Eq. 1 of the paper (Sec. 4.2) restricted to what the
synthetic workloads use: a factor risk model Sigma = B F B' + D shared by a
universe, and per account a budget, box bounds with exclusions (u = 0),
sector exposure bands, an L1 transition cost against the current holdings
w0, optionally convex tax-lot transition penalties, restriction caps
(u <= w0) and a turnover cap ||w - w0||_1 <= tau.

The paper's own instances (S&P 500 prices, its real-calibrated extension
and the E5 queue accounts; Sec. 9 and Sec. 8) are not available; these
seeded draws stand in for them with the shapes the workloads name:

  id  workload                                   N       K   M
  0   single account, plain method               100     10  1
  1   500 accounts on a shared universe          10,000  64  500
  2   ragged accounts on a shared universe       5,000   32  256
  3   tax-aware accounts with a turnover cap     1,924   48  200
  4   accounts for differentiation               2,000   32  128

Every draw uses ``Generator(PCG64(SeedSequence([seed, workload, tag...])))``
so that an account's data do not depend on the batch size or on the draw
order of other accounts.

Layout (the C-ABI ``prism_batch`` layout): per-account vectors are stored
ragged, account a owning entries ``offsets[a]:offsets[a+1]``; when
``asset_idx`` is None every account spans the full universe in universe
order, otherwise ``asset_idx`` gives each entry's universe row.
"""
from __future__ import annotations

import dataclasses
import hashlib
from typing import Optional

import numpy as np

UNIVERSE_TAG = 1_000_000
GRADIENT_TAG = 2_000_000


@dataclasses.dataclass
class Universe:
    """Universe-level data shared by every account (Eq. 1 risk and return inputs)."""

    B: np.ndarray        # (N, K) float64 factor loadings, row-major
    f: np.ndarray        # (K,) float64 factor variances, F = diag(f)
    d: np.ndarray        # (N,) float64 idiosyncratic variances, D = diag(d)
    mu: np.ndarray       # (N,) float64 return input
    sector: np.ndarray   # (N,) int32 sector id in [0, n_sectors)
    n_sectors: int

    @property
    def n_assets(self) -> int:
        return int(self.B.shape[0])

    @property
    def n_factors(self) -> int:
        return int(self.B.shape[1])


@dataclasses.dataclass
class Batch:
    """Per-account data of a book of accounts, ragged (C-ABI ``prism_batch``)."""

    offsets: np.ndarray                  # (M+1,) int64
    asset_idx: Optional[np.ndarray]      # (nnz,) int32 or None = full universe
    w0: np.ndarray                       # (nnz,) current holdings
    lower: np.ndarray                    # (nnz,) box lower bounds
    upper: np.ndarray                    # (nnz,) box upper bounds (0 = excluded)
    tc: np.ndarray                       # (nnz,) L1 transition cost per unit traded
    band_lo: np.ndarray                  # (M, S) sector band lower bounds
    band_hi: np.ndarray                  # (M, S) sector band upper bounds
    turnover_cap: np.ndarray             # (M,) tau, +inf = no cap
    lot_offsets: Optional[np.ndarray] = None   # (nnz+1,) int64 lots of each entry
    lot_size: Optional[np.ndarray] = None      # (n_lots,) lot size in weight units
    lot_kappa: Optional[np.ndarray] = None     # (n_lots,) marginal tax per unit sold
    redraws: Optional[np.ndarray] = None       # (M,) feasibility redraw count
    # further families of Eq. 1 (None = absent)
    mu_tilt: Optional[np.ndarray] = None       # (nnz,) per-account tilt of the return input
    w_bench: Optional[np.ndarray] = None       # (nnz,) benchmark weights of the risk term
    factor_lo: Optional[np.ndarray] = None     # (M, K) lower bounds on B'w (-inf = none)
    factor_hi: Optional[np.ndarray] = None     # (M, K) upper bounds on B'w (+inf = none)

    @property
    def n_accounts(self) -> int:
        return int(self.offsets.shape[0] - 1)

    def account_slice(self, a: int) -> slice:
        return slice(int(self.offsets[a]), int(self.offsets[a + 1]))

    def account_assets(self, a: int, n_universe: int) -> np.ndarray:
        if self.asset_idx is None:
            return np.arange(n_universe, dtype=np.int64)
        return self.asset_idx[self.account_slice(a)].astype(np.int64)

    def account_lots(self, a: int):
        """Per-entry list of (sizes, kappas) for account ``a`` (empty arrays when no lots)."""
        sl = self.account_slice(a)
        n = sl.stop - sl.start
        if self.lot_offsets is None:
            return [(np.zeros(0), np.zeros(0)) for _ in range(n)]
        out = []
        for e in range(sl.start, sl.stop):
            lo, hi = int(self.lot_offsets[e]), int(self.lot_offsets[e + 1])
            out.append((self.lot_size[lo:hi].copy(), self.lot_kappa[lo:hi].copy()))
        return out

    def subset(self, accounts) -> "Batch":
        """A batch holding only the listed accounts (same per-account data)."""
        accounts = [int(a) for a in accounts]
        offs = [0]
        take = []
        for a in accounts:
            sl = self.account_slice(a)
            take.append(np.arange(sl.start, sl.stop))
            offs.append(offs[-1] + sl.stop - sl.start)
        take = np.concatenate(take) if take else np.zeros(0, np.int64)
        lot_offsets = lot_size = lot_kappa = None
        if self.lot_offsets is not None:
            lo_list, sz, kp = [0], [], []
            for e in take:
                l0, l1 = int(self.lot_offsets[e]), int(self.lot_offsets[e + 1])
                sz.append(self.lot_size[l0:l1])
                kp.append(self.lot_kappa[l0:l1])
                lo_list.append(lo_list[-1] + l1 - l0)
            lot_offsets = np.asarray(lo_list, np.int64)
            lot_size = np.concatenate(sz) if sz else np.zeros(0)
            lot_kappa = np.concatenate(kp) if kp else np.zeros(0)
        return Batch(
            offsets=np.asarray(offs, np.int64),
            asset_idx=None if self.asset_idx is None else self.asset_idx[take].copy(),
            w0=self.w0[take].copy(), lower=self.lower[take].copy(),
            upper=self.upper[take].copy(), tc=self.tc[take].copy(),
            band_lo=self.band_lo[accounts].copy(), band_hi=self.band_hi[accounts].copy(),
            turnover_cap=self.turnover_cap[accounts].copy(),
            lot_offsets=lot_offsets, lot_size=lot_size, lot_kappa=lot_kappa,
            redraws=None if self.redraws is None else self.redraws[accounts].copy(),
            mu_tilt=None if self.mu_tilt is None else self.mu_tilt[take].copy(),
            w_bench=None if self.w_bench is None else self.w_bench[take].copy(),
            factor_lo=None if self.factor_lo is None else self.factor_lo[accounts].copy(),
            factor_hi=None if self.factor_hi is None else self.factor_hi[accounts].copy())


# Workload parameters. Distributions shared by every workload: B_ij ~ N(0, 0.3^2),
# f_k ~ U[0.01, 0.04], d_i ~ U[0.005, 0.05], mu_i ~ N(0.05, 0.02^2).
WORKLOADS = {
    0: dict(name="single-account N=100 K=10", N=100, K=10, M=1, S=10, band_hi=0.25,
            upper=(0.05, 0.05), excl=(0.0, 0.0), tc=(1e-3, 1e-3), held=None, dirichlet=1.0,
            lots=False, restrict=0.0, tau=np.inf, ragged=None),
    1: dict(name="batch M=500 N=10000 K=64", N=10_000, K=64, M=500, S=20, band_hi=0.15,
            upper=(0.01, 0.03), excl=(0.0, 0.2), tc=(5e-4, 5e-3), held=(200, 800),
            dirichlet=0.5, lots=False, restrict=0.0, tau=np.inf, ragged=None),
    2: dict(name="ragged M=256 universe 5000 K=32", N=5_000, K=32, M=256, S=20, band_hi=0.15,
            upper=(0.01, 0.03), excl=(0.0, 0.2), tc=(5e-4, 5e-3), held=(200, 800),
            dirichlet=0.5, lots=False, restrict=0.0, tau=np.inf, ragged=(100, 5000)),
    3: dict(name="tax-aware M=200 N=1924 K=48", N=1_924, K=48, M=200, S=20, band_hi=0.15,
            upper=(0.01, 0.03), excl=(0.0, 0.0), tc=(5e-4, 5e-3), held=(200, 800),
            dirichlet=0.5, lots=True, restrict=0.05, tau=0.2, ragged=None),
    4: dict(name="differentiation M=128 N=2000 K=32", N=2_000, K=32, M=128, S=20,
            band_hi=0.15, upper=(0.01, 0.03), excl=(0.0, 0.2), tc=(5e-4, 5e-3),
            held=(200, 800), dirichlet=0.5, lots=False, restrict=0.0, tau=np.inf, ragged=None),
}

MAX_REDRAWS = 200


def _rng(*tags) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(t) for t in tags])))


def make_universe(seed: int, workload: int, N: int, K: int, S: int) -> Universe:
    r = _rng(seed, workload, UNIVERSE_TAG)
    B = r.normal(0.0, 0.3, size=(N, K))
    f = r.uniform(0.01, 0.04, size=K)
    d = r.uniform(0.005, 0.05, size=N)
    mu = r.normal(0.05, 0.02, size=N)
    sector = r.integers(0, S, size=N).astype(np.int32)
    return Universe(B=np.ascontiguousarray(B), f=f, d=d, mu=mu, sector=sector, n_sectors=S)


def capacity(upper: np.ndarray, sector: np.ndarray, band_hi: np.ndarray) -> float:
    """sum_s min(hi_s, sum_{i in s} u_i): the largest budget the box and bands admit (lo = 0)."""
    per = np.bincount(sector, weights=upper, minlength=band_hi.shape[0])
    return float(np.minimum(per, band_hi).sum())


def min_turnover(w0, upper, sector, band_hi) -> float:
    """Least ||w - w0||_1 over the box and bands when sum(w0) = 1 and capacity is spare.

    Every unit that must leave a name (above its cap) or a sector (above its band)
    has to be bought back elsewhere, so the trade is twice the forced sale.
    """
    forced_names = np.maximum(w0 - upper, 0.0).sum()
    kept = np.minimum(w0, upper)
    per = np.bincount(sector, weights=kept, minlength=band_hi.shape[0])
    forced_sectors = np.maximum(per - band_hi, 0.0).sum()
    return float(2.0 * (forced_names + forced_sectors))


def _draw_account(p, seed, workload, a, redraw, n_universe, sector_u, S):
    """One account's data; returns a dict of per-entry arrays (local order)."""
    r = _rng(seed, workload, a, redraw)
    if p["ragged"] is not None:
        lo_n, hi_n = p["ragged"]
        n_a = int(np.rint(np.exp(r.uniform(np.log(lo_n), np.log(hi_n)))))
        n_a = min(max(n_a, lo_n), n_universe)
        idx = np.sort(r.choice(n_universe, size=n_a, replace=False)).astype(np.int32)
    else:
        n_a = n_universe
        idx = None
    sec = sector_u if idx is None else sector_u[idx]
    # current holdings w0
    if p["held"] is None:
        w0 = r.dirichlet(np.full(n_a, p["dirichlet"]))
    else:
        n_held = int(r.integers(p["held"][0], p["held"][1] + 1))
        n_held = min(n_held, n_a)
        held = r.choice(n_a, size=n_held, replace=False)
        w0 = np.zeros(n_a)
        w0[held] = r.dirichlet(np.full(n_held, p["dirichlet"]))
    # box and exclusions
    u_a = r.uniform(*p["upper"]) if p["upper"][0] != p["upper"][1] else p["upper"][0]
    upper = np.full(n_a, u_a)
    e_a = r.uniform(*p["excl"]) if p["excl"][1] > 0 else 0.0
    n_ex = int(np.rint(e_a * n_a))
    if n_ex > 0:
        upper[r.choice(n_a, size=n_ex, replace=False)] = 0.0
    lower = np.zeros(n_a)
    c_a = r.uniform(*p["tc"]) if p["tc"][0] != p["tc"][1] else p["tc"][0]
    tc = np.full(n_a, c_a)
    # tax lots (convex lot model: sizes split w0, kappa = marginal tax per unit sold)
    lots = None
    if p["lots"]:
        alpha, beta = r.uniform(0.0, 0.4), r.uniform(0.0, 0.4)
        lots = []
        for i in range(n_a):
            if w0[i] <= 0.0:
                lots.append((np.zeros(0), np.zeros(0)))
                continue
            n_l = int(r.integers(1, 5))
            sizes = r.dirichlet(np.ones(n_l)) * w0[i] if n_l > 1 else np.array([w0[i]])
            basis_ratio = r.uniform(0.5, 1.5, size=n_l)
            gain = 1.0 - basis_ratio
            kappa = np.where(gain >= 0.0, alpha * gain, beta * gain)
            lots.append((sizes, kappa))
    # restriction caps: w <= w0 on a fraction of names
    if p["restrict"] > 0:
        n_r = int(np.rint(p["restrict"] * n_a))
        if n_r > 0:
            pick = r.choice(n_a, size=n_r, replace=False)
            upper[pick] = np.minimum(upper[pick], w0[pick])
    band_lo = np.zeros(S)
    band_hi = np.full(S, p["band_hi"])
    # further Eq. 1 families, drawn after everything else so that the other draws do not move
    tilt = r.normal(0.0, p["tilt"], size=n_a) if p.get("tilt", 0.0) > 0 else None
    bench = None
    if p.get("bench", False):
        # a benchmark spread over the eligible names (Dirichlet(5): close to equal weights)
        elig = np.flatnonzero(upper > 0)
        bench = np.zeros(n_a)
        bench[elig] = r.dirichlet(np.full(elig.shape[0], 5.0))
    return dict(idx=idx, sec=sec, w0=w0, lower=lower, upper=upper, tc=tc, lots=lots,
                band_lo=band_lo, band_hi=band_hi, tau=p["tau"], tilt=tilt, bench=bench)


def _feasible(acc, S) -> bool:
    """Strict feasibility test for lo = 0 bands (Slater, Sec. 4.2)."""
    if capacity(acc["upper"], acc["sec"], acc["band_hi"]) <= 1.05:
        return False
    if np.isfinite(acc["tau"]):
        if min_turnover(acc["w0"], acc["upper"], acc["sec"], acc["band_hi"]) > 0.9 * acc["tau"]:
            return False
    return True


def make_workload(workload: int, seed: int = 0, first_account: int = 0, **overrides):
    """Build (universe, batch) for a workload id; ``overrides`` replace sizes (N, K, M, ...).

    Accounts are drawn with ids first_account .. first_account + M - 1, so disjoint
    shards of one large book can be generated independently.
    """
    p = dict(WORKLOADS[workload])
    p.update(overrides)
    N, K, M, S = int(p["N"]), int(p["K"]), int(p["M"]), int(p["S"])
    if p["ragged"] is not None:
        p["ragged"] = (min(p["ragged"][0], N), min(p["ragged"][1], N))
    uni = make_universe(seed, workload, N, K, S)
    accs, redraws = [], []
    for a in range(first_account, first_account + M):
        for r_ in range(MAX_REDRAWS):
            acc = _draw_account(p, seed, workload, a, r_, N, uni.sector, S)
            if _feasible(acc, S):
                break
        else:
            raise RuntimeError(f"account {a}: no strictly feasible draw in {MAX_REDRAWS} tries")
        accs.append(acc)
        redraws.append(r_)
    offsets = np.zeros(M + 1, np.int64)
    offsets[1:] = np.cumsum([acc["w0"].shape[0] for acc in accs])
    cat = lambda k: np.concatenate([acc[k] for acc in accs]).astype(np.float64)
    asset_idx = None
    if p["ragged"] is not None:
        asset_idx = np.concatenate([acc["idx"] for acc in accs]).astype(np.int32)
    lot_offsets = lot_size = lot_kappa = None
    if p["lots"]:
        lo_list, sz, kp = [0], [], []
        for acc in accs:
            for sizes, kappa in acc["lots"]:
                sz.append(sizes)
                kp.append(kappa)
                lo_list.append(lo_list[-1] + sizes.shape[0])
        lot_offsets = np.asarray(lo_list, np.int64)
        lot_size = np.concatenate(sz).astype(np.float64)
        lot_kappa = np.concatenate(kp).astype(np.float64)
    factor_lo = factor_hi = None
    if p.get("factor_bound") is not None:
        # the first n_rows factor exposures B'w of every account held to [-width, width]
        n_rows, width = p["factor_bound"]
        factor_lo = np.full((M, K), -np.inf)
        factor_hi = np.full((M, K), np.inf)
        factor_lo[:, :n_rows] = -width
        factor_hi[:, :n_rows] = width
    batch = Batch(
        offsets=offsets, asset_idx=asset_idx, w0=cat("w0"), lower=cat("lower"),
        upper=cat("upper"), tc=cat("tc"),
        band_lo=np.stack([acc["band_lo"] for acc in accs]),
        band_hi=np.stack([acc["band_hi"] for acc in accs]),
        turnover_cap=np.asarray([acc["tau"] for acc in accs], np.float64),
        lot_offsets=lot_offsets, lot_size=lot_size, lot_kappa=lot_kappa,
        redraws=np.asarray(redraws, np.int32),
        mu_tilt=cat("tilt") if accs and accs[0]["tilt"] is not None else None,
        w_bench=cat("bench") if accs and accs[0]["bench"] is not None else None,
        factor_lo=factor_lo, factor_hi=factor_hi)
    return uni, batch


def loss_weights(workload: int, batch: Batch, seed: int = 0) -> np.ndarray:
    """Seeded Gaussian weights g (ragged) of the loss L = sum_a g_a' w_a."""
    r = _rng(seed, workload, GRADIENT_TAG)
    return r.normal(0.0, 1.0, size=batch.w0.shape[0])


def instance_hash(uni: Universe, batch: Batch) -> str:
    """SHA-256 over every array of the instance, in a fixed order."""
    h = hashlib.sha256()
    for arr in (uni.B, uni.f, uni.d, uni.mu, uni.sector, batch.offsets,
                batch.asset_idx, batch.w0, batch.lower, batch.upper, batch.tc,
                batch.band_lo, batch.band_hi, batch.turnover_cap,
                batch.lot_offsets, batch.lot_size, batch.lot_kappa):
        if arr is None:
            h.update(b"none")
        else:
            h.update(np.ascontiguousarray(arr).tobytes())
    # the optional Eq. 1 families, only when present (the hashes of books without them stay)
    for arr in (batch.mu_tilt, batch.w_bench, batch.factor_lo, batch.factor_hi):
        if arr is not None:
            h.update(np.ascontiguousarray(arr).tobytes())
    return h.hexdigest()
