"""Production-queue and constraint-burden harness around prism_solve_batch.

The queue metrics are those of the paper's per-solve record and queue aggregates (Sec. 5.1):
for M accounts with per-account times t_1 .. t_M and a declared window tau, the completion
count C (accounts accepted inside the window), the empirical quantiles t_p50 and t_p99, the
missed-deadline rate rho = (1/M) sum_a 1{t_a > tau}, the total elapsed time T_queue,
the throughput Lambda = M / T_queue (Sec. 8.2) and the audit-record coverage. The capacity
bound of a sequential lane, floor(tau / t), is arithmetic on recorded times (Sec. 6.4).

Timing lanes (Sec. 5.4, Table "Timing lanes") are kept apart: an account's queue time runs
from the dispatch of the queue to the return of the call that carried it (queue lane); the
call's own host wall clock is the full-call lane; the library's CUDA-event time is the
device lane. No number of one lane is compared with another's.

Every solve emits an audit record (Sec. 6, "Auditability"): SHA-256 identities of the
account's inputs (with the universe's) and of its output, the elapsed time, the status and
the run metadata, so that the decision can be reconstructed later. The input identities are
taken when the book is received, before the queue's clock starts; the output identities are
taken inside the queue lane, as each call returns.

The queue runs the book in micro-batches, one library call each, one after another on one
GPU. An account whose call would start after the window closes is not dispatched and gets
status DEADLINE_EXCEEDED (the queue-lane status of Table "Status vocabulary"); an account
whose call returns after the window is counted as missed, whatever its status.
"""
from __future__ import annotations

import dataclasses
import hashlib
import math
import time
from typing import Callable, Dict, List, Optional

import numpy as np

from . import prism

ACCEPTED = (prism.PRISM_CERTIFIED, prism.PRISM_FEASIBLE_NONCERTIFIED)


def status_name(s: int) -> str:
    return prism.STATUS_NAMES[s] if 0 <= s < len(prism.STATUS_NAMES) else str(s)


def _h(*arrays) -> str:
    h = hashlib.sha256()
    for arr in arrays:
        if arr is None:
            h.update(b"none")
        else:
            a = np.ascontiguousarray(arr)
            h.update(str(a.dtype).encode())
            h.update(str(a.shape).encode())
            h.update(a.tobytes())
    return h.hexdigest()


def universe_identity(uni) -> str:
    """SHA-256 over the universe's arrays (B, f, d, mu, sector, sector count)."""
    return _h(uni.B, uni.f, uni.d, uni.mu, uni.sector, np.asarray([uni.n_sectors]))


def account_identity(universe_id: str, batch, a: int) -> str:
    """SHA-256 over one account's inputs (its ragged slice, bands, cap and lots), bound to
    the universe's identity."""
    sl = batch.account_slice(a)
    lots = (None, None, None)
    if batch.lot_offsets is not None:
        lo = batch.lot_offsets[sl.start:sl.stop + 1]
        lots = (lo - lo[0], batch.lot_size[lo[0]:lo[-1]], batch.lot_kappa[lo[0]:lo[-1]])
    aidx = None if batch.asset_idx is None else batch.asset_idx[sl]
    # the further Eq. 1 families, when the book has them (absent ones leave the identity as it was)
    fam = []
    for name, per_entry in (("mu_tilt", True), ("w_bench", True), ("factor_lo", False), ("factor_hi", False)):
        arr = getattr(batch, name, None)
        if arr is not None:
            fam.append(arr[sl] if per_entry else arr[a])
    return _h(np.frombuffer(universe_id.encode(), np.uint8), aidx, batch.w0[sl], batch.lower[sl],
              batch.upper[sl], batch.tc[sl], batch.band_lo[a], batch.band_hi[a],
              np.asarray([batch.turnover_cap[a]]), *lots, *fam)


def output_identity(w: np.ndarray, status: int, diag: np.ndarray) -> str:
    """SHA-256 over an account's returned weights, status and diagnostics."""
    return _h(np.ascontiguousarray(w, np.float64), np.asarray([status], np.int32),
              np.ascontiguousarray(diag, np.float64))


@dataclasses.dataclass
class QueueResult:
    accounts: int
    completed: int                      # C: accepted and returned inside the window
    p50_ms: float                       # queue-lane quantiles of the per-account times
    p99_ms: float
    missed_rate: float                  # rho
    t_queue_s: float                    # dispatch of the queue to the last return
    throughput: float                   # Lambda = M / T_queue, accounts/s
    audit_coverage: float               # fraction of accounts with an audit record
    window_s: float
    micro_batch: int
    calls: int
    call_ms: List[float]                # full-call lane, one entry per call
    device_ms: List[float]              # device lane, one entry per call
    status_counts: Dict[str, int]
    records: List[dict]
    w: Optional[np.ndarray] = None      # the book's weights (ragged), when kept
    status: Optional[np.ndarray] = None


    def capacity_bound(self) -> int:
        """floor(tau / t) accounts for a sequential lane at the recorded p99 (Sec. 6.4)."""
        return int(math.floor(self.window_s / (self.p99_ms / 1e3))) if self.p99_ms > 0 else 0

    def batched_capacity_bound(self) -> int:
        """The same arithmetic for this queue's lane: floor(tau / slowest call) calls of
        micro_batch accounts each."""
        t = max(self.call_ms) / 1e3 if self.call_ms else 0.0
        return int(math.floor(self.window_s / t)) * self.micro_batch if t > 0 else 0

    def summary(self) -> dict:
        d = {k: v for k, v in dataclasses.asdict(self).items() if k not in ("records", "w", "status")}
        d["capacity_bound_sequential"] = self.capacity_bound()
        d["capacity_bound_batched"] = self.batched_capacity_bound()
        return d


def quantile_ms(times_s: np.ndarray, q: float) -> float:
    """Empirical quantile (the smallest recorded time with at least a fraction q of the
    times at or below it), in ms."""
    if times_s.size == 0:
        return 0.0
    t = np.sort(times_s)
    k = max(0, int(math.ceil(q * t.size)) - 1)
    return float(t[k] * 1e3)


def run_queue(uni, batch, solve_fn: Callable, window_s: float = 1500.0, micro_batch: Optional[int] = None,
              meta: Optional[dict] = None, clock: Callable[[], float] = time.perf_counter,
              keep_outputs: bool = False) -> QueueResult:
    """Run the book as a queue of micro-batches through solve_fn(sub_batch, time_budget_s),
    which returns a prism.solve-style dict (w, status, diag, t_call_ms, t_device_ms).
    keep_outputs: also return the book's weights (accounts not dispatched keep NaN)."""
    M = batch.n_accounts
    mb = M if micro_batch is None else max(1, int(micro_batch))
    uid = universe_identity(uni)
    meta = dict(meta or {})
    if "solver_version" not in meta:
        try:
            meta["solver_version"] = prism.prism_version()
        except RuntimeError:                        # the library is not built: a test's fake solver
            meta["solver_version"] = "unknown"
    meta.setdefault("lane", "queue")
    input_ids = [account_identity(uid, batch, a) for a in range(M)]     # at intake
    t_acc = np.full(M, np.inf)
    status = np.full(M, prism.PRISM_DEADLINE_EXCEEDED, np.int32)
    records: List[Optional[dict]] = [None] * M
    call_ms, device_ms = [], []
    w_all = np.full(batch.w0.shape[0], np.nan) if keep_outputs else None
    t0 = clock()
    calls = 0
    for start in range(0, M, mb):
        ids = list(range(start, min(M, start + mb)))
        elapsed = clock() - t0
        if elapsed >= window_s:
            break                                   # the rest are not dispatched
        sub = batch.subset(ids)
        res = solve_fn(sub, window_s - elapsed)
        t_done = clock() - t0
        calls += 1
        call_ms.append(float(res.get("t_call_ms", (t_done - elapsed) * 1e3)))
        device_ms.append(float(res.get("t_device_ms", 0.0)))
        for k, a in enumerate(ids):
            st = int(res["status"][k])
            w = res["w"][sub.account_slice(k)]
            diag = np.asarray(res["diag"][k])
            status[a] = st
            t_acc[a] = t_done
            if keep_outputs:
                w_all[batch.account_slice(a)] = w
            records[a] = {
                "account": a, "input_sha256": input_ids[a],
                "universe_sha256": uid, "output_sha256": output_identity(w, st, diag),
                "status": status_name(st), "queue_time_ms": t_done * 1e3,
                "call_ms": call_ms[-1], "window_s": window_s, **meta,
            }
    t_queue = clock() - t0
    missed = ~(t_acc <= window_s)
    accepted = np.isin(status, ACCEPTED) & ~missed
    finite = t_acc[np.isfinite(t_acc)]
    counts: Dict[str, int] = {}
    for s in status.tolist():
        name = status_name(s)
        counts[name] = counts.get(name, 0) + 1
    return QueueResult(
        accounts=M, completed=int(accepted.sum()), p50_ms=quantile_ms(finite, 0.50),
        p99_ms=quantile_ms(finite, 0.99), missed_rate=float(missed.mean()) if M else 0.0,
        t_queue_s=t_queue, throughput=M / t_queue if t_queue > 0 else 0.0,
        audit_coverage=sum(r is not None for r in records) / M if M else 1.0, window_s=window_s,
        micro_batch=mb, calls=calls, call_ms=call_ms, device_ms=device_ms, status_counts=counts,
        records=[r for r in records if r is not None], w=w_all, status=status if keep_outputs else None)


def library_solver(handle, **opts) -> Callable:
    """solve_fn for run_queue: one prism_solve_batch call with host buffers (full-call lane)
    and the rest of the window as its time budget."""
    def solve(sub, budget_s):
        return prism.solve(handle, sub, time_budget_s=float(budget_s), **opts)
    return solve


# Constraint-burden bundles (Table "burden", E5): rule families added one at a time. B3
# (factor exposure bounds) needs a general exposure matrix, which this library does not
# take; it is listed and skipped.
# factor exposure bounds of the bundles from B3 on: the first four factor exposures B'w of
# every account held to [-0.03, 0.03]
FACTOR_BOUND = (4, 0.03)

BURDEN_BUNDLES = [
    ("B0", "budget, long-only, box", dict(tc=(0.0, 0.0), band_hi=np.inf, excl=(0.0, 0.0), lots=False)),
    ("B1", "+ turnover penalty", dict(band_hi=np.inf, excl=(0.0, 0.0), lots=False)),
    ("B2", "+ sector bands", dict(excl=(0.0, 0.0), lots=False)),
    ("B3", "+ factor exposure bounds", dict(excl=(0.0, 0.0), lots=False, factor_bound=FACTOR_BOUND)),
    ("B4", "+ account exclusions", dict(lots=False, factor_bound=FACTOR_BOUND)),
    ("B5", "+ tax-lot proxy", dict(lots=True, factor_bound=FACTOR_BOUND)),
]


def burden_books(N: int = 2000, K: int = 32, M: int = 64, seed: int = 0):
    """(bundle, rule family, universe, batch or None) for B0..B5 on the differentiation
    workload's shapes (the same universe for every bundle)."""
    from .workloads import make_workload
    out = []
    for name, family, over in BURDEN_BUNDLES:
        if over is None:
            out.append((name, family, None, None))
            continue
        uni, batch = make_workload(4, seed=seed, N=N, K=K, M=M, **over)
        out.append((name, family, uni, batch))
    return out
