#!/usr/bin/env python
"""Benchmark: certified accounts/s on 500 accounts x 10,000 assets (K = 64).

One step = one prism_solve_batch call over a book of 500 accounts (input
packing, ADMM iterations, FP64 polish and certification, output unpacking).
Only accounts returned with status CERTIFIED (KKT and feasibility <= 1e-6)
count. Under torchrun each rank solves its own disjoint book of 500 accounts
(weak scaling, no data-path collective).

  value  device-resident lane: inputs already in HBM, CUDA events on the solve stream
  e2e    the same call with pinned host inputs/outputs (copies inside the timed region)

--impl reference times the FP64 CPU oracle on the host cores instead (a
bounded sample of accounts per step), on the same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "accounts/s at KKT res<=1e-6, 500 accts x 10k assets; batched-BF16 vs plain FP32"
WORKLOAD = "500 accounts x 10,000 assets, K=64, 20 sector bands, L1 turnover (seeded synthetic)"
M_ACCOUNTS = 500
WORKLOADS_DESC = {
    0: "1 account x 100 assets, K=10, 10 sector bands (seeded synthetic)",
    2: "256 ragged accounts from 5,000 assets (100-5,000 names), K=32 (seeded synthetic)",
    3: "200 accounts x 1,924 assets, K=48, tax lots, turnover cap 0.2 (seeded synthetic)",
    4: "128 accounts x 2,000 assets, K=32 (seeded synthetic)",
}

# Algorithmic bytes per account-entry and iteration of the method: read z and y, write z and
# y (16 B, FP32), read the per-entry constants w0 and u (8 B; l and c are per-account constants
# in this book). Intermediates of this design (v, the split X, the candidate records) are
# overhead, not method bytes.
METHOD_BYTES = 24
# per account-entry moved by one launch of each kernel class, by the same rule
#   gemm_P : read X (its BF16 hi+lo split: 4 B) -- the operand of the product
#   gemm_x : read z, y (8 B), write v (4 B)
#   prox   : read v, z, y and w0, l, u, c (28 B); write z, y and X (12 B)
#   xprox  : the x-update fused with the streaming pass of the prox: the method's 24 B (read z,
#            y, w0, u; write z, y); v (4 B) and the split X (4 B) are reported as overhead
#   block  : the per-account kernel (every iteration of an account in one block): the method's 24 B
ALG_BYTES = {"gemm_P": 4, "gemm_x": 12, "prox": 40, "xprox": METHOD_BYTES, "block": METHOD_BYTES}
OVERHEAD_BYTES = {"xprox": 8}


def iter_histogram(iters, width: int = 10):
    """Counts of ADMM iterations per account in bins of `width` iterations: {"40-49": n, ...}."""
    out = {}
    for lo in range(0, int(max(iters)) + 1 if len(iters) else 0, width):
        c = int(((iters >= lo) & (iters < lo + width)).sum())
        if c:
            out[f"{lo}-{lo + width - 1}"] = c
    return out


def shard_first_account(rank: int, per_rank: int = M_ACCOUNTS) -> int:
    """First account id of a rank's book: ranks solve disjoint blocks of accounts."""
    return rank * per_rank


def reduce_over_ranks(dist, value: float, op: str, device) -> float:
    """max or sum of a per-rank scalar (host logic of the weak-scaling report)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo")
        return dist, dist.get_rank(), ws, int(os.environ.get("LOCAL_RANK", "0"))
    return None, 0, 1, 0


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def _oracle_worker(args):
    first, seed = args[0], args[1]
    want_w = len(args) > 2 and args[2]
    from oracle.active_set import account_problem
    from paper_2606_23367_gb300.workloads import make_workload
    uni, batch = make_workload(1, seed=seed, first_account=first, M=1)
    t = time.perf_counter()
    r = account_problem(uni, batch, 0).solve()
    dt = time.perf_counter() - t
    return (dt, r.w) if want_w else dt


def _oracle_pool(n):
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    return mp.get_context("spawn").Pool(n)


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_rate(pool, n_workers, accounts, per_account=None, weights=None):
    """Wall-clock accounts/s of the oracle over a list of account ids. per_account, when a
    list, receives each account's own solve time (one single-threaded worker per account);
    weights, when a dict, receives each account's oracle minimiser."""
    t = time.perf_counter()
    out = pool.map(_oracle_worker, [(a, 0, weights is not None) for a in accounts], chunksize=1)
    rate = len(accounts) / (time.perf_counter() - t)
    times = [o[0] for o in out] if weights is not None else out
    if weights is not None:
        for a, o in zip(accounts, out):
            weights[a] = o[1]
    if per_account is not None:
        per_account.extend(times)
    return rate


def _cpu_model():
    """The host CPU's name from /proc/cpuinfo ("model name" on x86; implementer and part
    numbers on Arm), else the machine type."""
    import platform
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return platform.machine()
    kv = {}
    for line in info:
        if ":" in line:
            k, v = line.split(":", 1)
            kv.setdefault(k.strip(), v.strip())
    if "model name" in kv:
        return kv["model name"]
    if "CPU part" in kv:
        return f"{platform.machine()} implementer {kv.get('CPU implementer', '?')} part {kv['CPU part']}"
    return platform.machine()


def run_reference(args, rank):
    if rank != 0:
        return
    n = _cores()
    pool = _oracle_pool(n)
    try:
        pool.map(_oracle_worker, [(a, 0) for a in range(n)], chunksize=1)       # spawn / import warm-up
        rates, per_acc = [], []
        for s in range(args.warmup + args.steps):
            acc = [(s * n + k) % M_ACCOUNTS for k in range(n)]
            r = oracle_rate(pool, n, acc, per_acc if s >= args.warmup else None)
            if s >= args.warmup:
                rates.append(r)
    finally:
        pool.close()
        pool.join()
    value = statistics.median(rates) if rates else 0.0
    sample = f"{n} accounts per step (one per worker), FP64 active-set oracle, workload accounts 0..{M_ACCOUNTS - 1}"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "accounts/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * n / value if value else None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "solver": "FP64 primal active-set oracle (CPU)"},
            "cpu_baseline": {"value": value, "unit": "accounts/s", "cores": n, "kind": "oracle",
                             "sample": sample, "cpu_model": _cpu_model(),
                             "s_per_account_one_core": statistics.median(per_acc) if per_acc else None},
            "e2e": {"value": value, "unit": "accounts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = "timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_id):
        self.proc = None
        self.path = None
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", str(gpu_id)], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self, t0=None, t1=None, min_samples=3):
        """Summarise the samples taken between wall-clock times t0 and t1 (all if None). A timed
        region shorter than the sampling period is widened symmetrically, up to 1 s on each side
        (the same workload runs back to back around it), until it holds min_samples samples;
        the widening is reported."""
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = [ln.strip().split(",") for ln in open(self.path) if ln.strip()]
        os.unlink(self.path)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        import datetime
        parsed = []
        for r in rows:
            try:
                ts = datetime.datetime.strptime(r[0].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
                parsed.append((ts, float(r[1]), float(r[2]),
                               {nm for k, nm in enumerate(names)
                                if len(r) > 4 + k and r[4 + k].strip().lower().startswith("active")}))
            except (ValueError, IndexError):
                continue

        def window(pad):
            return [p for p in parsed if t0 is None or (t0 - pad <= p[0] <= t1 + pad)]

        pad, sel = 0.0, window(0.0)
        while t0 is not None and len(sel) < min_samples and pad < 1.0:
            pad += 0.05
            sel = window(pad)
        if not sel:
            return None
        out = {"sm_mhz": statistics.median(p[1] for p in sel), "sm_max_mhz": max(p[2] for p in sel),
               "reasons": sorted(set().union(*(p[3] for p in sel))), "samples": len(sel)}
        if pad > 0:
            out["window"] = f"timed region widened by {pad * 1e3:.0f} ms on each side"
        return out


def profiled_traffic(kernel_class, entries_per_launch, kernel_name=None):
    """DRAM bytes per launch of a kernel class, from the committed ncu summary of the default
    workload: the captured launch's bytes per account-entry times the entries of this run's
    average launch. None when the kernel's source files have changed since the capture, or when
    kernel_name is given and the captured kernel is another one of the class."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", "dram_traffic_500x10000.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    # | class | `kernel` | entries | read MB | write MB | bytes | files | sha256 prefixes |
    pat = re.compile(r"^\| (\w+) \| `([^`]+)` \| (\d+) \| [\d.]+ \| [\d.]+ \| (\d+) \| (\S+) \| (\S+) \|$")
    for line in text.splitlines():
        m = pat.match(line.strip())
        if not m or m.group(1) != kernel_class:
            continue
        if kernel_name is not None and m.group(2).split("::")[-1] != kernel_name:
            return None
        for f, h in zip(m.group(5).split("+"), m.group(6).split("+")):
            try:
                cur = hashlib.sha256(open(os.path.join(ROOT, f), "rb").read()).hexdigest()
            except OSError:
                return None
            if not cur.startswith(h):
                return None
        return int(m.group(4)) / int(m.group(3)) * entries_per_launch
    return None


def adjoint_timing(stream, reps=5):
    """Forward (keeping the active set) and backward of the differentiation workload at its
    full size, outside the timed region: L = sum_a g_a'w_a with seeded g, device buffers."""
    import numpy as np
    import torch
    from paper_2606_23367_gb300 import prism
    from paper_2606_23367_gb300.workloads import make_workload
    uni, batch = make_workload(4)
    h = prism.create_universe(uni)
    try:
        nnz = int(batch.offsets[-1])
        g = torch.as_tensor(np.random.default_rng(4).normal(size=nnz), device="cuda")
        outs = dict(dmu=torch.zeros(uni.n_assets, dtype=torch.float64, device="cuda"),
                    dB=torch.zeros(uni.n_assets, uni.n_factors, dtype=torch.float64, device="cuda"),
                    dd=torch.zeros(uni.n_assets, dtype=torch.float64, device="cuda"),
                    dw0=torch.zeros(nnz, dtype=torch.float64, device="cuda"))
        fwd, bwd, res = [], [], None
        for _ in range(reps + 1):
            if res is not None:
                res["state"].close()
            res = prism.solve(h, batch, precision=prism.PRISM_BATCHED_BF16, keep_for_backward=1,
                              cuda_stream=stream.cuda_stream)
            fwd.append(res["t_call_ms"])
            t = time.perf_counter()
            prism.prism_solve_batch_backward(res["state"], g, **outs)
            bwd.append((time.perf_counter() - t) * 1e3)
        res["state"].close()
        cert = int((res["status"] == 0).sum())
        return {"workload": "128 accounts x 2,000 assets, K=32, L = sum_a g_a'w_a (seeded g)",
                "forward_ms": statistics.median(fwd[1:]), "backward_ms": statistics.median(bwd[1:]),
                "certified": cert, "accounts": batch.n_accounts,
                "timing": "host wall clock around each C-ABI call, device buffers, median of %d after one warm-up" % reps}
    finally:
        h.close()


# the other workloads, each measured on its own (outside the headline's timed region):
# (id, description, solve options, oracle sample size)
OTHER_WORKLOADS = [
    (0, "1 account x 100 assets, K=10, 10 sector bands (PLAIN_FP64)", dict(precision=3), 1),
    (0, "1 account x 100 assets, K=10, 10 sector bands (PLAIN_FP32)", dict(precision=0), 1),
    (2, "256 ragged accounts from 5,000 assets (100-5,000 names), K=32, dense-masked layout",
     dict(precision=2, ragged_layout=1), 64),
    (2, "256 ragged accounts from 5,000 assets (100-5,000 names), K=32, packed layout",
     dict(precision=2, ragged_layout=2), 64),
    (3, "200 accounts x 1,924 assets, K=48, tax lots, turnover cap 0.2", dict(precision=2), 32),
]


def _oracle_sample_worker(args):
    workload, a = args
    from oracle.active_set import account_problem
    from paper_2606_23367_gb300.workloads import make_workload
    uni, batch = make_workload(workload, first_account=a, M=1)
    t = time.perf_counter()
    r = account_problem(uni, batch, 0).solve()
    return time.perf_counter() - t, r.w


def other_workloads(stream, steps=5, with_cpu=True):
    """Certified accounts/s of each other workload: device lane (inputs resident, CUDA events on
    the solve stream) and e2e lane (pinned host buffers), the dominant kernel class's share and
    method-byte rate, the measured weight error against the oracle on a sample of accounts, and
    the oracle's own rate on that sample (all host cores)."""
    import numpy as np
    import torch
    from paper_2606_23367_gb300 import prism
    from paper_2606_23367_gb300.workloads import instance_hash, make_workload
    out = []
    pool = _oracle_pool(_cores()) if with_cpu else None
    try:
        for wid, desc, opts, n_cpu in OTHER_WORKLOADS:
            uni, batch = make_workload(wid)
            M, S, nnz = batch.n_accounts, uni.n_sectors, int(batch.offsets[-1])
            h = prism.create_universe(uni)
            try:
                def arrs(where):
                    def t(x, dt):
                        if x is None:
                            return None
                        tt = torch.from_numpy(np.ascontiguousarray(x)).to(dt)
                        return tt.cuda() if where == "dev" else tt.pin_memory()
                    f64, i32, i64 = torch.float64, torch.int32, torch.int64
                    inp = dict(offsets=t(batch.offsets, i64), asset_idx=t(batch.asset_idx, i32), w0=t(batch.w0, f64),
                               lower=t(batch.lower, f64), upper=t(batch.upper, f64), tc=t(batch.tc, f64),
                               band_lo=t(batch.band_lo, f64), band_hi=t(batch.band_hi, f64),
                               turnover_cap=t(batch.turnover_cap, f64), lot_offsets=t(batch.lot_offsets, i64),
                               lot_size=t(batch.lot_size, f64), lot_kappa=t(batch.lot_kappa, f64))
                    z = (lambda *sh, dt=torch.float64: torch.zeros(*sh, dtype=dt, device="cuda")) if where == "dev" \
                        else (lambda *sh, dt=torch.float64: torch.zeros(*sh, dtype=dt).pin_memory())
                    res = dict(w=z(nnz), status=torch.zeros(M, dtype=torch.int32).pin_memory(),
                               iters=z(M, dt=torch.int32), nu=z(M), lambda_band=z(M, S), theta=z(M),
                               diag=z(M, prism.PRISM_NDIAG), kappa=z(M, uni.n_factors))
                    return inp, res

                def step(inp, res, **extra):
                    return prism.prism_solve_batch(h, **inp, out=res, cuda_stream=stream.cuda_stream, **opts, **extra)

                def lane(where):
                    inp, res = arrs(where)
                    step(inp, res)
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    cert = 0
                    for _ in range(steps):
                        step(inp, res)
                        cert += int((res["status"].numpy() == 0).sum())
                    e1.record(stream)
                    torch.cuda.synchronize()
                    return cert / (e0.elapsed_time(e1) / 1e3), e0.elapsed_time(e1) / steps, inp, res

                value, ms, din, dres = lane("dev")
                w_dev = dres["w"].cpu().numpy()
                bound = dres["diag"].cpu().numpy()[:, prism.PRISM_DIAG_ERR_EST]
                iters = dres["iters"].cpu().numpy()
                e2e, ms_e2e, hin, hres = lane("host")
                h2d = sum(t.numel() * t.element_size() for t in hin.values() if t is not None)
                d2h = sum(t.numel() * t.element_size() for t in hres.values() if t is not None)
                prof = step(din, dres, profile=1)
                names = prism.KERNEL_CLASSES
                kms, kl = prof["kernel_ms"], prof["kernel_launches"]
                dom = max(range(len(names)), key=lambda i: kms[i])
                # method bytes of the iterations: 24 B per account-entry and iteration
                entries = float(sum((batch.offsets[a + 1] - batch.offsets[a]) * iters[a] for a in range(M)))
                it_ms = sum(kms[names.index(n)] for n in ("gemm_P", "solve_K", "gemm_x", "prox", "xprox", "roots",
                                                         "block"))
                line = {"workload": desc, "config_id": wid, "instance_sha256": instance_hash(uni, batch),
                        "metric": "certified accounts/s", "value": value, "ms_per_step": ms, "steps": steps,
                        "certified": int((dres["status"].numpy() == 0).sum()), "accounts": M,
                        "e2e": {"value": e2e, "ms_per_step": ms_e2e, "h2d_bytes_per_step": h2d,
                                "d2h_bytes_per_step": d2h},
                        "admm_iters": {"median": float(np.median(iters)), "max": int(iters.max())},
                        "dominant_kernel_class": names[dom], "kernel_share": {n: kms[i] / max(1e-9, sum(kms))
                                                                              for i, n in enumerate(names) if kms[i] > 0},
                        "iterations_method_gbs": 24.0 * entries / max(1e-9, it_ms / 1e3) / 1e9,
                        "stated_error_bound_max": float(bound.max())}
                if pool is not None:
                    acc = list(range(min(M, n_cpu)))
                    t0 = time.perf_counter()
                    outs = pool.map(_oracle_sample_worker, [(wid, a) for a in acc], chunksize=1)
                    rate = len(acc) / (time.perf_counter() - t0)
                    errs = [float(np.max(np.abs(w_dev[batch.account_slice(a)] - o[1]))) for a, o in zip(acc, outs)]
                    line["error_vs_oracle"] = {"max_w_err": max(errs), "accounts": len(acc)}
                    line["cpu_baseline"] = {"value": rate, "unit": "accounts/s", "cores": _cores(), "kind": "oracle",
                                            "sample": f"accounts 0..{len(acc) - 1}, one single-threaded FP64 "
                                                      "active-set solve per worker process"}
                out.append(line)
            finally:
                h.close()
    finally:
        if pool is not None:
            pool.close()
            pool.join()
    return out


def queue_and_burden(h, uni, batch, opts, micro_batch=100, window_s=1500.0):
    """The production-queue lane (Sec. 5.1 aggregates, E5 shape) of this book in micro-batches
    through the full-call API with host buffers, and the constraint-burden curve (Table
    "burden") on books of 64 accounts x 2,000 assets; both outside the timed region."""
    import numpy as np
    from paper_2606_23367_gb300 import prism
    from paper_2606_23367_gb300.queue import burden_books, library_solver, run_queue
    solve_opts = {k: v for k, v in opts.items() if k != "cuda_stream"}
    library_solver(h, **solve_opts)(batch.subset(list(range(micro_batch))), window_s)      # warm
    q = run_queue(uni, batch, library_solver(h, **solve_opts), window_s=window_s, micro_batch=micro_batch)
    queue = q.summary()
    queue.update(lane="queue wall clock: dispatch of the queue to the return of each account's call",
                 call_ms=[round(x, 3) for x in q.call_ms], device_ms=[round(x, 3) for x in q.device_ms])
    rows = []
    for name, family, u2, b2 in burden_books(N=2000, K=32, M=64):
        h2 = prism.create_universe(u2)
        try:
            solve_opts2 = {k: v for k, v in solve_opts.items() if k in ("precision",)}
            prism.solve(h2, b2, **solve_opts2)
            calls = []
            for _ in range(3):
                r2 = prism.solve(h2, b2, **solve_opts2)
                calls.append(r2["t_call_ms"])
            rows.append({"bundle": name, "rule_family": family, "taken": True, "accounts": b2.n_accounts,
                         "full_call_ms": statistics.median(calls),
                         "certified": int((r2["status"] == prism.PRISM_CERTIFIED).sum())})
        finally:
            h2.close()
    burden = {"workload": "64 accounts x 2,000 assets, K=32 (seeded synthetic), library default schedule",
              "lane": "full-call wall clock, host buffers, median of 3 after one warm-up", "rows": rows}
    return queue, burden


def run_gpu(args, dist, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2606_23367_gb300 import build, prism
    from paper_2606_23367_gb300.workloads import make_workload

    torch.cuda.set_device(local_rank)
    build.build()
    prism.load_library()
    precision = {"bf16": prism.PRISM_BATCHED_BF16, "fp32": prism.PRISM_BATCHED_FP32}[args.precision]
    if args.workload == 1:
        uni, batch = make_workload(1, first_account=shard_first_account(rank), M=M_ACCOUNTS)
    else:
        # another workload at its own size (profiling and comparisons; the headline is workload 1)
        from paper_2606_23367_gb300.workloads import WORKLOADS
        m_w = WORKLOADS[args.workload]["M"]
        uni, batch = make_workload(args.workload, first_account=rank * m_w)
    M, S = batch.n_accounts, uni.n_sectors
    nnz = int(batch.offsets[-1])
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    h = prism.create_universe(uni, device=local_rank)

    def tens(x, dt, where):
        t = torch.from_numpy(np.ascontiguousarray(x)).to(dt)
        return t.to(dev) if where == "dev" else t.pin_memory()

    def inputs(where):
        opt = lambda x, dt: None if x is None else tens(x, dt, where)
        return dict(offsets=tens(batch.offsets, torch.int64, where), w0=tens(batch.w0, torch.float64, where),
                    lower=tens(batch.lower, torch.float64, where), upper=tens(batch.upper, torch.float64, where),
                    tc=tens(batch.tc, torch.float64, where), band_lo=tens(batch.band_lo, torch.float64, where),
                    band_hi=tens(batch.band_hi, torch.float64, where),
                    turnover_cap=tens(batch.turnover_cap, torch.float64, where),
                    asset_idx=opt(batch.asset_idx, torch.int32), lot_offsets=opt(batch.lot_offsets, torch.int64),
                    lot_size=opt(batch.lot_size, torch.float64), lot_kappa=opt(batch.lot_kappa, torch.float64))

    def outputs(where):
        mk = (lambda *s, dt=torch.float64: torch.zeros(*s, dtype=dt, device=dev)) if where == "dev" else \
             (lambda *s, dt=torch.float64: torch.zeros(*s, dtype=dt).pin_memory())
        # the per-account status always comes back to pinned host memory (2 KB), so that
        # counting certified accounts launches no GPU work of its own
        return dict(w=mk(nnz), status=torch.zeros(M, dtype=torch.int32).pin_memory(),
                    iters=mk(M, dt=torch.int32), nu=mk(M), lambda_band=mk(M, S), theta=mk(M),
                    diag=mk(M, prism.PRISM_NDIAG))

    opts = dict(precision=precision, cuda_stream=stream.cuda_stream)
    if args.ragged_layout is not None:
        opts["ragged_layout"] = args.ragged_layout
    tuned = None
    if not args.no_autotune:
        # the library's autotuner picks the iteration schedule for this book (untimed setup)
        t = prism.autotune(h, batch, precision=precision)
        tuned = {k: t[k] for k in ("rho0", "alpha", "check_every", "stream_after", "chains", "eps_admm", "g2_sets",
                                   "fold_products", "adapt_every", "xupdate_form")}
        opts.update(tuned)

    if args.chains is not None:
        opts["chains"] = args.chains
        if tuned is not None:
            tuned["chains"] = args.chains
    if args.fold_products is not None:
        opts["fold_products"] = args.fold_products
        if tuned is not None:
            tuned["fold_products"] = args.fold_products
    if args.xupdate_form is not None:
        opts["xupdate_form"] = args.xupdate_form
        if tuned is not None:
            tuned["xupdate_form"] = args.xupdate_form

    def step(inp, out, **extra):
        return prism.prism_solve_batch(h, **inp, out=out, **opts, **extra)

    def barrier():
        if dist is not None:
            dist.barrier()

    call_ms = []

    def timed(inp, out, K):
        launches = 0
        cert = 0
        status_np = out["status"].numpy()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        call_ms.clear()
        for _ in range(K):
            r = step(inp, out)
            launches += r["n_launches"]
            call_ms.append((r["t_call_ms"], r["t_device_ms"]))
            cert += int(np.count_nonzero(status_np == prism.PRISM_CERTIFIED))   # host memory, call returned
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return e0.elapsed_time(e1), cert, launches

    def max_over_ranks(x):
        return reduce_over_ranks(dist, x, "max", dev)

    def sum_over_ranks(x):
        return reduce_over_ranks(dist, x, "sum", dev)

    # ---- device-resident lane (the clock sampler starts before the warm-up so that
    # its start-up does not overlap the timed region)
    gpu_id = local_rank
    try:
        gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
        if not gpu_id.startswith("GPU-"):
            gpu_id = "GPU-" + gpu_id
    except Exception:
        gpu_id = local_rank
    clk = Clocks(gpu_id)
    din, dout = inputs("dev"), outputs("dev")
    # untimed pre-warm (at least 2 s of solves) so that the GPU leaves its idle state,
    # then the W warm-up steps of the contract
    t_pre = time.time()
    while time.time() - t_pre < args.prewarm_s:
        step(din, dout)
    for _ in range(args.warmup):
        step(din, dout)
    torch.cuda.synchronize()
    t_wall0 = time.time()
    ms, cert, launches = timed(din, dout, args.steps)
    t_wall1 = time.time()
    dev_calls = list(call_ms)
    clocks = clk.stop(t_wall0, t_wall1)
    ms = max_over_ranks(ms)
    cert_all = sum_over_ranks(cert)
    value = cert_all / (ms / 1000.0)
    status = dout["status"].numpy().copy()
    iters = dout["iters"].cpu().numpy()
    diag = dout["diag"].cpu().numpy()
    w_dev = dout["w"].cpu().numpy()
    # ---- end-to-end lane: pinned host inputs and outputs, copies inside the call
    hin, hout = inputs("host"), outputs("host")
    for _ in range(max(1, args.warmup // 2)):
        step(hin, hout)
    ms_e2e, cert_e2e, _ = timed(hin, hout, args.steps)
    ms_e2e = max_over_ranks(ms_e2e)
    e2e_value = sum_over_ranks(cert_e2e) / (ms_e2e / 1000.0)
    h2d = sum(t.numel() * t.element_size() for t in hin.values() if t is not None)
    d2h = sum(t.numel() * t.element_size() for t in hout.values())
    # ---- per-kernel profile pass (CUDA events around every launch on the solve stream)
    prof = step(din, dout, profile=1)
    kms, kl = prof["kernel_ms"], prof["kernel_launches"]
    names = prism.KERNEL_CLASSES
    it_sum = int(dout["iters"].cpu().numpy().sum())
    N = uni.n_assets
    ix = names.index("xprox")
    classes = ("gemm_P", "gemm_x", "prox", "xprox", "block")
    step_ms = {n: kms[names.index(n)] for n in classes}
    n_launch = {n: kl[names.index(n)] for n in classes}
    # account-entries per launch of each class: the staged prox of the fused schedule runs only
    # the first iterations, over every account; without the fused form it runs every iteration
    # of the accounts still iterating
    fused = kl[ix] > 0
    ent = {"gemm_P": M * N, "gemm_x": M * N,
           "prox": M * N if fused else N * it_sum / max(1, n_launch["prox"])}
    if fused:
        ent["xprox"] = prof["stream_entries"] / kl[ix]
    if n_launch["block"] > 0:
        # the per-account kernel runs every iteration of its accounts in one launch: the
        # account's own names times its iterations
        own = np.diff(batch.offsets).astype(np.float64)
        ent["block"] = float((own * iters).sum()) / n_launch["block"]
    alg = {n: ALG_BYTES[n] * ent[n] for n in ent}
    dom = max(step_ms, key=lambda n: step_ms[n])
    avg_ms = step_ms[dom] / max(1, n_launch[dom])
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = alg[dom] / (avg_ms / 1000.0) / 1e9
    persistent = opts.get("xupdate_form", 0) == 0 and not opts.get("fold_products", 0)
    kernel_of = {"gemm_P": "k_tc_gemm_P", "gemm_x": "k_tc_gemm_x", "prox": "k_prox_stream / k_prox_smem",
                 "xprox": "k_tc_xprox_pers" if persistent else "k_tc_xprox", "block": "k_block_admm"}
    # the whole iteration: the method's bytes of every account-iteration of the step over the
    # step's device time (setup, polish and certification included in the time)
    iter_bytes = METHOD_BYTES * N * float(iters.sum())
    iter_gbs = iter_bytes / (ms / args.steps / 1000.0) / 1e9
    roofline = {"kernel": kernel_of.get(dom, dom), "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": profiled_traffic(dom, ent[dom], kernel_of.get(dom)),
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "alg_bytes_per_unit": ALG_BYTES[dom], "units_per_launch": ent[dom],
                "alg_bytes_per_launch": alg[dom], "avg_launch_ms": avg_ms,
                "overhead_bytes_per_launch": OVERHEAD_BYTES.get(dom, 0) * ent[dom],
                "kernel_share": {n: kms[i] / max(1e-9, sum(kms)) for i, n in enumerate(names)},
                "kernel_gbs": {n: alg[n] / (step_ms[n] / n_launch[n] / 1000.0) / 1e9
                               for n in alg if n_launch[n] > 0 and step_ms[n] > 0},
                "whole_iteration": {"alg_bytes_per_step": iter_bytes, "achieved": iter_gbs,
                                    "frac": iter_gbs / peak,
                                    "rule": f"{METHOD_BYTES} B per account-entry and ADMM iteration over the "
                                            "step's device time"}}
    # ---- plain FP32 single-account form (same GPU, one account per call), in the same lane as
    # value: device-resident inputs, device time of each call from the library's CUDA events
    plain = None
    if rank == 0 and args.plain_sample > 0 and batch.lot_offsets is None:
        np_ = min(args.plain_sample, M)
        e1 = int(batch.offsets[np_])
        sub_in = {k: (None if v is None else v[: np_ + 1] if k == "offsets"
                      else v[:e1] if k in ("w0", "lower", "upper", "tc", "asset_idx") else v[:np_])
                  for k, v in din.items() if not k.startswith("lot_")}
        sub_out = {k: (v[:e1] if k == "w" else v[:np_]) for k, v in dout.items()}
        stp = lambda: prism.prism_solve_batch(h, sub_in["offsets"], sub_in["w0"], sub_in["lower"],
                                              sub_in["upper"], sub_in["tc"], sub_in["band_lo"],
                                              sub_in["band_hi"], turnover_cap=sub_in["turnover_cap"],
                                              asset_idx=sub_in["asset_idx"],
                                              out=sub_out, precision=prism.PRISM_PLAIN_FP32,
                                              cuda_stream=stream.cuda_stream)
        stp()
        torch.cuda.synchronize()
        rp = stp()
        ncert = int((sub_out["status"].numpy() == 0).sum())
        plain = {"value": ncert / (rp["t_device_ms"] / 1000.0), "unit": "accounts/s",
                 "e2e_call": ncert / (rp["t_call_ms"] / 1000.0),
                 "sample": f"{np_} accounts of the same book, one launch sequence per account, FP32 B; "
                           "device-resident inputs, device time (CUDA events) as for value"}
    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only), on every host core;
    # its minimisers also give the measured weight error of the same accounts of this step
    cpu = None
    w_err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n = _cores()
        pool = _oracle_pool(n)
        try:
            pool.map(_oracle_worker, [(a, 0) for a in range(n)], chunksize=1)
            n_acc = min(M, args.cpu_accounts if args.cpu_accounts > 0 else 8 * n)
            acc = list(range(n_acc))
            per_acc, ref_w = [], {}
            rate = oracle_rate(pool, n, acc, per_acc, ref_w)
        finally:
            pool.close()
            pool.join()
        errs = [float(np.max(np.abs(w_dev[batch.account_slice(a)] - ref_w[a]))) for a in acc]
        bnd = diag[acc, prism.PRISM_DIAG_ERR_EST]
        w_err = {"max_w_err_vs_oracle": max(errs), "accounts": len(acc),
                 "max_stated_bound": float(bnd.max()), "bound_holds": bool(all(e <= b + 1e-10 for e, b in zip(errs, bnd)))}
        cpu = {"value": rate, "unit": "accounts/s", "cores": n, "kind": "oracle",
               "sample": f"accounts 0..{len(acc) - 1} of the same workload on {n} worker processes, one "
                         "single-threaded FP64 active-set solve per account",
               "cpu_model": _cpu_model(), "s_per_account_one_core": statistics.median(per_acc)}
    if rank != 0:
        return
    adj = None if args.no_adjoint else adjoint_timing(stream)
    others = None if args.no_others else other_workloads(stream, with_cpu=not args.no_cpu_baseline)
    queue = burden = None
    if not args.no_queue:
        queue, burden = queue_and_burden(h, uni, batch, opts)
    line = {
        "metric": METRIC, "value": value, "unit": "accounts/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16-products/f32-iterations/f64-polish" if args.precision == "bf16"
        else "f32-iterations/f64-polish", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.workload == 1 else WORKLOADS_DESC[args.workload],
                   "accounts_per_gpu": M, "assets": N, "factors": uni.n_factors,
                   "precision": "BATCHED_BF16" if args.precision == "bf16" else "BATCHED_FP32",
                   "l2": "inputs larger than L2 (160 MB of FP64 account data per step)",
                   "parallelism": f"accounts sharded over {world} GPU(s), no collective",
                   "schedule": tuned if tuned is not None else "library defaults"},
        "certified": int(cert_all), "certified_frac": cert_all / (args.steps * M * world),
        "status_counts": {prism.STATUS_NAMES[s]: int((status == s).sum()) for s in set(status.tolist())},
        "admm_iters": {"median": float(np.median(iters)), "max": int(iters.max()),
                       "p10": float(np.percentile(iters, 10)), "p90": float(np.percentile(iters, 90)),
                       "hist": iter_histogram(iters)},
        "max_residual": {"stat": float(diag[:, 4].max()), "budget": float(diag[:, 0].max()),
                         "box": float(diag[:, 1].max())},
        "error_vs_oracle": w_err,
        "stated_error_bound": {"max": float(diag[:, prism.PRISM_DIAG_ERR_EST].max()),
                               "median": float(np.median(diag[:, prism.PRISM_DIAG_ERR_EST])),
                               "what": "per-account a-posteriori bound on max|w - w*| (result diag column 7)"},
        "phase_ms": dict(zip(("setup", "iterate", "polish", "certify"), prof["t_phase_ms"])),
        "roofline": roofline, "cpu_baseline": cpu, "plain_fp32": plain,
        "e2e": {"value": e2e_value, "unit": "accounts/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "bytes_per_account": (h2d + d2h) / M, "ms_per_step": ms_e2e / args.steps},
        "gpu_launches": int(launches), "clocks": clocks,
        "per_call_ms": {"call_median": statistics.median(c for c, _ in dev_calls),
                        "device_median": statistics.median(d for _, d in dev_calls)},
        "adjoint": adj, "queue": queue, "burden": burden, "other_workloads": others,
    }
    print(json.dumps(line), flush=True)
    h.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--plain-sample", type=int, default=64)
    ap.add_argument("--cpu-accounts", type=int, default=0, help="oracle sample (0: 8 per host core)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--prewarm-s", type=float, default=2.0)
    ap.add_argument("--no-autotune", action="store_true", help="use the library's default schedule")
    ap.add_argument("--chains", type=int, default=None, help="account chains of the fused iterations "
                    "(overrides the schedule; 1 = one range, as in the profile pass)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the forward/backward timing of the "
                    "differentiation workload")
    ap.add_argument("--workload", type=int, default=1, choices=[0, 1, 2, 3, 4],
                    help="the book the GPU arm times (default 1, the headline; the others for profiling)")
    ap.add_argument("--fold-products", type=int, default=None, choices=[0, 1],
                    help="fused iterations: B'X of the pinned entries inside the x-update (1) or the separate "
                         "product kernels every iteration (0); default: the library's, or the autotuner's choice")
    ap.add_argument("--xupdate-form", type=int, default=None, choices=[0, 1],
                    help="fused x-update: persistent CTAs taking tiles from a counter (0) or one CTA per tile (1); "
                         "default: the library's, or the autotuner's choice")
    ap.add_argument("--ragged-layout", type=int, default=None, choices=[1, 2],
                    help="ragged books: 1 dense-masked, 2 packed per-account blocks")
    ap.add_argument("--no-others", action="store_true", help="skip the lines of the other workloads "
                    "(single account, ragged, tax-aware)")
    ap.add_argument("--no-queue", action="store_true", help="skip the production-queue and constraint-burden "
                    "lines")
    args = ap.parse_args()
    dist, rank, world, local_rank = _dist()
    if args.impl == "reference":
        run_reference(args, rank)
    else:
        run_gpu(args, dist, rank, world, local_rank)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
