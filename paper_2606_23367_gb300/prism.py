"""Thin Python binding of the C-ABI in include/prism.h (argument marshalling only).

Every step of the solve runs in libprism.so; this module only lays out the
C structs, passes host (numpy) or device (torch CUDA tensor) pointers and
raises on a negative return code. It fails loudly when the library has not
been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libprism.so")

PRISM_OK = 0
PRISM_ERR_ARGUMENT, PRISM_ERR_CUDA, PRISM_ERR_ALLOCATION, PRISM_ERR_UNSUPPORTED = -1, -2, -3, -4
PRISM_CERTIFIED, PRISM_FEASIBLE_NONCERTIFIED, PRISM_TIMEOUT, PRISM_DEADLINE_EXCEEDED = 0, 1, 2, 3
PRISM_NO_FEASIBLE_RETURN, PRISM_ALLOCATION_FAILURE, PRISM_NUMERICAL_FAILURE = 4, 5, 6
PRISM_PLAIN_FP32, PRISM_BATCHED_FP32, PRISM_BATCHED_BF16, PRISM_PLAIN_FP64 = 0, 1, 2, 3
PRISM_PRODUCTS_FUSED = 0x100        # prism_shared_b_products: P from the fused x-update kernel
PRISM_NDIAG = 8
(PRISM_DIAG_BUDGET, PRISM_DIAG_BOX, PRISM_DIAG_EXPOSURE, PRISM_DIAG_TURNOVER, PRISM_DIAG_STAT, PRISM_DIAG_COMP,
 PRISM_DIAG_OBJ, PRISM_DIAG_ERR_EST) = range(8)
KERNEL_CLASSES = ("gemm_P", "solve_K", "gemm_x", "prox", "polish", "pack", "other", "unpack", "xprox", "roots",
                  "block")
DIAG_NAMES = ("r_budget", "r_box", "r_exposure", "r_turnover", "r_stat", "r_comp", "obj", "w_err_bound")
STATUS_NAMES = ("CERTIFIED", "FEASIBLE_NONCERTIFIED", "TIMEOUT", "DEADLINE_EXCEEDED",
                "NO_FEASIBLE_RETURN", "ALLOCATION_FAILURE", "NUMERICAL_FAILURE")

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_lp = C.POINTER(C.c_int64)


class PrismError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"prism error {code}: {msg}")
        self.code = code


class _UniverseDesc(C.Structure):
    _fields_ = [("n_assets", C.c_int32), ("n_factors", C.c_int32), ("n_sectors", C.c_int32),
                ("B", C.c_void_p), ("f", C.c_void_p), ("d", C.c_void_p), ("mu", C.c_void_p),
                ("sector", C.c_void_p), ("device", C.c_int32)]


class _Batch(C.Structure):
    _fields_ = [("n_accounts", C.c_int32), ("offsets", C.c_void_p), ("asset_idx", C.c_void_p),
                ("w0", C.c_void_p), ("lower", C.c_void_p), ("upper", C.c_void_p), ("tc", C.c_void_p),
                ("band_lo", C.c_void_p), ("band_hi", C.c_void_p), ("turnover_cap", C.c_void_p),
                ("lot_offsets", C.c_void_p), ("lot_size", C.c_void_p), ("lot_kappa", C.c_void_p),
                ("mu_tilt", C.c_void_p), ("w_bench", C.c_void_p), ("factor_lo", C.c_void_p),
                ("factor_hi", C.c_void_p)]


class _Opts(C.Structure):
    _fields_ = [("eps_kkt", C.c_double), ("eps_admm", C.c_double), ("rho0", C.c_double),
                ("alpha", C.c_double), ("time_budget_s", C.c_double), ("max_iter", C.c_int32),
                ("check_every", C.c_int32), ("min_iter", C.c_int32), ("polish_rounds", C.c_int32),
                ("precision", C.c_int32), ("use_graph", C.c_int32), ("keep_for_backward", C.c_int32),
                ("profile", C.c_int32), ("polish_overlap", C.c_double), ("chains", C.c_int32), ("stream_after", C.c_int32), ("fuse_prox", C.c_int32),
                ("cuda_stream", C.c_void_p), ("ragged_layout", C.c_int32), ("g2_sets", C.c_int32),
                ("fold_products", C.c_int32), ("adapt_every", C.c_int32),
                ("xupdate_form", C.c_int32)]


class _Result(C.Structure):
    _fields_ = [("w", C.c_void_p), ("nu", C.c_void_p), ("lambda_band", C.c_void_p), ("theta", C.c_void_p),
                ("status", C.c_void_p), ("iters", C.c_void_p), ("diag", C.c_void_p),
                ("t_device_ms", C.c_double), ("t_call_ms", C.c_double), ("t_phase_ms", C.c_double * 4),
                ("device_bytes", C.c_int64), ("n_launches", C.c_int64),
                ("kernel_ms", C.c_double * len(KERNEL_CLASSES)), ("kernel_launches", C.c_int64 * len(KERNEL_CLASSES)),
                ("stream_entries", C.c_int64), ("stream_candidates", C.c_int64), ("state", C.c_void_p),
                ("kappa", C.c_void_p)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libprism.so (built by paper_2606_23367_gb300.build); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2606_23367_gb300.build.build()")
    lib = C.CDLL(path)
    lib.prism_create_universe.argtypes = [C.POINTER(_UniverseDesc), C.POINTER(C.c_void_p)]
    lib.prism_create_universe.restype = C.c_int
    lib.prism_destroy_universe.argtypes = [C.c_void_p]
    lib.prism_destroy_universe.restype = None
    lib.prism_default_opts.argtypes = [C.POINTER(_Opts)]
    lib.prism_default_opts.restype = None
    lib.prism_solve_batch.argtypes = [C.c_void_p, C.POINTER(_Batch), C.POINTER(_Opts), C.POINTER(_Result)]
    lib.prism_solve_batch.restype = C.c_int
    lib.prism_solve_batch_backward.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                               C.c_void_p, C.c_void_p]
    lib.prism_solve_batch_backward.restype = C.c_int
    lib.prism_shared_b_products.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32,
                                            C.c_void_p, C.c_void_p]
    lib.prism_shared_b_products.restype = C.c_int
    lib.prism_polish_noalloc.argtypes = [C.c_void_p, C.POINTER(_Batch), C.c_void_p, C.POINTER(_Opts),
                                         C.POINTER(_Result)]
    lib.prism_polish_noalloc.restype = C.c_int
    lib.prism_autotune.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.prism_autotune.restype = C.c_int
    lib.prism_free_state.argtypes = [C.c_void_p]
    lib.prism_free_state.restype = None
    lib.prism_last_error.argtypes = []
    lib.prism_last_error.restype = C.c_char_p
    lib.prism_version.argtypes = []
    lib.prism_version.restype = C.c_char_p
    _lib = lib
    return lib


def _check(rc):
    if rc != PRISM_OK:
        raise PrismError(rc, load_library().prism_last_error().decode())


class _Keep:
    """Holds the host arrays whose pointers were handed to C for the call's duration."""

    def __init__(self):
        self.refs = []

    def ptr(self, x, dtype):
        if x is None:
            return None
        if hasattr(x, "data_ptr"):            # torch tensor (host or CUDA)
            import torch
            want = {np.float64: torch.float64, np.int32: torch.int32, np.int64: torch.int64}[dtype]
            if x.dtype != want or not x.is_contiguous():
                raise TypeError(f"tensor must be contiguous {want}")
            self.refs.append(x)
            return x.data_ptr()
        a = np.ascontiguousarray(x, dtype=dtype)
        self.refs.append(a)
        return a.ctypes.data


def prism_version() -> str:
    return load_library().prism_version().decode()


def prism_last_error() -> str:
    return load_library().prism_last_error().decode()


class UniverseHandle:
    def __init__(self, handle, n_assets, n_factors, n_sectors):
        self.handle = handle
        self.n_assets, self.n_factors, self.n_sectors = n_assets, n_factors, n_sectors

    def close(self):
        if self.handle:
            load_library().prism_destroy_universe(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def prism_create_universe(B, f, d, mu, sector, n_sectors, device=0) -> UniverseHandle:
    lib = load_library()
    keep = _Keep()
    N, K = int(B.shape[0]), int(B.shape[1])
    desc = _UniverseDesc(N, K, int(n_sectors), keep.ptr(B, np.float64), keep.ptr(f, np.float64),
                         keep.ptr(d, np.float64), keep.ptr(mu, np.float64), keep.ptr(sector, np.int32),
                         int(device))
    h = C.c_void_p()
    _check(lib.prism_create_universe(C.byref(desc), C.byref(h)))
    return UniverseHandle(h.value, N, K, int(n_sectors))


def prism_destroy_universe(u: UniverseHandle):
    u.close()


def prism_default_opts() -> dict:
    o = _Opts()
    load_library().prism_default_opts(C.byref(o))
    return {name: getattr(o, name) for name, _ in _Opts._fields_}


def _to_numpy(x):
    return x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)


def prism_solve_batch(u: UniverseHandle, offsets, w0, lower, upper, tc, band_lo, band_hi,
                      asset_idx=None, turnover_cap=None, lot_offsets=None, lot_size=None,
                      lot_kappa=None, mu_tilt=None, w_bench=None, factor_lo=None, factor_hi=None,
                      out=None, **opts) -> dict:
    """Solve a book of accounts. Array arguments are numpy arrays (host) or torch
    tensors (host or CUDA). ``out`` may supply preallocated outputs with keys
    w/status/iters/nu/lambda_band/theta/diag (device or host); otherwise numpy
    outputs are allocated. Returns a dict of outputs and timings."""
    lib = load_library()
    keep = _Keep()
    M = int(len(offsets) - 1)
    nnz = int(_to_numpy(offsets[-1:])[0]) if hasattr(offsets, "cpu") else int(offsets[-1])
    S = u.n_sectors
    b = _Batch(M, keep.ptr(offsets, np.int64), keep.ptr(asset_idx, np.int32),
               keep.ptr(w0, np.float64), keep.ptr(lower, np.float64), keep.ptr(upper, np.float64),
               keep.ptr(tc, np.float64), keep.ptr(band_lo, np.float64), keep.ptr(band_hi, np.float64),
               keep.ptr(turnover_cap, np.float64), keep.ptr(lot_offsets, np.int64),
               keep.ptr(lot_size, np.float64), keep.ptr(lot_kappa, np.float64),
               keep.ptr(mu_tilt, np.float64), keep.ptr(w_bench, np.float64),
               keep.ptr(factor_lo, np.float64), keep.ptr(factor_hi, np.float64))
    o = _Opts()
    lib.prism_default_opts(C.byref(o))
    for k, v in opts.items():
        if k == "cuda_stream":
            o.cuda_stream = v
        elif not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        else:
            setattr(o, k, v)
    if out is None:
        out = dict(w=np.zeros(nnz), status=np.zeros(M, np.int32), iters=np.zeros(M, np.int32),
                   nu=np.zeros(M), lambda_band=np.zeros((M, S)), theta=np.zeros(M),
                   diag=np.zeros((M, PRISM_NDIAG)), kappa=np.zeros((M, u.n_factors)))
    r = _Result()
    r.w = keep.ptr(out["w"], np.float64)
    r.status = keep.ptr(out["status"], np.int32)
    for k in ("iters",):
        if out.get(k) is not None:
            setattr(r, k, keep.ptr(out[k], np.int32))
    for k in ("nu", "lambda_band", "theta", "diag", "kappa"):
        if out.get(k) is not None:
            setattr(r, k, keep.ptr(out[k], np.float64))
    holder = C.c_void_p(None)
    if o.keep_for_backward:
        r.state = C.addressof(holder)
    _check(lib.prism_solve_batch(u.handle, C.byref(b), C.byref(o), C.byref(r)))
    res = dict(out)
    res.update(t_device_ms=r.t_device_ms, t_call_ms=r.t_call_ms, t_phase_ms=list(r.t_phase_ms),
               device_bytes=r.device_bytes, n_launches=r.n_launches,
               kernel_ms=list(r.kernel_ms), kernel_launches=list(r.kernel_launches),
               stream_entries=int(r.stream_entries), stream_candidates=int(r.stream_candidates))
    if o.keep_for_backward:
        res["state"] = BackwardState(holder.value, u, nnz)
    return res


def prism_autotune(u: UniverseHandle, offsets, w0, lower, upper, tc, band_lo, band_hi,
                   asset_idx=None, turnover_cap=None, lot_offsets=None, lot_size=None, lot_kappa=None,
                   mu_tilt=None, w_bench=None, factor_lo=None, factor_hi=None, **base) -> dict:
    """Schedule chosen by the library's autotuner for this book (see prism.h): a dict of
    solve options (rho0, alpha, check_every, stream_after and the base options) to pass to a solve."""
    lib = load_library()
    keep = _Keep()
    M = int(len(offsets) - 1)
    b = _Batch(M, keep.ptr(offsets, np.int64), keep.ptr(asset_idx, np.int32),
               keep.ptr(w0, np.float64), keep.ptr(lower, np.float64), keep.ptr(upper, np.float64),
               keep.ptr(tc, np.float64), keep.ptr(band_lo, np.float64), keep.ptr(band_hi, np.float64),
               keep.ptr(turnover_cap, np.float64), keep.ptr(lot_offsets, np.int64),
               keep.ptr(lot_size, np.float64), keep.ptr(lot_kappa, np.float64),
               keep.ptr(mu_tilt, np.float64), keep.ptr(w_bench, np.float64),
               keep.ptr(factor_lo, np.float64), keep.ptr(factor_hi, np.float64))
    o = _Opts()
    lib.prism_default_opts(C.byref(o))
    for k, v in base.items():
        if k == "cuda_stream":
            o.cuda_stream = v
        elif not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        else:
            setattr(o, k, v)
    t = _Opts()
    _check(lib.prism_autotune(u.handle, C.byref(b), C.byref(o), C.byref(t)))
    out = {name: getattr(t, name) for name, _ in _Opts._fields_ if name != "cuda_stream"}
    return out


def autotune(handle: UniverseHandle, batch, **base) -> dict:
    return prism_autotune(handle, batch.offsets, batch.w0, batch.lower, batch.upper, batch.tc,
                          batch.band_lo, batch.band_hi, asset_idx=batch.asset_idx,
                          turnover_cap=batch.turnover_cap, lot_offsets=batch.lot_offsets,
                          lot_size=batch.lot_size, lot_kappa=batch.lot_kappa, **_families(batch), **base)


def prism_shared_b_products(u: UniverseHandle, X, Q, precision=PRISM_BATCHED_BF16):
    """P = X B and BQ = Q B' on the solver's kernels (diagnostic; see prism.h)."""
    lib = load_library()
    keep = _Keep()
    X = np.ascontiguousarray(X, np.float64)
    Q = np.ascontiguousarray(Q, np.float64)
    M = X.shape[0]
    P = np.zeros((M, u.n_factors))
    BQ = np.zeros((M, u.n_assets))
    _check(lib.prism_shared_b_products(u.handle, M, keep.ptr(X, np.float64), keep.ptr(Q, np.float64),
                                       int(precision), P.ctypes.data, BQ.ctypes.data))
    return P, BQ


def prism_polish_noalloc(u: UniverseHandle, offsets, w0, lower, upper, tc, band_lo, band_hi, w_in,
                         asset_idx=None, turnover_cap=None, out=None, **opts) -> dict:
    """Polish and certify the weights w_in without any device allocation (see prism.h)."""
    lib = load_library()
    keep = _Keep()
    M = int(len(offsets) - 1)
    nnz = int(_to_numpy(offsets[-1:])[0]) if hasattr(offsets, "cpu") else int(offsets[-1])
    S = u.n_sectors
    b = _Batch(M, keep.ptr(offsets, np.int64), keep.ptr(asset_idx, np.int32),
               keep.ptr(w0, np.float64), keep.ptr(lower, np.float64), keep.ptr(upper, np.float64),
               keep.ptr(tc, np.float64), keep.ptr(band_lo, np.float64), keep.ptr(band_hi, np.float64),
               keep.ptr(turnover_cap, np.float64), None, None, None, None, None, None, None)
    o = _Opts()
    lib.prism_default_opts(C.byref(o))
    for k, v in opts.items():
        setattr(o, k, v)
    if out is None:
        out = dict(w=np.zeros(nnz), status=np.zeros(M, np.int32), iters=np.zeros(M, np.int32),
                   nu=np.zeros(M), lambda_band=np.zeros((M, S)), theta=np.zeros(M),
                   diag=np.zeros((M, PRISM_NDIAG)))
    r = _Result()
    r.w = keep.ptr(out["w"], np.float64)
    r.status = keep.ptr(out["status"], np.int32)
    if out.get("iters") is not None:
        r.iters = keep.ptr(out["iters"], np.int32)
    for k in ("nu", "lambda_band", "theta", "diag"):
        if out.get(k) is not None:
            setattr(r, k, keep.ptr(out[k], np.float64))
    _check(lib.prism_polish_noalloc(u.handle, C.byref(b), keep.ptr(w_in, np.float64), C.byref(o), C.byref(r)))
    res = dict(out)
    res.update(t_call_ms=r.t_call_ms, device_bytes=r.device_bytes, n_launches=r.n_launches)
    return res


class BackwardState:
    """The active set kept by a solve with keep_for_backward=1 (owns the C state; keeps
    its universe alive)."""

    def __init__(self, ptr, universe, nnz):
        self.ptr = ptr
        self.universe = universe
        self.nnz = nnz

    def close(self):
        if self.ptr:
            prism_free_state(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def prism_solve_batch_backward(state, dL_dw, dmu=None, dB=None, dd=None, dw0=None) -> dict:
    """Gradients of L (given dL/dw, ragged) with respect to mu (N), B (N x K), d (N) and w0
    (ragged) through the polished KKT system. Outputs may be supplied (host or device);
    missing ones are allocated as numpy arrays."""
    lib = load_library()
    keep = _Keep()
    u = state.universe
    N, K = u.n_assets, u.n_factors
    dmu = np.zeros(N) if dmu is None else dmu
    dB = np.zeros((N, K)) if dB is None else dB
    dd = np.zeros(N) if dd is None else dd
    dw0 = np.zeros(state.nnz) if dw0 is None else dw0
    _check(lib.prism_solve_batch_backward(state.ptr, keep.ptr(dL_dw, np.float64), keep.ptr(dmu, np.float64),
                                          keep.ptr(dB, np.float64), keep.ptr(dd, np.float64),
                                          keep.ptr(dw0, np.float64)))
    return dict(dmu=dmu, dB=dB, dd=dd, dw0=dw0)


def prism_free_state(state):
    load_library().prism_free_state(state)


# ---- conveniences over the workload dataclasses (duck-typed) -------------

def create_universe(uni, device=0) -> UniverseHandle:
    return prism_create_universe(uni.B, uni.f, uni.d, uni.mu, uni.sector, uni.n_sectors, device)


def _families(batch) -> dict:
    """The optional Eq. 1 families of a batch (tilt, benchmark, factor-exposure bounds)."""
    return {k: getattr(batch, k, None) for k in ("mu_tilt", "w_bench", "factor_lo", "factor_hi")}


def solve(handle: UniverseHandle, batch, **opts) -> dict:
    return prism_solve_batch(handle, batch.offsets, batch.w0, batch.lower, batch.upper, batch.tc,
                             batch.band_lo, batch.band_hi, asset_idx=batch.asset_idx,
                             turnover_cap=batch.turnover_cap, lot_offsets=batch.lot_offsets,
                             lot_size=batch.lot_size, lot_kappa=batch.lot_kappa, **_families(batch),
                             **opts)
