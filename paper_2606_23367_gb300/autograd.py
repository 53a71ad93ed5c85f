"""torch.autograd wrapper: weights as a differentiable function of (mu, B, d, w0).

The forward solves the book with the batched solver and keeps the polished active
set; the backward runs the library's adjoint (prism_solve_batch_backward), which
differentiates the KKT system of Sec. 4.4 on that active set. Argument marshalling
only: both directions run in the library's kernels, on the tensors' own memory.

CUDA tensors stay on the device: their pointers go to the C-ABI as they are, the
forward runs on ``torch.cuda.current_stream()``, and the weights and gradients are
written into device tensors (no host round trip). One universe handle is kept per
(mu, B, d, f, sector) state and reused while those tensors are unchanged (same
storage and version counter). Accounts that do not certify contribute zero
gradient (their active set is not identified).
"""
from __future__ import annotations

import numpy as np
import torch

from . import prism

_UNIVERSES = {}
_MAX_CACHED = 4


def _key(t):
    return (t.device.type, t.device.index, t.data_ptr(), tuple(t.shape), t._version)


def _content(t):
    """Key of a small fixed input (f, sector) by its bytes: callers pass them as new arrays."""
    import hashlib
    return hashlib.sha1(t.detach().cpu().numpy().tobytes()).hexdigest()


def _arg(x, dtype, device):
    """A contiguous tensor of the C-ABI's dtype on ``device`` (numpy arrays are moved there)."""
    if x is None:
        return None
    t = x if isinstance(x, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(x))
    return t.detach().to(device=device, dtype=dtype).contiguous()


def _universe(mu, B, d, spec):
    f = _arg(spec["f"], torch.float64, B.device)
    sector = _arg(spec["sector"], torch.int32, B.device)
    key = (_key(mu), _key(B), _key(d), _content(f), _content(sector), int(spec["n_sectors"]))
    h = _UNIVERSES.get(key)
    if h is None or h.handle is None:
        device = B.device.index if B.is_cuda else int(spec.get("device", 0))
        h = prism.prism_create_universe(B, f, d, mu, sector, int(spec["n_sectors"]), device)
        if len(_UNIVERSES) >= _MAX_CACHED:
            # dropped, not closed: a backward state of an earlier forward may still hold it
            _UNIVERSES.pop(next(iter(_UNIVERSES)))
        _UNIVERSES[key] = h
        h._keep = (mu, B, d)                     # the key's storages stay alive with the handle
    return h


class RebalanceFunction(torch.autograd.Function):
    """w = RebalanceFunction.apply(mu, B, d, w0, spec) with ``spec`` a dict of the fixed
    inputs: f, sector, n_sectors, offsets, lower, upper, tc, band_lo, band_hi and
    optionally asset_idx, turnover_cap, lot_offsets, lot_size, lot_kappa, precision."""

    @staticmethod
    def forward(ctx, mu, B, d, w0, spec):
        dev = w0.device
        f64, i32, i64 = torch.float64, torch.int32, torch.int64
        mu_, B_, d_ = (_arg(t, f64, dev) for t in (mu, B, d))
        u = _universe(mu_, B_, d_, spec)
        offsets = _arg(spec["offsets"], i64, dev)
        nnz, M, S = int(offsets[-1]), int(offsets.shape[0]) - 1, int(spec["n_sectors"])
        out = dict(w=torch.zeros(nnz, dtype=f64, device=dev), status=torch.zeros(M, dtype=i32),
                   iters=None, nu=None, lambda_band=None, theta=None, diag=None)
        if dev.type == "cuda":
            out["status"] = out["status"].pin_memory()
        stream = torch.cuda.current_stream(dev).cuda_stream if dev.type == "cuda" else None
        opt = {"cuda_stream": stream} if stream is not None else {}
        res = prism.prism_solve_batch(
            u, offsets, _arg(w0, f64, dev), _arg(spec["lower"], f64, dev), _arg(spec["upper"], f64, dev),
            _arg(spec["tc"], f64, dev), _arg(spec["band_lo"], f64, dev), _arg(spec["band_hi"], f64, dev),
            asset_idx=_arg(spec.get("asset_idx"), i32, dev), turnover_cap=_arg(spec.get("turnover_cap"), f64, dev),
            lot_offsets=_arg(spec.get("lot_offsets"), i64, dev), lot_size=_arg(spec.get("lot_size"), f64, dev),
            lot_kappa=_arg(spec.get("lot_kappa"), f64, dev),
            precision=int(spec.get("precision", prism.PRISM_BATCHED_BF16)), keep_for_backward=1, out=out, **opt)
        ctx.state = res["state"]
        ctx.status = res["status"]
        ctx.shapes = (mu.shape, B.shape, d.shape, w0.shape)
        return out["w"]

    @staticmethod
    def backward(ctx, grad_w):
        dev = grad_w.device
        g = grad_w.detach().to(torch.float64).contiguous()
        if dev.type == "cuda":
            # the library's adjoint runs on its own stream: the gradient must be written first
            torch.cuda.current_stream(dev).synchronize()
        z = lambda shape: torch.zeros(shape, dtype=torch.float64, device=dev)
        sm, sB, sd, sw0 = ctx.shapes
        out = dict(dmu=z(sm), dB=z(sB), dd=z(sd), dw0=z(sw0))
        prism.prism_solve_batch_backward(ctx.state, g, **out)   # returns after its stream is done
        return out["dmu"], out["dB"], out["dd"], out["dw0"], None


def solve(mu, B, d, w0, **spec):
    """Differentiable solve: returns the ragged weights; gradients flow to mu, B, d, w0."""
    return RebalanceFunction.apply(mu, B, d, w0, spec)
