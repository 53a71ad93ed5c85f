"""torch.autograd wrapper: weights as a differentiable function of (mu, B, d, w0).

The forward solves the book with the batched solver and keeps the polished active
set; the backward runs the library's adjoint (prism_solve_batch_backward), which
differentiates the KKT system of Sec. 4.4 on that active set. Argument marshalling
only: both directions run in the library's kernels. Accounts that do not certify
contribute zero gradient (their active set is not identified).
"""
from __future__ import annotations

import numpy as np
import torch

from . import prism


def _np(t):
    return t.detach().to("cpu", torch.float64).numpy()


class RebalanceFunction(torch.autograd.Function):
    """w = RebalanceFunction.apply(mu, B, d, w0, spec) with ``spec`` a dict of the fixed
    inputs: f, sector, n_sectors, offsets, lower, upper, tc, band_lo, band_hi and
    optionally asset_idx, turnover_cap, lot_offsets, lot_size, lot_kappa, precision."""

    @staticmethod
    def forward(ctx, mu, B, d, w0, spec):
        u = prism.prism_create_universe(_np(B), np.asarray(spec["f"], np.float64), _np(d), _np(mu),
                                        np.asarray(spec["sector"], np.int32), int(spec["n_sectors"]),
                                        int(spec.get("device", 0)))
        res = prism.prism_solve_batch(
            u, np.asarray(spec["offsets"], np.int64), _np(w0), spec["lower"], spec["upper"], spec["tc"],
            spec["band_lo"], spec["band_hi"], asset_idx=spec.get("asset_idx"),
            turnover_cap=spec.get("turnover_cap"), lot_offsets=spec.get("lot_offsets"),
            lot_size=spec.get("lot_size"), lot_kappa=spec.get("lot_kappa"),
            precision=int(spec.get("precision", prism.PRISM_BATCHED_BF16)), keep_for_backward=1)
        ctx.state = res["state"]
        ctx.status = res["status"]
        return torch.as_tensor(res["w"], dtype=torch.float64, device=w0.device)

    @staticmethod
    def backward(ctx, grad_w):
        g = _np(grad_w.contiguous())
        out = prism.prism_solve_batch_backward(ctx.state, g)
        dev = grad_w.device
        t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)
        return t(out["dmu"]), t(out["dB"]), t(out["dd"]), t(out["dw0"]), None


def solve(mu, B, d, w0, **spec):
    """Differentiable solve: returns the ragged weights; gradients flow to mu, B, d, w0."""
    return RebalanceFunction.apply(mu, B, d, w0, spec)
