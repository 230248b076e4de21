"""Expected degrees as a differentiable torch op and weight calibration.

``ExpectedDegree`` is a ``torch.autograd.Function`` whose forward and backward
are the library's hand-written kernels (``cl_expected_degree`` and
``cl_expected_degree_adjoint``); torch only holds the tensors.  ``calibrate``
calls ``cl_calibrate`` (preconditioned gradient descent on
sum (E - d)^2 / d, all steps in the library's kernels).
"""
from __future__ import annotations

import torch

from . import (cl_calib_opts, cl_calibrate, cl_calibrate_workspace_bytes, cl_expected_degree,
               cl_expected_degree_adjoint, cl_expected_degree_workspace_bytes)


def _ws(n: int, device) -> torch.Tensor:
    return torch.empty(cl_expected_degree_workspace_bytes(n), dtype=torch.uint8, device=device)


class ExpectedDegree(torch.autograd.Function):
    """E_u = sum_{v != u} min(1, w_u w_v / S), S = sum w, for float64 weights on
    the GPU sorted non-increasing; backward applies the exact adjoint."""

    @staticmethod
    def forward(ctx, w: torch.Tensor) -> torch.Tensor:
        if w.dtype != torch.float64 or not w.is_cuda:
            raise TypeError("weights must be a float64 CUDA tensor")
        w = w.contiguous()
        n = w.numel()
        E = torch.empty_like(w)
        ws = _ws(n, w.device)
        cl_expected_degree(w, n, 0.0, E, ws, ws.numel())
        ctx.save_for_backward(w)
        return E

    @staticmethod
    def backward(ctx, gE: torch.Tensor):
        (w,) = ctx.saved_tensors
        n = w.numel()
        gw = torch.empty_like(w)
        ws = _ws(n, w.device)
        cl_expected_degree_adjoint(w, gE.contiguous().to(torch.float64), n, 0.0, gw, ws, ws.numel())
        return gw


def expected_degree(w: torch.Tensor) -> torch.Tensor:
    return ExpectedDegree.apply(w)


def calibrate(target: torch.Tensor, tol: float = 1e-9, max_iter: int = 100, w0: torch.Tensor | None = None):
    """Weights whose expected degrees match ``target`` (float64, sorted
    non-increasing, on the GPU) within ``tol`` relative.  Returns (w, report)."""
    n = target.numel()
    w = (w0.clone() if w0 is not None else torch.empty_like(target)).contiguous()
    ws = torch.empty(cl_calibrate_workspace_bytes(n), dtype=torch.uint8, device=target.device)
    opts = cl_calib_opts(tol, max_iter, 1 if w0 is not None else 0)
    st, rep = cl_calibrate(target.contiguous(), n, w, opts, ws, ws.numel())
    rep["converged"] = st == 0
    return w, rep
