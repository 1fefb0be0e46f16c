"""Differentiable reweighting of population annealing (Sec. 2 step 2 of
arXiv:1704.01888) as torch.autograd.Functions.

For a population with energies E (CUDA int32 tensor) and a temperature step
dbeta (CUDA float64 scalar tensor), with tau_j = exp(-dbeta E_j) / Q:

    ln Q(dbeta)   = ln( sum_j exp(-dbeta E_j) / R )     d/d dbeta = -<E>_tau
    <E>_tau       = sum_j E_j tau_j / R                  d/d dbeta = -var_tau(E)
    var_tau(E)                                           d/d dbeta = -k3_tau(E)
    <O>_tau       = sum_j O_j tau_j / R                  d/d dbeta = -cov_tau(O, E),
                                                         d/d O_j   = tau_j / R

Forward values come from the library's reweighting kernel
(pa_reweight_forward); the backward passes are the library's kernels
pa_reweight_scale (gradient with respect to dbeta) and pa_reweight_grad_O
(gradient with respect to O).  Second derivatives (create_graph=True) chain
the same Functions, so d^2 ln Q / d dbeta^2 = var_tau(E) comes out of autograd.
"""
from __future__ import annotations

import torch

from . import _check, load_library

# forward output index of each moment order: ln Q, <E>, var, k3
_IDX = (0, 1, 2, 7)


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _as_dbeta(dbeta, device) -> torch.Tensor:
    if not torch.is_tensor(dbeta):
        dbeta = torch.tensor(float(dbeta), dtype=torch.float64, device=device)
    if dbeta.dtype != torch.float64 or dbeta.device.type != "cuda" or dbeta.numel() != 1:
        raise ValueError("dbeta must be a CUDA float64 scalar tensor")
    return dbeta


def _check_E(E: torch.Tensor):
    if E.dtype != torch.int32 or E.device.type != "cuda" or not E.is_contiguous() or E.dim() != 1:
        raise ValueError("E must be a contiguous 1-d CUDA int32 tensor")


def reweight_forward(E: torch.Tensor, dbeta: torch.Tensor, O: torch.Tensor | None = None) -> torch.Tensor:
    """All reweighting outputs (float64[8], see include/pa.h)."""
    _check_E(E)
    out = torch.empty(8, dtype=torch.float64, device=E.device)
    if O is not None:
        O = O.contiguous()
        if O.dtype != torch.float64 or O.numel() != E.numel():
            raise ValueError("O must be float64 with one value per replica")
    _check(load_library().pa_reweight_forward(E.data_ptr(), O.data_ptr() if O is not None else None, E.numel(),
                                              dbeta.data_ptr(), out.data_ptr(), _stream()), "pa_reweight_forward")
    return out


def _scale(src: torch.Tensor, idx: int, sign: float, g: torch.Tensor) -> torch.Tensor:
    g = g.to(torch.float64).contiguous()
    dst = torch.empty((), dtype=torch.float64, device=src.device)
    _check(load_library().pa_reweight_scale(src.data_ptr(), idx, float(sign), g.data_ptr(), dst.data_ptr(), _stream()),
           "pa_reweight_scale")
    return dst


class _Moment(torch.autograd.Function):
    """Moment `order` (0: ln Q, 1: <E>_tau, 2: var_tau(E), 3: k3_tau(E)) as a
    function of dbeta; its derivative is minus the next moment."""

    @staticmethod
    def forward(ctx, dbeta, E, order):
        out = reweight_forward(E, dbeta)
        ctx.save_for_backward(dbeta, E, out)
        ctx.order = order
        return out[_IDX[order]].clone()

    @staticmethod
    def backward(ctx, g):
        dbeta, E, out = ctx.saved_tensors
        order = ctx.order
        if order >= 3:
            raise NotImplementedError("derivatives beyond the third cumulant are not provided")
        if torch.is_grad_enabled():
            # differentiable backward (create_graph=True): chain the next moment
            return -(g * _Moment.apply(dbeta, E, order + 1)), None, None
        return _scale(out, _IDX[order + 1], -1.0, g), None, None


class _Reweighted(torch.autograd.Function):
    """<O>_tau as a function of O and dbeta."""

    @staticmethod
    def forward(ctx, O, dbeta, E):
        out = reweight_forward(E, dbeta, O)
        ctx.save_for_backward(O, dbeta, E, out)
        return out[3].clone()

    @staticmethod
    def backward(ctx, g):
        O, dbeta, E, out = ctx.saved_tensors
        g = g.to(torch.float64).contiguous()
        grad_O = None
        if ctx.needs_input_grad[0]:
            grad_O = torch.empty_like(O, dtype=torch.float64)
            _check(load_library().pa_reweight_grad_O(E.data_ptr(), E.numel(), dbeta.data_ptr(), out.data_ptr(),
                                                     g.data_ptr(), grad_O.data_ptr(), _stream()), "pa_reweight_grad_O")
        grad_d = _scale(out, 4, -1.0, g) if ctx.needs_input_grad[1] else None
        return grad_O, grad_d, None


def lnQ(dbeta, E: torch.Tensor) -> torch.Tensor:
    """ln Q(dbeta; E), differentiable in dbeta (to third order)."""
    return _Moment.apply(_as_dbeta(dbeta, E.device), E, 0)


def mean_energy(dbeta, E: torch.Tensor) -> torch.Tensor:
    """<E>_tau(dbeta), differentiable in dbeta."""
    return _Moment.apply(_as_dbeta(dbeta, E.device), E, 1)


def reweighted_mean(O: torch.Tensor, dbeta, E: torch.Tensor) -> torch.Tensor:
    """<O>_tau(dbeta), differentiable in O and dbeta."""
    return _Reweighted.apply(O, _as_dbeta(dbeta, E.device), E)


def overlap(dbeta, E: torch.Tensor) -> torch.Tensor:
    """(alpha, alpha') of the weight overlap at dbeta (float64[2], no autograd)."""
    _check_E(E)
    d = _as_dbeta(dbeta, E.device)
    out = torch.empty(2, dtype=torch.float64, device=E.device)
    _check(load_library().pa_overlap(E.data_ptr(), E.numel(), d.data_ptr(), out.data_ptr(), _stream()), "pa_overlap")
    return out
