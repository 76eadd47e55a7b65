"""torch.autograd.Function over hp_trace_inv_grad.

forward(mu) returns Re T_s (the probing estimate of Tr(A^-1) after s
probes) for the operator with per-site mass field mu; backward returns
grad_output * dT_s/dmu(x).  The derivative is computed by the library in the
same pass as the estimate, from the forward solutions (the Laplacian is
symmetric and the Wilson matrix gamma_5-hermitian, so no adjoint solve is
needed), and kept for backward.
"""
from __future__ import annotations

import torch

from .hprobe import OP_LAPLACIAN, OP_WILSON, Context


class TraceInvFunction(torch.autograd.Function):
    @staticmethod
    def forward(fctx, mass_field, hctx: Context, dims, kind, mass, kappa, links, s_max, tol, opts):
        mf = mass_field.detach().to(torch.float64).contiguous()
        grad = torch.empty_like(mf)
        op = Context.make_operator(kind, mass, kappa, links, mf)
        T, dTdm, stats = hctx.trace_inv_grad(op, dims, s_max, tol, opts, grad)
        fctx.save_for_backward(grad)
        fctx.stats = stats
        return torch.tensor(T[-1].real, dtype=torch.float64, device=mass_field.device)

    @staticmethod
    def backward(fctx, grad_output):
        (grad,) = fctx.saved_tensors
        return (grad_output * grad,) + (None,) * 9


def trace_inv_estimate(mass_field: torch.Tensor, hctx: Context, dims, s_max: int, tol: float, opts,
                       kind: int = OP_WILSON, mass: float = 0.0, kappa: float = 0.0, links=None) -> torch.Tensor:
    """Differentiable Re T_{s_max} as a function of the per-site mass field."""
    return TraceInvFunction.apply(mass_field, hctx, dims, kind, mass, kappa, links, s_max, tol, opts)


__all__ = ["TraceInvFunction", "trace_inv_estimate", "OP_LAPLACIAN", "OP_WILSON"]
