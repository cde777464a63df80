"""Differentiable IBDL solve: a ``torch.autograd.Function`` around the C ABI.

Forward: build the geometry from (X, n, Δs) and solve A Q = U_b (``ibdl_solve``). Backward, for
an upstream gradient G = ∂J/∂Q: one transposed solve λ = A⁻ᵀ G (``ibdl_solve_transpose``), then
∂J/∂U_b = λ and ∂J/∂(X, n, Δs) = −∂(λᵀ A Q)/∂(X, n, Δs) (``ibdl_solve_vjp``). Every step runs in
libibdl.so; PyTorch supplies the tensors and the autograd graph. Scalar PDE with the analytic
dipole spread (the operator of Sec. 5.3.2). The normals and weights are independent inputs, so a
caller that computes them from X in torch gets their chain rule from autograd.

The Krylov basis is not kept between forward and backward: the backward pass is a fresh GMRES
solve with the transposed operator, so the memory held across the pair is the geometry (point
tables and spectra) and Q.
"""
from __future__ import annotations

import torch

from .ibdl import Geometry

class IbdlSolve(torch.autograd.Function):
    """Q = A(X, n, Δs)⁻¹ U_b; inputs are CUDA float64 tensors U_b [M], X [d][M], n [d][M], Δs [M]."""

    @staticmethod
    def forward(ctx, Ub, X, normals, weights, geom_kw: dict, solve_kw: dict):
        geom = Geometry(X, normals, weights, pde="scalar", dipole="analytic", **geom_kw)
        Q, info, _ = geom.solve(Ub.detach().contiguous().reshape(-1), **solve_kw)
        ctx.geom, ctx.solve_kw, ctx.info = geom, solve_kw, info
        ctx.save_for_backward(Q)
        return Q.view_as(Ub)

    @staticmethod
    def backward(ctx, gQ):
        (Q,) = ctx.saved_tensors
        geom = ctx.geom
        lam, info, _ = geom.solve_transpose(gQ.detach().contiguous().reshape(-1), **ctx.solve_kw)
        ctx.backward_info = info
        want = ctx.needs_input_grad[1:4]
        dX = dn = dw = None
        if any(want):
            dX, dn, dw = geom.solve_vjp(Q, lam, want=want)
        dUb = lam.view_as(gQ) if ctx.needs_input_grad[0] else None
        return dUb, dX, dn, dw, None, None


def solve(Ub, X, normals, weights, n: int, *, box: float = 1.0, origin=(0.0, 0.0, 0.0), lam: float = 0.0,
          delta: str = "cos", symbol: str = "spectral", rtol: float = 1e-10, precision: str = "fp64",
          restart: int = 50, maxit: int = 200, inner_rtol: float = 1e-5, max_refine: int = 6):
    """Differentiable solve of the scalar IBDL system; returns Q with the shape of U_b."""
    geom_kw = dict(n=n, box=box, origin=origin, lam=lam, delta=delta, symbol=symbol)
    solve_kw = dict(rtol=rtol, precision=precision, restart=restart, maxit=maxit, inner_rtol=inner_rtol,
                    max_refine=max_refine)
    return IbdlSolve.apply(Ub, X, normals, weights, geom_kw, solve_kw)
