"""Differentiable IBDL solves and probe values: ``torch.autograd.Function``s around the C ABI.

``Boundary(X, n, Δs, …)`` builds the geometry once from CUDA float64 tensors. Its ``solve`` and
``probe`` return tensors that autograd differentiates with respect to U_b, X, n and Δs:

  solve   forward  Q = A⁻¹U_b                                   (ibdl_solve)
          backward λ = A⁻ᵀ ∂J/∂Q (ibdl_solve_transpose); ∂J/∂U_b = λ and
                   ∂J/∂(X, n, Δs) = −∂(λᵀ A Q)/∂(X, n, Δs)      (ibdl_solve_vjp)
  probe   forward  U = E Q, the grid solution at the probe points (ibdl_probe_evaluate)
          backward ∂J/∂Q = Eᵀ ∂J/∂U and ∂J/∂(X, n, Δs) = ∂(νᵀ E Q)/∂(…) (ibdl_probe_vjp)

Every step runs in libibdl.so; PyTorch supplies tensors, streams and the autograd graph. The
scalar operator of Sec. 5.3.2 and the Stokes operator of Sec. 6.3.3, analytic dipole spread. The
normals and weights are independent inputs, so a caller that computes them from X in torch gets
their chain rule from autograd. The probes are fixed (no gradient with respect to them).

The Krylov basis is not kept between forward and backward: the backward pass is a fresh GMRES
solve with the transposed operator, so the memory held across the pair is the geometry (point
tables, spectra and two to five FP64 grid fields) and Q.
"""
from __future__ import annotations

import torch

from .ibdl import Geometry


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Ub, X, normals, weights, geom: Geometry, solve_kw: dict):
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


class _Probe(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Q, X, normals, weights, geom: Geometry, P):
        Qf = Q.detach().contiguous().reshape(-1)
        U = geom.probe_evaluate(P, Qf)
        ctx.geom, ctx.P, ctx.qshape = geom, P, Q.shape
        ctx.save_for_backward(Qf)
        return U

    @staticmethod
    def backward(ctx, gU):
        (Q,) = ctx.saved_tensors
        want = (ctx.needs_input_grad[0],) + tuple(ctx.needs_input_grad[1:4])
        if not any(want):
            return None, None, None, None, None, None
        dQ, dX, dn, dw = ctx.geom.probe_vjp(ctx.P, Q, gU.detach().contiguous(), want=want)
        if dQ is not None:
            dQ = dQ.view(ctx.qshape)
        return dQ, dX, dn, dw, None, None


class Boundary:
    """An immersed boundary (X [d][M], n [d][M], Δs [M], CUDA float64 tensors) on an n^d periodic
    grid, with differentiable ``solve`` and ``probe``."""

    def __init__(self, X, normals, weights, n: int, *, box: float = 1.0, origin=(0.0, 0.0, 0.0),
                 pde: str = "scalar", lam: float = 0.0, mu: float = 1.0, delta: str = "cos",
                 symbol: str = "spectral"):
        self.X, self.normals, self.weights = X, normals, weights
        self.geom = Geometry(X, normals, weights, n, box=box, origin=origin, pde=pde, lam=lam, mu=mu, delta=delta,
                             dipole="analytic", symbol=symbol)

    def solve(self, Ub, *, rtol: float = 1e-10, precision: str = "fp64", restart: int = 50, maxit: int = 200,
              inner_rtol: float = 1e-5, max_refine: int = 6):
        """Q = A⁻¹U_b with the shape of U_b ([M] scalar, [d][M] or [d·M] Stokes)."""
        kw = dict(rtol=rtol, precision=precision, restart=restart, maxit=maxit, inner_rtol=inner_rtol,
                  max_refine=max_refine)
        return _Solve.apply(Ub, self.X, self.normals, self.weights, self.geom, kw)

    def probe(self, Q, P):
        """Grid solution of Q at the probe points P [2][n_p]: shape [c][n_p]."""
        return _Probe.apply(Q, self.X, self.normals, self.weights, self.geom, P)

    def close(self):
        self.geom.close()


def solve(Ub, X, normals, weights, n: int, *, box: float = 1.0, origin=(0.0, 0.0, 0.0), pde: str = "scalar",
          lam: float = 0.0, mu: float = 1.0, delta: str = "cos", symbol: str = "spectral", **solve_kw):
    """Differentiable solve on a boundary built for this call; returns Q with the shape of U_b."""
    b = Boundary(X, normals, weights, n, box=box, origin=origin, pde=pde, lam=lam, mu=mu, delta=delta,
                 symbol=symbol)
    return b.solve(Ub, **solve_kw)
