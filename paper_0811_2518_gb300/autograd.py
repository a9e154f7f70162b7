"""Differentiable GaBP solve: x = A^{-1} b as a torch.autograd.Function.

Forward: one GaBP solve through the C ABI (by default FP32 messages + FP64
refinement).  Backward, for an upstream gradient g = dL/dx:

* lambda = A^{-T} g = A^{-1} g (A is symmetric), a second GaBP solve on the SAME
  handle: the precision messages depend on A only (eq_prec, eq_prec_message), so
  the converged precision state and frozen coefficients of the forward solve are
  reused and only the mean messages run;
* dL/db = lambda;
* dL/dA restricted to A's stored pattern and symmetrised (A stays symmetric):
  -(lambda_i x_j + lambda_j x_i) / 2 for a stored off-diagonal entry (i, j),
  -lambda_i x_i on the diagonal (library kernel ``gabp_grad_values``).

With ``save_x=False`` the forward result is not kept for backward; x is
recomputed by a third solve (the memory-saving mode for large batches).

``solver``: a Solver created once for the sparsity pattern and reused across
calls (a training loop whose parameters are A's values): the forward sets the
new values on it (gabp_set_values) instead of building a handle, and the
backward puts them back first if another forward changed them meanwhile.
"""
from __future__ import annotations

import torch

from . import GABP_OK, GABP_PREC_FP32_REFINE, GaBPError, Solver

__all__ = ["GaBPSolve", "gabp_solve_autograd"]


class GaBPSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, b, rowptr, col, tol, max_iter, precision, save_x, solver=None):
        n = b.shape[0]
        ctx.own = solver is None
        if ctx.own:
            solver = Solver(n, rowptr, col, vals.detach(), precision=precision, reuse_precisions=1)
        else:
            solver.set_values(vals)
            ctx.vals = vals.detach()
            ctx.version = solver.values_version
        x, st, it, rel = solver.solve(b.detach(), tol=tol, max_iter=max_iter)
        if st != GABP_OK:
            if ctx.own:
                solver.close()
            raise GaBPError(st, "GaBPSolve.forward")
        ctx.solver = solver
        ctx.tol, ctx.max_iter, ctx.save_x = tol, max_iter, save_x
        ctx.b = b.detach() if not save_x else None
        ctx.x = x if save_x else None
        ctx.stats = {"forward_rounds": solver.stats()["rounds"], "forward_relres": rel}
        return x.clone()

    @staticmethod
    def backward(ctx, gx):
        solver = ctx.solver
        try:
            if not ctx.own and solver.values_version != ctx.version:
                solver.set_values(ctx.vals)  # another forward used the solver since
            gx = gx.contiguous().to(torch.float64)
            lam, st, it, rel = solver.solve(gx, tol=ctx.tol, max_iter=ctx.max_iter)
            if st != GABP_OK:
                raise GaBPError(st, "GaBPSolve.backward (adjoint solve)")
            x = ctx.x
            if x is None:  # recompute instead of storing
                x, st, it, rel = solver.solve(ctx.b, tol=ctx.tol, max_iter=ctx.max_iter)
                if st != GABP_OK:
                    raise GaBPError(st, "GaBPSolve.backward (recompute x)")
            gvals = solver.grad_values(lam, x) if ctx.needs_input_grad[0] else None
            gb = lam if ctx.needs_input_grad[1] else None
        finally:
            if ctx.own:
                solver.close()
            ctx.solver = None
            ctx.x = None
            ctx.vals = None
        return gvals, gb, None, None, None, None, None, None, None


def gabp_solve_autograd(rowptr, col, vals, b, tol=1e-10, max_iter=5000, precision=GABP_PREC_FP32_REFINE,
                        save_x=True, solver=None):
    """x = A^{-1} b, differentiable in ``vals`` (the full symmetric CSR values,
    diagonal included) and ``b``.  ``rowptr``/``col`` are int32 CUDA tensors,
    ``vals``/``b`` float64 CUDA tensors; ``solver`` an optional Solver of the
    same pattern reused across calls."""
    return GaBPSolve.apply(vals, b, rowptr, col, tol, max_iter, precision, save_x, solver)
