"""Differentiation through the solver: a ``torch.autograd.Function`` over
factor + solve whose backward pass is the adjoint of the linear solve.

For x = A^-1 b and a loss L(x) with upstream gradient g = dL/dx:

    lambda = A^-T g                    (hssmf_solve_T: the transposed ULV and
                                        multifrontal sweeps, GMRES on A^T)
    dL/db     = lambda
    dL/dA_ij  = -sum_c lambda_ic x_jc  on the sparsity pattern
                                        (hssmf_pattern_grad)

Every step runs in the library's kernels; this module only marshals
tensors.  The matrix values are given in the CSR order of the pattern the
solver was analyzed with (natural numbering), float64 on the GPU.

    s = Solver(Options.defaults(...)); s.analyze_grid(dims, rowptr, colind)
    x = sparse_solve(s, values, b)     # values, b: CUDA float64, requires_grad
    loss = ((x - xt) ** 2).sum(); loss.backward()
"""
from __future__ import annotations

import torch


def _colmajor(t):
    """The same values with column-major storage (what the C ABI expects)."""
    if t.dim() == 1:
        return t.contiguous()
    return t.t().contiguous().t()


class SparseSolve(torch.autograd.Function):
    """x = A(values)^-1 b with the solver's factorization; differentiable in
    ``values`` and ``b``."""

    @staticmethod
    def forward(ctx, values, b, solver):
        if values.dtype != torch.float64 or b.dtype != torch.float64 or not values.is_cuda or not b.is_cuda:
            raise TypeError("sparse_solve takes CUDA float64 tensors")
        vals = values.detach().contiguous()
        bc = _colmajor(b.detach())
        solver.factor(vals)
        x = solver.solve(bc)
        ctx.solver = solver
        ctx.factorization = solver.factorizations
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        solver = ctx.solver
        if solver.factorizations != ctx.factorization:
            # the adjoint needs the factorization of the forward pass's A
            raise RuntimeError("sparse_solve: the solver was factored again between forward and backward; "
                               "use one solver per differentiated solve or call backward first")
        (x,) = ctx.saved_tensors
        lam = solver.solve_T(_colmajor(gx.detach()))
        gvals = None
        if ctx.needs_input_grad[0]:
            gvals = torch.empty(solver.nnz, dtype=torch.float64, device=x.device)
            solver.pattern_grad(lam, x, gvals)
        gb = lam if ctx.needs_input_grad[1] else None
        return gvals, gb, None


def sparse_solve(solver, values, b):
    """Differentiable x = A^-1 b (A given by ``values`` on the solver's pattern)."""
    return SparseSolve.apply(values, b, solver)
