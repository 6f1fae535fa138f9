"""The differentiable solve: torch.autograd Functions around the library.

``SparseSolve`` maps (stored values of A, b) to the solution x of A x = b by
the double-precision CG of Section III (``gbcg_solve``).  Its backward
solves the adjoint system A lambda = dL/dx with the same handle (A is
symmetric), returns dL/db = lambda and dL/d(values) from the sampled outer
product kernel (``gbcg_grad_values``).  ``Assembly`` maps finite-element
coefficients to the stored values (``gbcg_assemble``); its backward is the
chain rule through the element map (``gbcg_element_grad``).  Composed, they
give dL/dcoef per element.  Every step runs in the library's kernels; torch
only holds the tensors and the graph.
"""
from __future__ import annotations

import numpy as np


def _torch():
    import torch
    return torch


class SparseSolve:
    """x = A(values)^-1 b, differentiable in values and b.

    ``fmt``, ``ptr``, ``idx``, ``val``: the pattern and initial values as for
    ``Matrix`` (numpy arrays, 0-based).  ``tol`` is the relative residual of
    the forward solve, ``adjoint_tol`` that of the adjoint solve (default:
    tol).  ``maxit`` <= 0 means n; ``fixed_iterations`` > 0 runs exactly that
    many iterations in both solves instead (a smooth map of the inputs, for
    finite-difference checks).
    """

    def __init__(self, fmt, ptr, idx, val, tol: float = 1e-12, adjoint_tol: float | None = None, maxit: int = 0,
                 fixed_iterations: int = 0, device=None):
        from . import Matrix

        torch = _torch()
        self.fmt = fmt
        self.device = torch.device("cuda") if device is None else torch.device(device)
        self.matrix = Matrix(fmt, ptr, idx, val)
        self.ptr = torch.from_numpy(np.ascontiguousarray(ptr, dtype=np.int32)).to(self.device)
        self.idx = torch.from_numpy(np.ascontiguousarray(idx, dtype=np.int32)).to(self.device)
        self.nnz = int(self.idx.numel())
        self.n = int(self.ptr.numel()) - 1
        self.tol = float(tol)
        self.adjoint_tol = float(tol if adjoint_tol is None else adjoint_tol)
        self.maxit = int(maxit)
        self.fixed_iterations = int(fixed_iterations)
        self.last_info = None

    def close(self):
        self.matrix.close()

    def _solve(self, vals, rhs, tol):
        self.matrix.update_values(vals)
        if self.fixed_iterations > 0:
            x, info = self.matrix.solve(rhs, tol=0.0, maxit=self.fixed_iterations, precision="fp64",
                                        max_restarts=0, raise_on_error=False)
            if info.status not in ("OK", "MAXIT"):
                raise RuntimeError(f"solve failed: {info}")
        else:
            x, info = self.matrix.solve(rhs, tol=tol, maxit=self.maxit, precision="fp64")
            if info.status != "OK":
                raise RuntimeError(f"solve did not converge: {info}")
        return x, info

    def __call__(self, vals, b):
        return _SolveFn.apply(vals, b, self)


class Assembly:
    """Stored values = sum_e coef_e Kh_e from an element map (see
    ``femgen.element_map`` / ``femgen.assembly_map``), differentiable in coef."""

    def __init__(self, pos, w, tptr, telem, tw, device=None):
        torch = _torch()
        dev = torch.device("cuda") if device is None else torch.device(device)
        self.pos = torch.from_numpy(np.ascontiguousarray(pos, dtype=np.int32)).to(dev)
        self.w = torch.from_numpy(np.ascontiguousarray(w, dtype=np.float64)).to(dev)
        self.tptr = torch.from_numpy(np.ascontiguousarray(tptr, dtype=np.int64)).to(dev)
        self.telem = torch.from_numpy(np.ascontiguousarray(telem, dtype=np.int32)).to(dev)
        self.tw = torch.from_numpy(np.ascontiguousarray(tw, dtype=np.float64)).to(dev)

    def __call__(self, coef):
        return _AssembleFn.apply(coef, self)


def _make_functions():
    torch = _torch()
    from . import assemble, element_grad, grad_values

    class SolveFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, vals, b, S):
            vals_c = vals.detach().to(torch.float64).contiguous()
            x, info = S._solve(vals_c, b.detach().to(torch.float64).contiguous(), S.tol)
            S.last_info = info
            ctx.S = S
            ctx.save_for_backward(vals_c, x)
            return x

        @staticmethod
        def backward(ctx, gx):
            S = ctx.S
            vals_c, x = ctx.saved_tensors
            lam, info = S._solve(vals_c, gx.detach().to(torch.float64).contiguous(), S.adjoint_tol)
            S.last_adjoint_info = info
            gvals = grad_values(S.fmt, S.ptr, S.idx, lam, x) if ctx.needs_input_grad[0] else None
            gb = lam if ctx.needs_input_grad[1] else None
            return gvals, gb, None

    class AssembleFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, coef, M):
            c = coef.detach().to(torch.float64).contiguous()
            ctx.M = M
            return assemble(M.tptr, M.telem, M.tw, c)

        @staticmethod
        def backward(ctx, gvals):
            M = ctx.M
            return element_grad(M.pos, M.w, gvals.detach().to(torch.float64).contiguous()), None

    return SolveFn, AssembleFn


class _Lazy:
    def __init__(self, k):
        self.k = k

    def apply(self, *a):
        global _FNS
        if _FNS is None:
            _FNS = _make_functions()
        return _FNS[self.k].apply(*a)


_FNS = None
_SolveFn = _Lazy(0)
_AssembleFn = _Lazy(1)
