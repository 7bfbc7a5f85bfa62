"""Differentiable Laplacian solve: x = A(w)^+ b as a ``torch.autograd.Function``.

Forward: LAMG setup on the current edge weights (cached while the weight
tensor is unchanged) and a LAMG solve.  Backward (adjoint method): with the
same hierarchy solve A lambda = g - mean(g) (``lamg_adjoint``); then

    dL/db    = lambda
    dL/dw_uv = -(lambda_u - lambda_v)(x_u - x_v)

because dA/dw_uv = (e_u - e_v)(e_u - e_v)^T for the graph Laplacian of Eq. (1.1)
and x = A^+ b with b and x in the zero-sum subspace.  Both the solve and the
per-edge gradient run in the CUDA library; this module only lays out the
arguments (the CSR pattern of the edge list and the weight gather into it).
"""
from __future__ import annotations

import weakref

import torch

from . import lamg as _L


class GraphPattern:
    """Sparsity pattern of an undirected graph given by its edge list (u, v),
    u != v, no repeated pair.  Holds the symmetric CSR pattern on the device and,
    for every CSR entry, the index of its edge, so that a weight vector over the
    edges maps to CSR weights by one gather.  With ``gptr`` (host int64 node
    ranges) the graph is a block-diagonal union of independent graphs, set up by
    lamg_setup_graphs and solved per graph."""

    def __init__(self, n: int, eu: torch.Tensor, ev: torch.Tensor, gptr=None, **opts):
        if eu.shape != ev.shape or eu.dim() != 1:
            raise ValueError("eu, ev must be 1-D and of equal length")
        dev = eu.device
        self.n = int(n)
        self.m = int(eu.numel())
        u = eu.to(torch.int64)
        v = ev.to(torch.int64)
        rows = torch.cat([u, v])
        cols = torch.cat([v, u])
        eid = torch.arange(self.m, device=dev, dtype=torch.int64).repeat(2)
        order = torch.argsort(rows * self.n + cols)
        counts = torch.bincount(rows, minlength=self.n)
        self.row_ptr = torch.zeros(self.n + 1, dtype=torch.int64, device=dev)
        self.row_ptr[1:] = torch.cumsum(counts, 0)
        self.col = cols[order].to(torch.int32).contiguous()
        self.entry_edge = eid[order].contiguous()
        self.eu = u.to(torch.int32).contiguous()
        self.ev = v.to(torch.int32).contiguous()
        self.gptr = gptr
        self.opts = opts
        self._solver = None
        self._key = None

    def solver(self, w: torch.Tensor) -> "_L.Solver":
        """The LAMG hierarchy of weights w: rebuilt unless w is the same tensor object,
        unchanged in place since the hierarchy was built."""
        ref = self._key[0]() if self._key is not None else None
        hit = self._solver is not None and ref is w and self._key[1] == w._version
        if not hit:
            # the previous hierarchy is freed when no pending backward holds it
            self._solver = None
            wc = w.detach()[self.entry_edge].contiguous()
            if wc.dtype not in (torch.float32, torch.float64):
                wc = wc.to(torch.float64)
            self._solver = _L.Solver(self.n, self.row_ptr, self.col, wc, gptr=self.gptr, **self.opts)
            self._key = (weakref.ref(w), w._version)
        return self._solver

    def close(self):
        if self._solver is not None:
            self._solver.close()
            self._solver = None


class LaplacianSolve(torch.autograd.Function):
    """x = A(w)^+ b for the graph Laplacian of ``pattern`` with edge weights w.

    w: (m,) FP32 or FP64 CUDA tensor over the pattern's edges (positive).
    b: (n,) FP64 CUDA tensor, zero-sum.
    Returns x: (n,) FP64, zero-mean, ||b - A x|| <= tol ||b||.
    """

    @staticmethod
    def forward(ctx, w, b, pattern: GraphPattern, tol: float = 1e-10, precision: int = _L.LAMG_FP64):
        s = pattern.solver(w)
        x, _ = s.solve(b.detach().contiguous(), tol=tol, precision=precision)
        ctx.solver = s          # the backward reuses this hierarchy
        ctx.pattern = pattern
        ctx.tol = tol
        ctx.precision = precision
        ctx.w_dtype = w.dtype
        ctx.save_for_backward(w, x)
        return x

    @staticmethod
    def backward(ctx, gx):
        w, x = ctx.saved_tensors
        pattern: GraphPattern = ctx.pattern
        s = ctx.solver
        lam = torch.zeros_like(x)
        need_w = ctx.needs_input_grad[0]
        dw = torch.zeros(pattern.m, dtype=torch.float64, device=x.device) if need_w else None
        _L.lamg_adjoint(s.h, x.contiguous(), gx.detach().to(torch.float64).contiguous(), lam,
                        pattern.eu if need_w else None, pattern.ev if need_w else None, dw,
                        tol=ctx.tol, precision=ctx.precision)
        gw = dw.to(ctx.w_dtype) if need_w else None
        gb = lam if ctx.needs_input_grad[1] else None
        return gw, gb, None, None, None


def laplacian_solve(w, b, pattern: GraphPattern, tol: float = 1e-10, precision: int = _L.LAMG_FP64):
    return LaplacianSolve.apply(w, b, pattern, tol, precision)
