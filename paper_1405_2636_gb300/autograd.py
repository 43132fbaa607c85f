"""Differentiable sparse SPD solve and log-determinant (torch.autograd).

``SparseSPD`` wraps one analysed pattern.  ``solve(values, b)`` and
``logdet(values)`` are autograd functions of the CSC values (each stored
entry independent) and of b.  Their backward passes are hand-written
adjoints that reuse the device-resident FP64 factor:

  x = A^{-1} b:     lambda = A^{-T} g (one more solve with the same factor),
                    dL/db = lambda,  dL/dA = -lambda x^T on A's pattern;
  log det A:        dL/dA = g (A^{-1})^T on A's pattern, from the selected
                    inverse computed by the library's supernodal kernel.

Every step runs in libspx's kernels; this module only moves tensors.  The
factor is refreshed whenever it was made from another tensor or the
tensor was modified in place since, so a backward pass after such a change
refactorizes first.
"""
from __future__ import annotations

import weakref

import torch

from . import spx


class SparseSPD:
    """Analysis of one SPD pattern (Cholesky), shared by solve and logdet."""

    def __init__(self, colptr, rowind, **analyze_opts):
        self.handle = spx.analyze(colptr, rowind, "llt", **analyze_opts)
        self.n = self.handle.n
        self.nnz = self.handle.nnz
        self._ref = None
        self._version = -1

    def _factor(self, values: torch.Tensor):
        """Factorize unless the factor already belongs to this very tensor
        (same object, not modified in place since)."""
        if not (values.is_cuda and values.dtype == torch.float64 and values.numel() == self.nnz):
            raise ValueError("values must be a CUDA float64 tensor with one entry per stored entry")
        if self._ref is None or self._ref() is not values or self._version != values._version:
            self.handle.factorize(values.detach().contiguous(), "fp64")
            self._ref = weakref.ref(values)
            self._version = values._version

    def solve(self, values: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
        return _Solve.apply(values, b, self)

    def logdet(self, values: torch.Tensor) -> torch.Tensor:
        return _Logdet.apply(values, self)

    def free(self):
        self.handle.free()


def _colmajor(t: torch.Tensor) -> torch.Tensor:
    return t.contiguous() if t.dim() == 1 else t.t().contiguous().t()


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, values, b, op: SparseSPD):
        op._factor(values)
        bb = _colmajor(b.detach())
        x, _ = op.handle.solve(bb)
        ctx.op = op
        ctx.save_for_backward(values, x)
        return x

    @staticmethod
    def backward(ctx, gx):
        values, x = ctx.saved_tensors
        op = ctx.op
        op._factor(values)
        lam, _ = op.handle.solve(_colmajor(gx))            # A^{-T} g, A symmetric
        gvals = op.handle.solve_grad(lam, x) if ctx.needs_input_grad[0] else None
        return gvals, (lam if ctx.needs_input_grad[1] else None), None


class _Logdet(torch.autograd.Function):
    @staticmethod
    def forward(ctx, values, op: SparseSPD):
        op._factor(values)
        ctx.op = op
        ctx.save_for_backward(values)
        return torch.tensor(op.handle.logdet(), dtype=torch.float64, device=values.device)

    @staticmethod
    def backward(ctx, g):
        (values,) = ctx.saved_tensors
        op = ctx.op
        op._factor(values)
        grad = torch.empty(op.nnz, dtype=torch.float64, device=values.device)
        op.handle.logdet_grad(grad)
        return grad * g, None
