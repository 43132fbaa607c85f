"""Solves with more right-hand sides than one pass of the sweep kernels
holds (16 columns per pass): 20 columns take a pass of 16 and a pass of 4.

Checked for Cholesky, LU and LDL^T factors in FP64, Cholesky and LDL^T in
refined TF32, with host and device buffers: the normwise backward error of
every column on the host (the oracle's formula), the FP64 solutions against
the oracle's solve on the same ordering, and the 20-column solve against the
same columns solved in groups that each fit one pass.  The two FP64 solves
differ only in the order of their atomic sums; with 2-norm condition numbers
of at most 754 for these matrices (computed densely) their solutions agree
to far better than the 1e-11 the test asks.
"""
import numpy as np
import pytest

import oracle
from paper_1405_2636_gb300 import inputs, spx

pytestmark = pytest.mark.gpu

NRHS = 20


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    import __graft_entry__

    __graft_entry__.build()
    assert _t.cuda.is_available()
    return _t


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _cases():
    qd = inputs.quasi_definite_3d(8, 7, 6, 3)
    cd, _ = inputs.convection_diffusion_2d(30, 5)
    return [
        ("llt", inputs.diffusion_3d(12, 11, 10, 3), dict(ordering=1, grid=(12, 11, 10), max_width=24)),
        ("lu", cd, dict(ordering=1, grid=(30, 30, 1), max_width=16)),
        ("ldlt", qd, dict(ordering=1, grid=(8, 7, 6), dof=2, max_width=24)),
    ]


@pytest.mark.parametrize("method,A,opts", _cases(), ids=["llt", "lu", "ldlt"])
def test_fp64_solve_with_two_passes(torch, method, A, opts):
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, method, **opts)
    h.factorize(vals, "fp64")
    B = inputs.rhs(A.shape[0], NRHS, 17)
    X, info = h.solve(B)
    assert X.shape == (A.shape[0], NRHS)
    assert oracle.backward_error(A, X, B) <= 1e-13
    # the oracle's solve on the same ordering
    F = {"llt": oracle.cholesky, "lu": oracle.lu, "ldlt": oracle.ldlt}[method](A, h.perm())
    Xo = oracle.solve(F, B)
    assert _rel(X, Xo) <= 1e-10
    # the same columns in groups that each fit one pass
    X16, _ = h.solve(np.asfortranarray(B[:, :16]))
    X4, _ = h.solve(np.asfortranarray(B[:, 16:]))
    assert _rel(X[:, :16], X16) <= 1e-11 and _rel(X[:, 16:], X4) <= 1e-11
    h.free()


@pytest.mark.parametrize("method,A,opts", [c for c in _cases() if c[0] != "lu"], ids=["llt", "ldlt"])
def test_refined_tf32_solve_with_two_passes(torch, method, A, opts):
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, method, **opts)
    h.factorize(vals, "tf32")
    B = inputs.rhs(A.shape[0], NRHS, 19)
    X, info = h.solve(B, refine=spx.default_refine(tol=1e-12))
    assert info["converged"], info
    assert oracle.backward_error(A, X, B) <= 1e-12
    h.free()


def test_device_buffers_with_two_passes(torch):
    A = inputs.diffusion_3d(12, 11, 10, 3)
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "llt", ordering=1, grid=(12, 11, 10), max_width=24)
    h.factorize(torch.from_numpy(vals).cuda(), "tf32")
    B = inputs.rhs(A.shape[0], NRHS, 23)
    Bd = torch.from_numpy(np.ascontiguousarray(B.T)).cuda().t()          # column-major n x 20
    Xd, info = h.solve(Bd, refine=spx.default_refine(tol=1e-12))
    assert info["converged"], info
    assert oracle.backward_error(A, Xd.cpu().numpy(), B) <= 1e-12
    h.free()
