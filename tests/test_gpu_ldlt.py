"""LDL^T with static pivoting (updates C = C - L D L^T through a stored D L^T
operand) against the oracle: factors and pivots on the oracle's pattern,
inertia, solves; the tensor-core and FP32 modes with refinement."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_1405_2636_gb300 import inputs, spx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    import __graft_entry__

    __graft_entry__.build()
    assert _t.cuda.is_available()
    return _t


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [
    ("quasidef_6x5x4", lambda: inputs.quasi_definite_3d(6, 5, 4, 1), dict(ordering=1, grid=(6, 5, 4), dof=2)),
    ("quasidef_12x11x10_w24", lambda: inputs.quasi_definite_3d(12, 11, 10, 2),
     dict(ordering=1, grid=(12, 11, 10), dof=2, max_width=24)),
    ("quasidef_16x15x14_w64", lambda: inputs.quasi_definite_3d(16, 15, 14, 3),
     dict(ordering=1, grid=(16, 15, 14), dof=2, max_width=64)),
    ("diffusion_spd_14x13x12", lambda: inputs.diffusion_3d(14, 13, 12, 4), dict(ordering=1, grid=(14, 13, 12))),
]


@pytest.mark.parametrize("name,maker,opts", CASES, ids=[c[0] for c in CASES])
def test_ldlt_fp64_matches_oracle(torch, name, maker, opts):
    A = maker()
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "ldlt", **opts)
    h.factorize(vals, "fp64")
    F = oracle.ldlt(A, h.perm())
    Lx = h.factor_on_pattern(F.sym.Lp, F.sym.Li)
    assert _rel(Lx, F.Lx) <= 1e-12
    d_gpu, d_ora = Lx[F.sym.Lp[:-1]], F.Lx[F.sym.Lp[:-1]]
    assert np.max(np.abs(d_gpu - d_ora) / np.abs(d_ora)) <= 1e-12
    info = h.info()
    assert info["npivot_repl"] == F.nrepl == 0
    assert info["npivot_neg"] == oracle.inertia(F)[1]
    B = inputs.rhs(A.shape[0], 3, 9)
    X, sinfo = h.solve(B)
    assert oracle.backward_error(A, X, B) <= 1e-13
    h.free()


def test_ldlt_inertia_quasi_definite_full(torch):
    A = inputs.quasi_definite_3d(10, 9, 8, 5)
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "ldlt", ordering=1, grid=(10, 9, 8), dof=2)
    h.factorize(vals, "fp64")
    assert h.info()["npivot_neg"] == A.shape[0] // 2
    h.free()


def test_ldlt_static_pivot_hand_example(torch):
    A = sp.csc_matrix(np.array([[0.0, 1.0], [1.0, 1.0]]))
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "ldlt", ordering=4)
    h.factorize(vals, "fp64")
    F = oracle.ldlt(A, h.perm())
    Lx = h.factor_on_pattern(F.sym.Lp, F.sym.Li)
    assert h.info()["npivot_repl"] == 1 == F.nrepl
    assert np.array_equal(Lx, F.Lx)


def test_ldlt_zero_pivot_is_an_error_without_static_pivoting(torch):
    A = sp.csc_matrix(np.array([[0.0, 1.0], [1.0, 1.0]]))
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "ldlt", ordering=4, pivot_tau=0.0)
    with pytest.raises(spx.SpxError) as e:
        h.factorize(vals, "fp64")
    assert e.value.status == spx.SPX_ERR_ZERO_PIVOT and h.info()["bad_col"] == 0


@pytest.mark.parametrize("prec,bound", [("fp32", 1e-4), ("tf32", 2e-2), ("bf16", 1e-1)])
def test_ldlt_mixed_precision_and_refinement(torch, prec, bound):
    A = inputs.quasi_definite_3d(16, 15, 14, 6)
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "ldlt", ordering=1, grid=(16, 15, 14), dof=2, max_width=64)
    F = oracle.ldlt(A, h.perm())
    h.factorize(vals, prec)
    Lx = h.factor_on_pattern(F.sym.Lp, F.sym.Li)
    assert _rel(Lx, F.Lx) <= bound
    assert np.max(np.abs(Lx - F.Lx)) <= bound * np.max(np.abs(F.Lx))   # entry by entry
    B = inputs.rhs(A.shape[0], 4, 10)
    X, sinfo = h.solve(B, refine=spx.default_refine(tol=1e-12))
    assert sinfo["converged"]
    assert oracle.backward_error(A, X, B) <= 1e-12
    h.free()
