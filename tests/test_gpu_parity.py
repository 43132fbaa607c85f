"""Parity of the CUDA factorization and solves with the CPU oracle.

Every case runs through the C ABI (spx_analyze / spx_factorize / spx_solve /
spx_get_factor) and compares, element by element on the oracle's exact
pattern and on the same ordering, the GPU factor with the oracle's.

Tolerances:
  * FP64 factor: relative Frobenius error <= 1e-12 and every entry within
    1e-12 * max|L| (the target accuracy of the FP64 path; the two sides differ
    only in the order of the rounded sums);
  * FP64 solve: normwise backward error <= 1e-13;
  * single-precision factor (mixed modes): relative error <= 1e-4 against the
    FP64 oracle (FP32 storage, unit roundoff 6e-8, amplified by the growth
    of the Schur complements), and backward error <= 1e-12 after refinement.
"""
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
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


LLT_CASES = [
    ("laplace2d_31x31", lambda: inputs.laplacian_2d(31, 31), dict(ordering=1, grid=(31, 31, 1))),
    ("diffusion_12^3_w16", lambda: inputs.diffusion_3d(12, 12, 12, 5),
     dict(ordering=1, grid=(12, 12, 12), max_width=16)),
    ("diffusion_17x13x11_w40", lambda: inputs.diffusion_3d(17, 13, 11, 6),
     dict(ordering=1, grid=(17, 13, 11), max_width=40)),
    ("diffusion_20^3_w128", lambda: inputs.diffusion_3d(20, 20, 20, 8),
     dict(ordering=1, grid=(20, 20, 20), max_width=128)),
    ("elasticity_6x5x4x3_w24", lambda: inputs.elasticity_27pt(6, 5, 4, 7),
     dict(ordering=1, grid=(6, 5, 4), dof=3, max_width=24)),
    ("elasticity_7^3x3_w160", lambda: inputs.elasticity_27pt(7, 7, 7, 9),
     dict(ordering=1, grid=(7, 7, 7), dof=3, max_width=160)),
    ("random_graph_2000_w32", lambda: inputs.random_spd_graph(2000, 6.0, 9),
     dict(ordering=2, max_width=32)),
    ("single_unknown", lambda: sp.csc_matrix(np.array([[4.0]])), dict(ordering=4)),
    ("tridiagonal_natural_w7", lambda: sp.diags([-np.ones(299), 2.5 * np.ones(300), -np.ones(299)],
                                                [-1, 0, 1]).tocsc(), dict(ordering=4, max_width=7)),
    ("no_amalgamation", lambda: inputs.diffusion_3d(9, 9, 9, 2),
     dict(ordering=1, grid=(9, 9, 9), amalg_ratio=0.0, max_width=5)),
]


@pytest.mark.parametrize("name,maker,opts", LLT_CASES, ids=[c[0] for c in LLT_CASES])
def test_cholesky_fp64_matches_oracle(torch, name, maker, opts):
    A = maker()
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "llt", **opts)
    F = oracle.cholesky(A, h.perm())
    h.factorize(torch.from_numpy(vals).cuda(), "fp64")
    Lx = h.factor_on_pattern(F.sym.Lp, F.sym.Li)
    assert _rel(Lx, F.Lx) <= 1e-12
    assert np.max(np.abs(Lx - F.Lx)) <= 1e-12 * np.max(np.abs(F.Lx))
    # the pivots (square roots taken on the GPU by Newton steps) entry by entry
    d_gpu, d_ora = Lx[F.sym.Lp[:-1]], F.Lx[F.sym.Lp[:-1]]
    assert np.max(np.abs(d_gpu - d_ora) / d_ora) <= 1e-13
    n = A.shape[0]
    B = inputs.rhs(n, 3, 11)
    X, info = h.solve(B)
    assert oracle.backward_error(A, X, B) <= 1e-13
    assert info["backward_error"] <= 1e-13
    Xo = oracle.solve(F, B)
    assert _rel(X, Xo) <= 1e-10
    h.free()


def test_cholesky_device_rhs_and_values(torch):
    """Device-resident values, right-hand sides and solution (on_device=1)."""
    A = inputs.diffusion_3d(10, 11, 12, 3)
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "llt", ordering=1, grid=(10, 11, 12))
    h.factorize(torch.from_numpy(vals).cuda(), "fp64")
    B = inputs.rhs(A.shape[0], 5, 4)
    Bd = torch.from_numpy(np.ascontiguousarray(B.T)).cuda().t()   # column-major view
    Xd, info = h.solve(Bd)
    X = Xd.cpu().numpy()
    assert oracle.backward_error(A, X, B) <= 1e-13
    # a second factorization with new values on the same pattern
    A2 = inputs.diffusion_3d(10, 11, 12, 4)
    _, _, vals2 = inputs.csc_arrays(A2)
    h.factorize(vals2, "fp64")
    X2, _ = h.solve(B)
    assert oracle.backward_error(A2, X2, B) <= 1e-13


def test_lower_only_values(torch):
    A = inputs.laplacian_2d(21, 17)
    Lo = sp.tril(A).tocsc()
    cp, ri, vals = inputs.csc_arrays(Lo)
    h = spx.analyze(cp, ri, "llt", ordering=1, grid=(21, 17, 1), lower_only=1)
    F = oracle.cholesky(A, h.perm())
    h.factorize(vals, "fp64")
    Lx = h.factor_on_pattern(F.sym.Lp, F.sym.Li)
    assert _rel(Lx, F.Lx) <= 1e-12
    b = inputs.rhs(A.shape[0], 1, 2)
    x, _ = h.solve(b)
    assert oracle.backward_error(A, x, b) <= 1e-13


def test_not_positive_definite_reports_oracle_column(torch):
    A = inputs.laplacian_2d(15, 15).tolil()
    A[100, 100] = -1.0
    A = A.tocsc()
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "llt", ordering=1, grid=(15, 15, 1))
    with pytest.raises(oracle.NotPositiveDefinite) as e:
        oracle.cholesky(A, h.perm())
    with pytest.raises(spx.SpxError) as g:
        h.factorize(vals, "fp64")
    assert g.value.status == spx.SPX_ERR_NOT_SPD
    assert h.info()["bad_col"] == e.value.col


LU_CASES = [
    ("convdiff_31", lambda: inputs.convection_diffusion_2d(31, 1)[0], dict(ordering=1, grid=(31, 31, 1))),
    ("convdiff_47_w24", lambda: inputs.convection_diffusion_2d(47, 2)[0],
     dict(ordering=1, grid=(47, 47, 1), max_width=24)),
    ("convdiff_80_w160", lambda: inputs.convection_diffusion_2d(80, 3)[0],
     dict(ordering=1, grid=(80, 80, 1), max_width=160)),
]


@pytest.mark.parametrize("name,maker,opts", LU_CASES, ids=[c[0] for c in LU_CASES])
def test_lu_fp64_matches_oracle(torch, name, maker, opts):
    A = maker()
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "lu", **opts)
    F = oracle.lu(A, h.perm())
    h.factorize(vals, "fp64")
    Lx, Ut = h.factor_on_pattern(F.sym.Lp, F.sym.Li, lu=True)
    assert _rel(Lx, F.Lx) <= 1e-12
    assert _rel(Ut, F.Ut) <= 1e-12
    assert h.info()["npivot_repl"] == F.nrepl == 0
    B = inputs.rhs(A.shape[0], 2, 5)
    X, _ = h.solve(B)
    assert oracle.backward_error(A, X, B) <= 1e-13


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16"])
@pytest.mark.parametrize("name,maker,opts", LU_CASES[:2], ids=[c[0] for c in LU_CASES[:2]])
def test_lu_single_precision_factor_and_refinement(torch, name, maker, opts, prec):
    """The single-system LU with a single-precision factor (the panel
    updates run on the CUDA cores in FP32 for every single-precision mode of
    LU): L and U against the FP64 oracle, relative and entry by entry, then
    FP64 refinement to backward error 1e-12."""
    A = maker()
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "lu", **opts)
    F = oracle.lu(A, h.perm())
    h.factorize(vals, prec)
    Lx, Ut = h.factor_on_pattern(F.sym.Lp, F.sym.Li, lu=True)
    for got, ref in ((Lx, F.Lx), (Ut, F.Ut)):
        assert _rel(got, ref) <= 1e-4
        assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))
    assert h.info()["npivot_repl"] == 0
    B = inputs.rhs(A.shape[0], 3, 8)
    X, info = h.solve(B, refine=spx.default_refine(tol=1e-12))
    assert info["converged"], info
    assert oracle.backward_error(A, X, B) <= 1e-12
    h.free()


def test_lu_static_pivot_hand_example(torch):
    """[[0, 1], [1, 1]]: the zero pivot becomes tau = 2^-25 (Sec. III static
    pivoting, threshold sqrt(eps) ||A||_inf); L(1,0) = 2^25, U(1,1) = 1 - 2^25."""
    A = sp.csc_matrix(np.array([[0.0, 1.0], [1.0, 1.0]]))
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "lu", ordering=4)
    h.factorize(vals, "fp64")
    F = oracle.lu(A, h.perm())
    Lx, Ut = h.factor_on_pattern(F.sym.Lp, F.sym.Li, lu=True)
    assert h.info()["npivot_repl"] == 1
    assert np.array_equal(Lx, F.Lx) and np.array_equal(Ut, F.Ut)
    assert Ut[0] == 2.0 ** -25 and Lx[1] == 2.0 ** 25


def test_lu_zero_pivot_is_an_error_without_static_pivoting(torch):
    A = sp.csc_matrix(np.array([[0.0, 1.0], [1.0, 1.0]]))
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "lu", ordering=4, pivot_tau=0.0)
    with pytest.raises(spx.SpxError) as e:
        h.factorize(vals, "fp64")
    assert e.value.status == spx.SPX_ERR_ZERO_PIVOT and h.info()["bad_col"] == 0


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16"])
def test_mixed_precision_factor_and_refinement(torch, prec):
    A = inputs.diffusion_3d(16, 15, 14, 12)
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "llt", ordering=1, grid=(16, 15, 14), max_width=64)
    F = oracle.cholesky(A, h.perm())
    h.factorize(vals, prec)
    Lx = h.factor_on_pattern(F.sym.Lp, F.sym.Li)
    err = _rel(Lx, F.Lx)
    bound = {"fp32": 1e-4, "tf32": 2e-2, "bf16": 1e-1}[prec]
    assert err <= bound
    # entry by entry as well: no entry may be off by more than the bound
    # times the largest entry (a dropped or misplaced update would be)
    assert np.max(np.abs(Lx - F.Lx)) <= bound * np.max(np.abs(F.Lx))
    B = inputs.rhs(A.shape[0], 4, 3)
    X, info = h.solve(B, refine=spx.default_refine(tol=1e-12))
    assert info["converged"], info
    assert oracle.backward_error(A, X, B) <= 1e-12


def test_update_kernel_on_the_papers_synthetic_panels(torch):
    """Sec. V-B kernel study: C = C - A B^T with B the first rows of A, C a
    panel twice as tall as A cut into random blocks of ~200 rows, A's blocks
    inside C's blocks; FP64 through the factorization's CUDA-core update
    kernel (spx.update), against the oracle's panel update."""
    for (m, k, nb, lower, seed) in [(300, 64, 100, 0, 1), (1000, 128, 257, 1, 2),
                                    (65, 1, 65, 1, 3), (777, 33, 64, 0, 4), (2048, 160, 511, 1, 5)]:
        A, C, rowmap, colmap = inputs.gapped_update_case(m, k, nb, seed)
        expect = oracle.panel_update(A, A[:nb], C, rowmap, colmap, bool(lower))
        tA = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
        tC = torch.from_numpy(np.ascontiguousarray(C.T)).cuda().t()
        spx.update(tA, tC, rowmap, colmap, nb, lower=bool(lower))
        got = tC.cpu().numpy()
        assert np.max(np.abs(got - expect)) <= 1e-12 * max(1.0, np.max(np.abs(expect)))


def test_fgmres_takes_over_when_plain_refinement_stalls(torch):
    """High coefficient contrast (exp(3g)) with BF16 updates: plain refinement
    stops contracting; FGMRES preconditioned by the same factor reaches 1e-12."""
    g = 24
    A = inputs.diffusion_3d(g, g, g, 7, sigma=3.0)
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "llt", ordering=1, grid=(g, g, g), max_width=64)
    h.factorize(vals, "bf16")
    B = inputs.rhs(A.shape[0], 4, 7)
    _, plain = h.solve(B, refine=spx.default_refine(tol=1e-12, mode=1, max_iter=10))
    assert not plain["converged"]
    X, auto = h.solve(B, refine=spx.default_refine(tol=1e-12, mode=2, max_iter=10))
    assert auto["converged"] and auto["gmres_iters"] > 0
    assert oracle.backward_error(A, X, B) <= 1e-12


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_fgmres_alone_reaches_target(torch, prec):
    A = inputs.diffusion_3d(15, 14, 13, 4)
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "llt", ordering=1, grid=(15, 14, 13), max_width=32)
    h.factorize(vals, prec)
    B = inputs.rhs(A.shape[0], 3, 4)
    X, info = h.solve(B, refine=spx.default_refine(tol=1e-12, mode=2, max_iter=0, gmres_restart=5))
    assert info["converged"] and info["iters"] == 0 and info["gmres_iters"] > 0
    assert oracle.backward_error(A, X, B) <= 1e-12
