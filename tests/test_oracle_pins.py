"""Pins of the CPU oracle against facts fixed by the paper or by mathematics.

Nothing here compares the oracle with itself: each test checks it against a
hand-derived fixture, a closed form, a brute-force dense factorization or an
invariant, so that a dropped term, a wrong sign, a wrong index or a
transposed operand in the oracle fails at least one of them.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import oracle
from paper_1405_2636_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_grid_orders():
    out = []
    with open(os.path.join(GOLDEN, "nd_grid_orders.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            dims, perm = line.split(":")
            out.append((tuple(int(v) for v in dims.split()), [int(v) for v in perm.split()]))
    return out


@pytest.mark.parametrize("dims,expected", _read_grid_orders())
def test_nd_grid_matches_hand_derived_order(dims, expected):
    nx, ny, nz, dof = dims
    assert oracle.nd_grid(nx, ny, nz, dof).tolist() == expected


def test_nd_graph_path_matches_hand_derived_order():
    with open(os.path.join(GOLDEN, "nd_graph_path200.txt")) as f:
        toks = [t for line in f if not line.startswith("#") for t in line.split()]
    expected = []
    for t in toks:
        if "-" in t:
            a, b = t.split("-")
            expected += list(range(int(a), int(b) + 1))
        else:
            expected.append(int(t))
    n = 200
    A = sp.diags([np.full(n - 1, -1.0), np.full(n, 2.0), np.full(n - 1, -1.0)], [-1, 0, 1]).tocsc()
    assert oracle.nd_graph(A).tolist() == expected


@pytest.mark.parametrize("dims", [(7, 5, 1, 1), (6, 6, 6, 1), (5, 4, 3, 3), (31, 31, 1, 1)])
def test_nd_grid_separators_separate(dims):
    """Each separator plane disconnects the two halves: the etree of the
    reordered Laplacian has the two halves as disjoint subtrees, which shows as
    no nonzero of L coupling the halves."""
    nx, ny, nz, dof = dims
    perm = oracle.nd_grid(nx, ny, nz, dof)
    assert sorted(perm.tolist()) == list(range(nx * ny * nz * dof))
    A = inputs.laplacian_3d(nx, ny, nz, shift=1.0, two_d=(nz == 1))
    if dof > 1:
        A = sp.kron(A, np.ones((dof, dof)) + np.eye(dof) * 10, format="csc")
    F = oracle.cholesky(A, perm)
    # top split: the last separator plane; everything before splits into halves
    node_perm = perm[::dof] // dof
    coords = np.stack([node_perm % nx, (node_perm // nx) % ny, node_perm // (nx * ny)], 1)
    lens = [nx, ny, nz]
    if nx * ny * nz <= 8:
        return
    ax = int(np.argmax(lens))
    cut = lens[ax] // 2
    side = np.where(coords[:, ax] < cut, 0, np.where(coords[:, ax] > cut, 1, 2))
    side = np.repeat(side, dof)
    L = F.L().tocoo()
    bad = (side[L.row] == 0) & (side[L.col] == 1) | (side[L.row] == 1) & (side[L.col] == 0)
    assert not bad.any()


def _random_spd(n, seed, deg=4.0):
    return inputs.random_spd_graph(n, deg, seed)


@pytest.mark.parametrize("n,seed", [(30, 1), (120, 2), (200, 3)])
def test_symbolic_and_etree_match_dense_brute_force(n, seed):
    A = _random_spd(n, seed)
    perm = oracle.nd_graph(A)
    F = oracle.cholesky(A, perm)
    Pa = oracle.permute(A, perm).toarray()
    Ld = np.linalg.cholesky(Pa)
    nz_dense = Ld != 0.0
    L = F.L().toarray()
    nz_sym = np.zeros_like(nz_dense)
    s = F.sym
    for j in range(n):
        nz_sym[s.Li[s.Lp[j]:s.Lp[j + 1]], j] = True
    assert np.array_equal(nz_dense, nz_sym)
    # column counts from row subtrees == fill of the symbolic pattern
    assert np.array_equal(s.counts, nz_dense.sum(axis=0))
    assert s.Lp[-1] == nz_dense.sum()
    # elimination tree: parent(j) = min{i > j : L(i,j) != 0}
    for j in range(n):
        below = np.nonzero(nz_dense[j + 1:, j])[0]
        expect = j + 1 + below[0] if below.size else -1
        assert s.parent[j] == expect and s.parent_sym[j] == expect
    np.testing.assert_allclose(L, Ld, rtol=0, atol=1e-13 * np.abs(Ld).max())


@pytest.mark.parametrize("maker", [
    lambda: inputs.laplacian_2d(31, 31),
    lambda: inputs.diffusion_3d(9, 8, 7, 5),
    lambda: inputs.elasticity_27pt(4, 4, 3, 6),
])
def test_factor_reconstructs_matrix(maker):
    A = maker()
    n = A.shape[0]
    F = oracle.cholesky(A, oracle.nd_graph(A))
    Pa = oracle.permute(A, F.perm)
    L = F.L()
    err = sp.linalg.norm(Pa - L @ L.T) / sp.linalg.norm(Pa)
    assert err <= 1e-14
    assert n == Pa.shape[0]


def test_tridiagonal_closed_form():
    """Cholesky of tridiag(-1, 2, -1): L(j,j) = sqrt((j+2)/(j+1)),
    L(j+1,j) = -sqrt((j+1)/(j+2)) (0-based)."""
    n = 150
    A = sp.diags([np.full(n - 1, -1.0), np.full(n, 2.0), np.full(n - 1, -1.0)], [-1, 0, 1]).tocsc()
    F = oracle.cholesky(A, np.arange(n))
    L = F.L().toarray()
    j = np.arange(n)
    np.testing.assert_allclose(np.diag(L), np.sqrt((j + 2.0) / (j + 1.0)), rtol=1e-15)
    np.testing.assert_allclose(np.diag(L, -1), -np.sqrt((j[:-1] + 1.0) / (j[:-1] + 2.0)), rtol=1e-15)
    assert F.sym.Lp[-1] == 2 * n - 1


def test_laplacian_logdet_closed_form():
    """det of the 31x31 Dirichlet 5-point Laplacian + 1e-2 I from its spectrum
    lambda_ij = 4 - 2cos(i pi/32) - 2cos(j pi/32) + 0.01."""
    A = inputs.laplacian_2d(31, 31)
    F = oracle.cholesky(A, oracle.nd_grid(31, 31))
    Ldiag = F.Lx[F.sym.Lp[:-1]]
    i = np.arange(1, 32)
    lam = 4 - 2 * np.cos(i[:, None] * np.pi / 32) - 2 * np.cos(i[None, :] * np.pi / 32) + 0.01
    assert abs(2 * np.log(Ldiag).sum() - np.log(lam).sum()) < 1e-10


def test_flop_count_closed_form_dense():
    """Dense n x n pattern: column counts n-j, so sum c_j^2 = n(n+1)(2n+1)/6."""
    n = 60
    rng = inputs.rng(11, 0)
    M = rng.standard_normal((n, n))
    A = sp.csc_matrix(M @ M.T + n * np.eye(n))
    F = oracle.cholesky(A, np.arange(n))
    assert np.array_equal(F.sym.counts, np.arange(n, 0, -1))
    assert oracle.flops(F.sym.counts, "llt") == n * (n + 1) * (2 * n + 1) / 6
    # LU: sum 2(c-1)^2 + (c-1) = dense LU count 2n^3/3 - n^2/2 - n/6
    assert oracle.flops(F.sym.counts, "lu") == pytest.approx(2 * n**3 / 3 - n**2 / 2 - n / 6)


def test_not_positive_definite_is_reported():
    A = sp.csc_matrix(np.array([[1.0, 2.0], [2.0, 1.0]]))
    with pytest.raises(oracle.NotPositiveDefinite) as e:
        oracle.cholesky(A, np.arange(2))
    assert e.value.col == 1


def _coldominant_unsym(n, seed):
    """Unsymmetric values on a symmetric pattern, strictly column diagonally
    dominant (so partial pivoting never swaps rows)."""
    A = _random_spd(n, seed)
    rng = inputs.rng(seed, 2)
    B = A.tocoo()
    vals = B.data * rng.uniform(0.2, 1.8, size=B.data.size)
    off = B.row != B.col
    C = sp.coo_matrix((np.where(off, vals, 0.0), (B.row, B.col)), shape=A.shape).tocsc()
    d = np.asarray(abs(C).sum(axis=0)).ravel() * 1.5 + 1.0
    return (C + sp.diags(d)).tocsc()


@pytest.mark.parametrize("n,seed", [(40, 4), (180, 5)])
def test_lu_matches_dense_no_pivot_lu(n, seed):
    A = _coldominant_unsym(n, seed)
    perm = oracle.nd_graph(A)
    F = oracle.lu(A, perm)
    assert F.nrepl == 0
    Pa = oracle.permute(A, perm).toarray()
    lu, piv = sla.lu_factor(Pa)
    assert np.array_equal(piv, np.arange(n))  # partial pivoting chose the diagonal
    Ld = np.tril(lu, -1) + np.eye(n)
    Ud = np.triu(lu)
    L = F.L().toarray()
    U = F.U().toarray()
    np.testing.assert_allclose(L, Ld, atol=1e-13 * np.abs(Ld).max(), rtol=0)
    np.testing.assert_allclose(U, Ud, atol=1e-13 * np.abs(Ud).max(), rtol=0)


def test_static_pivot_hand_example():
    """A = [[0, 1], [1, 1]]: ||A||_inf = 2, tau = 2^-26 * 2 = 2^-25; the zero
    pivot becomes +tau, L(1,0) = 2^25, U(0,1) = 1, U(1,1) = 1 - 2^25."""
    A = sp.csc_matrix(np.array([[0.0, 1.0], [1.0, 1.0]]))
    F = oracle.lu(A, np.arange(2))
    assert F.tau == 2.0 ** -25
    assert F.nrepl == 1
    L, U = F.L().toarray(), F.U().toarray()
    assert L[1, 0] == 2.0 ** 25 and L[0, 0] == 1.0 and L[1, 1] == 1.0
    assert U[0, 0] == 2.0 ** -25 and U[0, 1] == 1.0 and U[1, 1] == 1.0 - 2.0 ** 25
    # a tiny negative pivot keeps its sign
    B = sp.csc_matrix(np.array([[-1e-20, 1.0], [1.0, 1.0]]))
    G = oracle.lu(B, np.arange(2))
    assert G.nrepl == 1 and G.U().toarray()[0, 0] == -G.tau


def test_convection_diffusion_needs_no_pivot_replacement():
    for seed in range(4):
        A, _ = inputs.convection_diffusion_2d(14 + 5 * seed, seed)
        F = oracle.lu(A, oracle.nd_grid(14 + 5 * seed, 14 + 5 * seed))
        assert F.nrepl == 0
        b = inputs.rhs(A.shape[0], 2, seed)
        x = oracle.solve(F, b)
        assert oracle.backward_error(A, x, b) < 1e-14


def test_solve_matches_dense_solve():
    A = _random_spd(150, 8)
    F = oracle.cholesky(A, oracle.nd_graph(A))
    b = inputs.rhs(150, 3, 8)
    x = oracle.solve(F, b)
    np.testing.assert_allclose(x, np.linalg.solve(A.toarray(), b), rtol=1e-12, atol=1e-13)
    assert oracle.backward_error(A, x, b) < 1e-15


def test_c1_solve_backward_error():
    A = inputs.laplacian_2d(31, 31)
    F = oracle.cholesky(A, oracle.nd_grid(31, 31))
    b = inputs.rhs(A.shape[0], 1, 1)
    assert oracle.backward_error(A, oracle.solve(F, b), b) <= 1e-15


def test_spmv_matches_scipy():
    A = _coldominant_unsym(70, 9)
    x = inputs.rhs(70, 1, 9)[:, 0]
    np.testing.assert_allclose(oracle.spmv(A, x), A @ x, rtol=1e-14, atol=1e-14)


def test_lu_solve_matches_dense_solve():
    """The LU solve on an unsymmetric, column-dominant matrix (no pivot is
    replaced) equals the dense solve; solving with A^T instead of A, or with
    L and U swapped, would not."""
    A = _coldominant_unsym(120, 12)
    for perm in (np.arange(120), oracle.nd_graph(A)):
        F = oracle.lu(A, perm)
        assert F.nrepl == 0
        B = inputs.rhs(120, 3, 12)
        X = oracle.solve(F, B)
        np.testing.assert_allclose(X, np.linalg.solve(A.toarray(), B), rtol=1e-11, atol=1e-13)
        assert np.abs(A.toarray() - A.toarray().T).max() > 0.1      # the check would see a transpose
        assert oracle.backward_error(A, X, B) < 1e-15
