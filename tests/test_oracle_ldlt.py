"""Pins of the oracle's LDL^T (static pivoting) against mathematics only:
reconstruction by brute force, Sylvester's law of inertia against dense
eigenvalues, the Cholesky factor as L sqrt(D) on SPD matrices, the closed
form of the 1-D Laplacian, and a hand-computed static-pivot replacement."""
import numpy as np
import scipy.sparse as sp

import oracle
from paper_1405_2636_gb300 import inputs


def _dense(F):
    s = F.sym
    L = sp.csc_matrix((F.Lx, s.Li, s.Lp), shape=(s.n, s.n)).toarray()
    d = np.diag(L).copy()
    np.fill_diagonal(L, 1.0)
    return L, d


def test_reconstruction_and_inertia_quasi_definite():
    for dims, seed in (((3, 3, 2), 1), ((4, 3, 3), 2), ((5, 4, 3), 3)):
        A = inputs.quasi_definite_3d(*dims, seed)
        perm = oracle.nd_grid(*dims, dof=2)
        F = oracle.ldlt(A, perm)
        assert F.nrepl == 0
        L, d = _dense(F)
        Pa = oracle.permute(A, perm).toarray()
        assert np.linalg.norm(Pa - L @ np.diag(d) @ L.T) <= 1e-14 * np.linalg.norm(Pa)
        ev = np.linalg.eigvalsh(A.toarray())
        pos, neg = oracle.inertia(F)
        assert (pos, neg) == (int(np.sum(ev > 0)), int(np.sum(ev < 0)))
        assert neg == A.shape[0] // 2
        B = inputs.rhs(A.shape[0], 2, seed)
        assert oracle.backward_error(A, oracle.solve(F, B), B) <= 1e-14


def test_inertia_of_a_shifted_laplacian():
    """-Laplacian - sigma I with sigma between eigenvalues: the number of
    negative pivots is the number of eigenvalues below sigma."""
    A = inputs.laplacian_2d(9, 8, 0.0)
    ev = np.linalg.eigvalsh(A.toarray())
    sigma = 0.5 * (ev[6] + ev[7])
    As = (A - sigma * sp.identity(A.shape[0])).tocsc()
    F = oracle.ldlt(As, oracle.nd_grid(9, 8))
    assert F.nrepl == 0
    assert oracle.inertia(F) == (A.shape[0] - 7, 7)


def test_cholesky_is_l_sqrt_d_on_spd():
    A = inputs.diffusion_3d(6, 5, 4, 7)
    perm = oracle.nd_grid(6, 5, 4)
    F = oracle.ldlt(A, perm)
    C = oracle.cholesky(A, perm)
    s = F.sym
    cols = np.repeat(np.arange(s.n), np.diff(s.Lp))
    d = F.Lx[s.Lp[:-1]]
    Lc = np.where(s.Li == cols, np.sqrt(d[cols]), F.Lx * np.sqrt(d[cols]))
    np.testing.assert_allclose(Lc, C.Lx, rtol=1e-14, atol=1e-15)


def test_1d_laplacian_closed_form():
    """tridiag(-1, 2, -1): d_j = (j+2)/(j+1), L(j+1, j) = -(j+1)/(j+2), 0-based."""
    n = 40
    A = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(n, n), format="csc")
    F = oracle.ldlt(A, np.arange(n))
    L, d = _dense(F)
    j = np.arange(n)
    np.testing.assert_allclose(d, (j + 2.0) / (j + 1.0), rtol=1e-15)
    np.testing.assert_allclose(np.diag(L, -1), -(j[:-1] + 1.0) / (j[:-1] + 2.0), rtol=1e-15)


def test_static_pivot_hand_example():
    """[[0, 1], [1, 1]]: d_0 = 0 becomes tau = sqrt(2^-52) * 2 = 2^-25, then
    L(1,0) = 2^25 and d_1 = 1 - 2^25 exactly."""
    A = sp.csc_matrix(np.array([[0.0, 1.0], [1.0, 1.0]]))
    F = oracle.ldlt(A, np.arange(2))
    L, d = _dense(F)
    assert F.nrepl == 1
    assert d[0] == 2.0 ** -25 and L[1, 0] == 2.0 ** 25 and d[1] == 1.0 - 2.0 ** 25
