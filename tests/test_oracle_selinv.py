"""Pins of the oracle's selected inverse and log-determinant (the adjoint
pieces of the differentiable solve), against mathematics only: the dense
inverse by brute force, the closed-form inverse of the 1-D Laplacian, the
closed-form spectrum of the 2-D Laplacian, and trace(A A^{-1}) = n."""
import numpy as np
import scipy.sparse as sp

import oracle
from paper_1405_2636_gb300 import inputs


def _dense_pattern_values(M, F):
    s = F.sym
    cols = np.repeat(np.arange(s.n), np.diff(s.Lp))
    return M[s.Li, cols]


def test_selected_inverse_matches_dense_inverse():
    for n, deg, seed in ((60, 4.0, 1), (120, 6.0, 2), (17, 2.0, 3)):
        A = inputs.random_spd_graph(n, deg, seed)
        perm = oracle.nd_graph(A)
        F = oracle.cholesky(A, perm)
        Z = oracle.selected_inverse(F)
        Pa = oracle.permute(A, perm).toarray()
        ref = _dense_pattern_values(np.linalg.inv(Pa), F)
        assert np.max(np.abs(Z - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_selected_inverse_1d_laplacian_closed_form():
    """(tridiag(-1, 2, -1))^{-1}_{ij} = min(i,j) (n+1-max(i,j)) / (n+1), 1-based."""
    n = 50
    A = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(n, n), format="csc")
    F = oracle.cholesky(A, np.arange(n))
    Z = oracle.selected_inverse(F)
    s = F.sym
    cols = np.repeat(np.arange(n), np.diff(s.Lp)) + 1
    rows = s.Li + 1
    expect = np.minimum(rows, cols) * (n + 1 - np.maximum(rows, cols)) / (n + 1)
    np.testing.assert_allclose(Z, expect, rtol=1e-13)
    assert len(Z) == 2 * n - 1


def test_logdet_2d_laplacian_spectrum():
    A = inputs.laplacian_2d(31, 31)
    F = oracle.cholesky(A, oracle.nd_grid(31, 31))
    i = np.arange(1, 32)
    lam = 4 - 2 * np.cos(i[:, None] * np.pi / 32) - 2 * np.cos(i[None, :] * np.pi / 32) + 0.01
    assert abs(oracle.logdet(F) - np.log(lam).sum()) <= 1e-12 * abs(np.log(lam).sum())


def test_logdet_gradient_trace_identity_and_dense():
    # sum over A's entries of A_ij (A^{-1})_ji = trace(A A^{-1}) = n
    A = inputs.diffusion_3d(9, 8, 7, 5)
    F = oracle.cholesky(A, oracle.nd_grid(9, 8, 7))
    g = oracle.logdet_gradient(A, F)
    n = A.shape[0]
    assert abs(np.dot(A.tocsc().data, g) - n) <= 1e-10 * n
    # small case against the dense inverse, entry by entry
    A = inputs.diffusion_3d(4, 3, 3, 6)
    F = oracle.cholesky(A, oracle.nd_grid(4, 3, 3))
    g = oracle.logdet_gradient(A, F)
    Ainv = np.linalg.inv(A.toarray())
    coo = A.tocsc().tocoo()
    np.testing.assert_allclose(g, Ainv.T[coo.row, coo.col], rtol=1e-12, atol=1e-15)


def test_coefficient_map_reproduces_generator():
    """values = M kappa reproduces diffusion_3d's CSC values exactly."""
    nx, ny, nz, seed = 7, 6, 5, 9
    A = inputs.diffusion_3d(nx, ny, nz, seed)
    cp, ri, M = inputs.diffusion_3d_coefficient_map(nx, ny, nz)
    kappa = inputs.diffusion_3d_kappa(nx, ny, nz, seed)
    assert np.array_equal(cp, A.indptr) and np.array_equal(ri, A.indices)
    np.testing.assert_allclose(M @ kappa, A.data, rtol=1e-15, atol=0)
