"""Pins of the oracle's panel update (Sec. V-B: C = C - A B^T, B the first
rows of A, subtracted at the target's block positions), checked against what
the mathematics fixes rather than against a retyped formula."""
import numpy as np

import oracle


def test_hand_computed_gapped_update():
    # A = [[1, 2], [3, 4], [5, 6]], B = first 2 rows; rows of A go to target
    # rows 0, 2, 5 of a 6 x 3 zero target; B's rows face columns 1 and 2.
    A = np.array([[1.0, 2.0], [3.0, 4.0], [5.0, 6.0]])
    C = np.zeros((6, 3))
    rowmap = np.array([0, 2, 5])
    colmap = np.array([1, 2])
    full = oracle.panel_update(A, A[:2], C, rowmap, colmap, lower=False)
    expect = np.zeros((6, 3))
    # A A[:2]^T = [[5, 11], [11, 25], [17, 39]]
    expect[0, 1], expect[2, 1], expect[5, 1] = -5.0, -11.0, -17.0
    expect[0, 2], expect[2, 2], expect[5, 2] = -11.0, -25.0, -39.0
    assert np.array_equal(full, expect)
    low = oracle.panel_update(A, A[:2], C, rowmap, colmap, lower=True)
    expect[0, 2] = 0.0            # source row 0 < facing row 1: above the diagonal
    assert np.array_equal(low, expect)


def test_schur_complement_of_a_dense_cholesky_factor():
    """With A = L21 (the rows below the first s columns of chol(M)), the
    update of M22 scattered into a gapped target leaves L22 L22^T at the
    mapped positions (lower part), where L22 is the trailing block of the
    same dense factor; every other target entry is untouched."""
    g = np.random.default_rng(11)
    s, t = 7, 9
    X = g.standard_normal((s + t, s + t))
    M = X @ X.T + (s + t) * np.eye(s + t)
    L = np.linalg.cholesky(M)
    L21, L22 = L[s:, :s], L[s:, s:]
    ldc, nc = 25, 14
    rowmap = np.sort(g.choice(ldc, size=t, replace=False))
    colmap = np.sort(g.choice(nc, size=t, replace=False))
    C = g.standard_normal((ldc, nc))
    for i in range(t):
        for j in range(i + 1):
            C[rowmap[i], colmap[j]] = M[s + i, s + j]
    out = oracle.panel_update(L21, L21, C, rowmap, colmap, lower=True)
    S = L22 @ L22.T
    touched = np.zeros_like(C, dtype=bool)
    for i in range(t):
        for j in range(i + 1):
            assert abs(out[rowmap[i], colmap[j]] - S[i, j]) <= 1e-13 * abs(M).max()
            touched[rowmap[i], colmap[j]] = True
    assert np.array_equal(out[~touched], C[~touched])
