"""Host-side analysis of the batched LU (no GPU): pattern classes, orderings,
exact flop and nnz(L) counts against the oracle's own symbolic code."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_1405_2636_gb300 import inputs, spx


def _systems(sides, seed=7):
    mats = [inputs.convection_diffusion_2d(k, seed * 100 + i)[0] for i, k in enumerate(sides)]
    return mats, [inputs.csc_arrays(A)[:2] for A in mats]


def test_patterns_are_shared_by_class():
    sides = [12, 13, 12, 20, 13, 12]
    mats, systems = _systems(sides)
    b = spx.batch_analyze(systems, grids=[(k, k, 1) for k in sides], ordering=spx.SPX_ORDER_GRID)
    info = b.info()
    assert info["nsys"] == 6 and info["nclasses"] == 3
    assert info["n_total"] == sum(k * k for k in sides)
    assert info["n_max"] == 400
    assert info["nnz_total"] == sum(A.nnz for A in mats)
    b.free()


def test_orderings_and_counts_match_the_oracle():
    sides = [5, 12, 17, 31]
    mats, systems = _systems(sides, seed=3)
    b = spx.batch_analyze(systems, grids=[(k, k, 1) for k in sides], ordering=spx.SPX_ORDER_GRID)
    flops = 0.0
    nnzl = 0
    for s, (A, k) in enumerate(zip(mats, sides)):
        perm = b.perm(s)
        assert np.array_equal(perm, oracle.nd_grid(k, k))
        sym = oracle.symbolic(oracle.symmetrized_pattern(oracle.permute(A, perm)))
        flops += oracle.flops(sym.counts, "lu")
        nnzl += int(sym.Lp[-1])
    info = b.info()
    assert info["flops"] == flops
    assert info["nnz_l_total"] == nnzl
    b.free()


def test_same_pattern_with_another_grid_is_another_class():
    # a 6 x 6 grid and a 36 x 1 "grid" of the same 1-D chain pattern differ
    A = sp.diags([-1.0, 2.5, -1.0], [-1, 0, 1], shape=(36, 36), format="csc")
    cp, ri, _ = inputs.csc_arrays(A)
    b = spx.batch_analyze([(cp, ri), (cp, ri)], grids=[(36, 1, 1), (36, 1, 1)],
                          ordering=spx.SPX_ORDER_GRID)
    assert b.info()["nclasses"] == 1
    b.free()
    b = spx.batch_analyze([(cp, ri), (cp, ri)], grids=[(36, 1, 1), (6, 6, 1)],
                          ordering=spx.SPX_ORDER_GRID)
    assert b.info()["nclasses"] == 2
    b.free()


def test_bad_arguments_are_rejected():
    A = inputs.convection_diffusion_2d(4, 1)[0]
    cp, ri, _ = inputs.csc_arrays(A)
    bad = cp.copy()
    bad += 1
    with pytest.raises(spx.SpxError) as e:
        spx.batch_analyze([(bad, ri)])
    assert e.value.status == spx.SPX_ERR_ARG
    with pytest.raises(spx.SpxError):
        spx.batch_analyze([(cp, ri)], lower_only=1)


def test_empty_batch():
    b = spx.batch_analyze([])
    assert b.info()["nsys"] == 0
    b.free()


def test_generator_recipe():
    mats, sides, rhs = inputs.batched_convection_diffusion(16, 4)
    assert all(12 <= k <= 80 for k in sides)
    assert [A.shape[0] for A in mats] == [k * k for k in sides]
    assert rhs.shape == (sum(k * k for k in sides),)
    # unsymmetric values, symmetric pattern, row-diagonally dominant (an M-matrix)
    A = mats[0]
    P = (A != 0).astype(np.int8)
    assert (P != P.T).nnz == 0
    assert abs(A - A.T).max() > 0
    d = A.diagonal()
    off = np.asarray(abs(A).sum(axis=1)).ravel() - abs(d)
    assert np.all(d >= off - 1e-12)
