"""The deterministic update mode: the updates of each level run in rounds
(one task per target panel per round, in task order), so every entry of a
target panel receives its contributions in a fixed order.  Two
factorizations -- on the same handle and on a second handle analysed from the
same pattern -- must give bit-identical factors, which must still match the
oracle within the usual tolerances."""
import numpy as np
import pytest

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


CASES = [  # method, precision, bound against the oracle
    ("llt", "fp64", 1e-12), ("llt", "tf32", 2e-2), ("llt", "bf16", 1e-1), ("llt", "fp32", 1e-4),
    ("ldlt", "tf32", 2e-2), ("ldlt", "fp32", 1e-4), ("lu", "fp64", 1e-12), ("lu", "fp32", 1e-4),
]


def _system(method):
    if method == "lu":
        A = inputs.convection_diffusion_2d(60, 31)[0]
        return A, dict(ordering=spx.SPX_ORDER_GRID, grid=(60, 60, 1), max_width=32)
    if method == "ldlt":
        A = inputs.quasi_definite_3d(12, 11, 10, 31)
        return A, dict(ordering=spx.SPX_ORDER_GRID, grid=(12, 11, 10), dof=2, max_width=64)
    A = inputs.diffusion_3d(22, 21, 20, 31)
    return A, dict(ordering=spx.SPX_ORDER_GRID, grid=(22, 21, 20), max_width=64)


@pytest.mark.parametrize("method,prec,bound", CASES)
def test_deterministic_factors_are_bit_identical(torch, method, prec, bound):
    A, opts = _system(method)
    cp, ri, vals = inputs.csc_arrays(A)
    h1 = spx.analyze(cp, ri, method, deterministic=1, **opts)
    h2 = spx.analyze(cp, ri, method, deterministic=1, **opts)
    F = {"llt": oracle.cholesky, "ldlt": oracle.ldlt, "lu": oracle.lu}[method](A, h1.perm())
    lu = method == "lu"
    got = []
    for h in (h1, h1, h2):
        h.factorize(vals, prec)
        f = h.factor_on_pattern(F.sym.Lp, F.sym.Li, lu=lu)
        got.append(np.concatenate(f) if lu else f)
    assert np.array_equal(got[0], got[1]) and np.array_equal(got[0], got[2])
    ref = np.concatenate([F.Lx, F.Ut]) if lu else F.Lx
    assert _rel(got[0], ref) <= bound
    h1.set_profiling(True)       # more launches than levels: the rounds
    h1.factorize(vals, prec)
    h1.set_profiling(False)
    ks = h1.kernel_stats()
    assert ks["queue"]["launches"] == 0
    assert ks["update"]["launches"] + ks["update_tc"]["launches"] > h1.info()["nlevels"]
    f = h1.factor_on_pattern(F.sym.Lp, F.sym.Li, lu=lu)
    assert np.array_equal(np.concatenate(f) if lu else f, got[0])
    h1.free()
    h2.free()
