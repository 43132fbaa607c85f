"""The distributed factorization by subtrees with fan-in, on one GPU: the
ranks are emulated one after another, each with its own handle on the same
pattern (no kernel of one rank ever waits on another).  Each rank factors its
subtrees on the device task queue with its updates into the top panels; the
ranks' packed top panels are summed (the fan-in) into rank 0, which factors
the top; the other ranks' parts are copied in, and rank 0's handle then
holds the whole factor, which must match the oracle on its pattern and solve
to the usual backward error."""
import numpy as np
import pytest

import oracle
from paper_1405_2636_gb300 import fanin, inputs, spx

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


def _system(method):
    if method == "ldlt":
        g = (12, 11, 10)
        return inputs.quasi_definite_3d(*g, 41), dict(ordering=spx.SPX_ORDER_GRID, grid=g, dof=2, max_width=48)
    g = (20, 19, 18)
    return inputs.diffusion_3d(*g, 41), dict(ordering=spx.SPX_ORDER_GRID, grid=g, max_width=64)


@pytest.mark.parametrize("method,prec", [("llt", "fp64"), ("llt", "tf32"), ("llt", "bf16"), ("ldlt", "fp64"),
                                         ("ldlt", "tf32")])
@pytest.mark.parametrize("nranks", [2, 3])
def test_distributed_factor_matches_oracle(torch, method, prec, nranks):
    A, opts = _system(method)
    cp, ri, vals = inputs.csc_arrays(A)
    hs = [spx.analyze(cp, ri, method, **opts) for _ in range(nranks)]
    parts = [h.partition(nranks) for h in hs]
    assert all(np.array_equal(p["owner"], parts[0]["owner"]) for p in parts)
    assert (parts[0]["owner"] < 0).any() and all((parts[0]["owner"] == r).any() for r in range(nranks))
    for r, h in enumerate(hs):
        h.factorize_part(vals, prec, r)
    top = sum(h.part_get(-1) for h in hs)          # the fan-in
    h0 = hs[0]
    h0.part_set(-1, top)
    h0.factorize_part(None, prec, -1)
    for r in range(1, nranks):
        h0.part_set(r, hs[r].part_get(r, with_inverses=True), with_inverses=True)
    F = (oracle.ldlt if method == "ldlt" else oracle.cholesky)(A, h0.perm())
    Lx = h0.factor_on_pattern(F.sym.Lp, F.sym.Li)
    bound = {"fp64": 1e-12, "tf32": 2e-2, "bf16": 1e-1}[prec]
    assert _rel(Lx, F.Lx) <= bound
    B = inputs.rhs(A.shape[0], 3, 41)
    X, info = h0.solve(B, refine=None if prec == "fp64" else spx.default_refine(tol=1e-12))
    assert info["converged"]
    assert oracle.backward_error(A, X, B) <= (1e-13 if prec == "fp64" else 1e-12)
    for h in hs:
        h.free()


def test_one_rank_through_the_module(torch):
    """world = 1: one part holds every panel, the top is empty, and the
    module's driver leaves a complete factor."""
    A, opts = _system("llt")
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "llt", **opts)
    part = fanin.factorize_distributed(h, vals, "fp64", world=1, rank=0)
    assert (part["owner"] == 0).all() and part["values"][1] == 0
    F = oracle.cholesky(A, h.perm())
    assert _rel(h.factor_on_pattern(F.sym.Lp, F.sym.Li), F.Lx) <= 1e-12
    B = inputs.rhs(A.shape[0], 2, 3)
    X, _ = h.solve(B)
    assert oracle.backward_error(A, X, B) <= 1e-13
    h.free()


def test_part_calls_check_their_state(torch):
    A, opts = _system("llt")
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "llt", **opts)
    with pytest.raises(spx.SpxError) as e:
        h.factorize_part(vals, "fp64", 0)              # before spx_partition
    assert e.value.status == spx.SPX_ERR_STATE
    h.partition(2)
    with pytest.raises(spx.SpxError) as e:
        h.factorize_part(None, "fp64", -1)             # the top before this handle's own part
    assert e.value.status == spx.SPX_ERR_STATE
    with pytest.raises(spx.SpxError) as e:
        h.factorize_part(vals, "fp64", 2)              # no rank 2
    assert e.value.status == spx.SPX_ERR_ARG
    h.free()
