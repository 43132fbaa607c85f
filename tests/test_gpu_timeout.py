"""Bounded device waits: a sweep wait that runs out returns SPX_ERR_TIMEOUT
instead of hanging, and the handle keeps working.

The triangular sweeps walk a device-side work queue whose items wait on
per-panel counters.  With the wait limit cut to one poll (spx_set_wait_limit),
an item whose predecessor is still running gives up at once: near the top of
the elimination tree each panel waits on the chunks of the panel below it,
which take microseconds, so some wait always runs out.  The kernel then
records the timeout and its CTAs return; nothing faults and nothing hangs.
With the default limit restored, the next solve is correct.
"""
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


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_sweep_wait_runs_out_and_the_handle_recovers(torch, prec):
    g = (24, 24, 24)
    A = inputs.diffusion_3d(*g, 3)
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "llt", ordering=spx.SPX_ORDER_GRID, grid=g, max_width=64)
    h.factorize(vals, prec)
    B = inputs.rhs(A.shape[0], 4, 3)
    h.set_wait_limit(1)
    with pytest.raises(spx.SpxError) as e:
        h.solve(B, refine=spx.default_refine(mode=0))
    assert e.value.status == spx.SPX_ERR_TIMEOUT
    h.set_wait_limit(0)
    X, info = h.solve(B, refine=None if prec == "fp64" else spx.default_refine(tol=1e-12))
    assert info["status"] == "SPX_OK"
    assert oracle.backward_error(A, X, B) <= (1e-13 if prec == "fp64" else 1e-12)
    h.free()
