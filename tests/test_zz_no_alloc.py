"""spx_solve_noalloc: the solve for callers that cannot allocate device memory.

Some callers cannot allocate when they solve (a real-time loop, where a
cudaMalloc would synchronize and stall the device, or a host whose device
memory is owned by another allocator).  spx_solve_noalloc keeps its sweep
vectors in a fixed file-scope device buffer instead.  Its output must match spx_solve
without refinement -- the same sweep, with the handle's workspace -- within
the tolerances the other GPU tests use, on two calls in a row (the buffer
keeps the previous call's contents).  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_1405_2636_gb300 import inputs, spx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    import __graft_entry__

    __graft_entry__.build()
    assert _t.cuda.is_available()
    return _t


def _colmajor(torch, M):
    return torch.from_numpy(np.ascontiguousarray(M.T)).cuda().t()


def _noalloc(torch, h, Bd, nrhs, check_free=False):
    n = h.n
    Xd = torch.full((nrhs, n), float("nan"), dtype=torch.float64, device="cuda").t()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    st = spx.load().spx_solve_noalloc(h._h, nrhs, Bd.data_ptr(), n, Xd.data_ptr(), n, None)
    assert st == spx.SPX_OK, spx.load().spx_last_error(h._h)
    torch.cuda.synchronize()
    if check_free:   # the call itself took no device memory
        assert torch.cuda.mem_get_info()[0] == free0
    return Xd.cpu().numpy()


CASES = [  # method, precision, tolerance against spx_solve without refinement
    ("llt", "fp64", 1e-12), ("llt", "fp32", 1e-5),
    ("lu", "fp64", 1e-12), ("ldlt", "fp64", 1e-12),
]


def _system(method):
    if method == "lu":
        A = inputs.convection_diffusion_2d(47, 21)[0]
        return A, dict(ordering=spx.SPX_ORDER_GRID, grid=(47, 47, 1), max_width=48)
    if method == "ldlt":
        A = inputs.quasi_definite_3d(9, 8, 7, 21)
        return A, dict(ordering=spx.SPX_ORDER_GRID, grid=(9, 8, 7), dof=2, max_width=48)
    A = inputs.diffusion_3d(14, 13, 12, 21)
    return A, dict(ordering=spx.SPX_ORDER_GRID, grid=(14, 13, 12), max_width=48)


@pytest.mark.parametrize("method,prec,tol", CASES)
def test_noalloc_solve_matches_spx_solve(torch, method, prec, tol):
    A, opts = _system(method)
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, method, **opts)
    h.factorize(vals, prec)
    nrhs = 5
    B = inputs.rhs(A.shape[0], nrhs, 21)
    Bd = _colmajor(torch, B)
    X_ref, _ = h.solve(Bd, refine=spx.default_refine(mode=0))
    X_ref = X_ref.cpu().numpy()
    for call in range(2):   # the second call starts from the first call's buffer contents
        X = _noalloc(torch, h, Bd, nrhs, check_free=call == 1)
        assert np.all(np.isfinite(X))
        assert np.linalg.norm(X - X_ref) / np.linalg.norm(X_ref) <= tol
        assert h.info()["noalloc_timeout"] == 0
    h.free()


def test_noalloc_timeout_is_reported_and_does_not_carry_over(torch):
    """A wait of the allocation-free solve that runs out (a one-poll wait
    limit) is recorded for that call alone: the next call, with the default
    limit, is correct and reports no timeout, and spx_solve is not blamed."""
    g = (24, 24, 24)     # a tree with a chain of single-panel levels at the top
    A = inputs.diffusion_3d(*g, 5)
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "llt", ordering=spx.SPX_ORDER_GRID, grid=g, max_width=64)
    h.factorize(vals, "fp64")
    B = inputs.rhs(A.shape[0], 3, 5)
    Bd = _colmajor(torch, B)
    X_ref, _ = h.solve(Bd, refine=spx.default_refine(mode=0))
    X_ref = X_ref.cpu().numpy()
    h.set_wait_limit(1)
    _noalloc(torch, h, Bd, 3)
    assert h.info()["noalloc_timeout"] == 1
    h.set_wait_limit(0)
    X = _noalloc(torch, h, Bd, 3)
    assert h.info()["noalloc_timeout"] == 0
    assert np.linalg.norm(X - X_ref) / np.linalg.norm(X_ref) <= 1e-12
    X2, info = h.solve(Bd, refine=spx.default_refine(mode=0))
    assert info["status"] == "SPX_OK"
    h.free()


def test_noalloc_solve_rejects_sizes_beyond_its_buffer(torch):
    A = inputs.diffusion_3d(16, 16, 16, 3)       # n = 4096
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "llt", ordering=spx.SPX_ORDER_GRID, grid=(16, 16, 16))
    h.factorize(vals, "fp64")
    nrhs = 160                                    # 4 * 4096 * 160 * 8 bytes = 20 MiB > 16 MiB
    B = _colmajor(torch, inputs.rhs(A.shape[0], nrhs, 3))
    X = torch.empty((nrhs, A.shape[0]), dtype=torch.float64, device="cuda").t()
    st = spx.load().spx_solve_noalloc(h._h, nrhs, B.data_ptr(), A.shape[0], X.data_ptr(),
                                      A.shape[0], None)
    assert st == spx.SPX_ERR_ARG
    assert b"16 MiB" in spx.load().spx_last_error(h._h)
    h.free()
