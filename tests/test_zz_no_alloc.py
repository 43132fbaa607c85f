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


def _noalloc(torch, h, Bd, nrhs):
    n = h.n
    Xd = torch.full((nrhs, n), float("nan"), dtype=torch.float64, device="cuda").t()
    st = spx.load().spx_solve_noalloc(h._h, nrhs, Bd.data_ptr(), n, Xd.data_ptr(), n, None)
    assert st == spx.SPX_OK, spx.load().spx_last_error(h._h)
    torch.cuda.synchronize()
    return Xd.cpu().numpy()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_noalloc_solve_matches_spx_solve(torch, prec, tol):
    A = inputs.diffusion_3d(14, 13, 12, 21)
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "llt", ordering=spx.SPX_ORDER_GRID, grid=(14, 13, 12), max_width=48)
    h.factorize(vals, prec)
    nrhs = 5
    B = inputs.rhs(A.shape[0], nrhs, 21)
    Bd = _colmajor(torch, B)
    X_ref, _ = h.solve(Bd, refine=spx.default_refine(mode=0))
    X_ref = X_ref.cpu().numpy()
    for _ in range(2):   # the second call starts from the first call's buffer contents
        X = _noalloc(torch, h, Bd, nrhs)
        assert np.all(np.isfinite(X))
        assert np.linalg.norm(X - X_ref) / np.linalg.norm(X_ref) <= tol
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
