"""Differentiation: selected inverse, log-determinant and the adjoints of the
solve, against the oracle and against dense FP64 autograd; the gradient of
w^T x + log det A with respect to the node coefficients of the 48^3
diffusion problem against central differences along 32 random directions."""
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
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [
    ("laplace2d_31", lambda: inputs.laplacian_2d(31, 31), dict(ordering=1, grid=(31, 31, 1))),
    ("diffusion_12x11x10_w24", lambda: inputs.diffusion_3d(12, 11, 10, 3),
     dict(ordering=1, grid=(12, 11, 10), max_width=24)),
    ("diffusion_17x16x15_w64", lambda: inputs.diffusion_3d(17, 16, 15, 4),
     dict(ordering=1, grid=(17, 16, 15), max_width=64)),
    ("graph_600", lambda: inputs.random_spd_graph(600, 5.0, 8), dict(ordering=2, max_width=64)),
]


@pytest.mark.parametrize("name,maker,opts", CASES, ids=[c[0] for c in CASES])
def test_selected_inverse_logdet_and_gradients_match_oracle(torch, name, maker, opts):
    A = maker()
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "llt", **opts)
    h.factorize(vals, "fp64")
    F = oracle.cholesky(A, h.perm())
    assert abs(h.logdet() - oracle.logdet(F)) <= 1e-13 * abs(oracle.logdet(F))
    h.selected_inverse()
    Z = h.selected_inverse_on_pattern(F.sym.Lp, F.sym.Li)
    assert _rel(Z, oracle.selected_inverse(F)) <= 1e-12
    g = h.logdet_grad()
    assert _rel(g, oracle.logdet_gradient(A, F)) <= 1e-12
    # adjoint of the solve, 2 right-hand sides, against oracle solves
    B = inputs.rhs(A.shape[0], 2, 7)
    G = inputs.rhs(A.shape[0], 2, 8)
    X = oracle.solve(F, B)
    Lam = oracle.solve(F, G)
    coo = A.tocsc().tocoo()
    ref = -np.einsum("er,er->e", Lam[coo.row], X[coo.col])
    assert _rel(h.solve_grad(Lam, X), ref) <= 1e-14
    h.free()


def test_logdet_closed_form_spectrum(torch):
    A = inputs.laplacian_2d(31, 31)
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "llt", ordering=1, grid=(31, 31, 1))
    h.factorize(vals, "fp64")
    i = np.arange(1, 32)
    lam = 4 - 2 * np.cos(i[:, None] * np.pi / 32) - 2 * np.cos(i[None, :] * np.pi / 32) + 0.01
    assert abs(h.logdet() - np.log(lam).sum()) <= 1e-12 * abs(np.log(lam).sum())


def test_autograd_against_dense_fp64_autograd(torch):
    from paper_1405_2636_gb300.autograd import SparseSPD

    A = inputs.diffusion_3d(4, 3, 3, 11)
    n = A.shape[0]
    cp, ri, vals = inputs.csc_arrays(A)
    op = SparseSPD(cp, ri, ordering=1, grid=(4, 3, 3))
    coo = A.tocsc().tocoo()
    rows = torch.from_numpy(coo.row.astype(np.int64)).cuda()
    cols = torch.from_numpy(coo.col.astype(np.int64)).cuda()
    g = np.random.default_rng(3)
    for nrhs in (1, 3):
        v = torch.from_numpy(vals).cuda().requires_grad_(True)
        shape = (n,) if nrhs == 1 else (n, nrhs)
        b = torch.from_numpy(g.standard_normal(shape)).cuda().requires_grad_(True)
        w = torch.from_numpy(g.standard_normal(shape)).cuda()
        loss = (w * op.solve(v, b)).sum() + op.logdet(v)
        gv, gb = torch.autograd.grad(loss, (v, b))
        v2 = torch.from_numpy(vals).cuda().requires_grad_(True)
        b2 = b.detach().clone().requires_grad_(True)
        Ad = torch.zeros(n, n, dtype=torch.float64, device="cuda").index_put((rows, cols), v2, accumulate=True)
        loss2 = (w * torch.linalg.solve(Ad, b2)).sum() + torch.logdet(Ad)
        gv2, gb2 = torch.autograd.grad(loss2, (v2, b2))
        assert abs(loss.item() - loss2.item()) <= 1e-12 * abs(loss2.item())
        assert (torch.linalg.norm(gv - gv2) / torch.linalg.norm(gv2)).item() <= 1e-10
        assert (torch.linalg.norm(gb - gb2) / torch.linalg.norm(gb2)).item() <= 1e-10
    op.free()


def test_coefficient_gradient_against_central_differences_48(torch):
    """loss(g) = w^T x + log det A(exp(g)) on the 48^3 diffusion problem;
    grad_g = exp(g) * M^T dL/dvalues against (f(g + e d) - f(g - e d)) / 2e
    along 32 random unit directions, e = 1e-2.  Relative error <= 1e-6,
    relative to the directional derivative but not below its RMS size over
    random unit directions, ||grad|| / sqrt(n): a random direction can be
    nearly orthogonal to the gradient, and there any finite difference has
    a large error relative to a near-zero value.  (The truncation error of
    the central difference is O(e^2); rounding in two 48^3 factorizations
    is ~1e-13 in f, so smaller steps lose accuracy: 3e-7 at e = 1e-4.)"""
    from paper_1405_2636_gb300.autograd import SparseSPD

    nx = ny = nz = 48
    seed = 5
    cp, ri, M = inputs.diffusion_3d_coefficient_map(nx, ny, nz)
    g0 = np.log(inputs.diffusion_3d_kappa(nx, ny, nz, seed))
    n = nx * ny * nz
    rng = np.random.default_rng([seed, 9])
    w = torch.from_numpy(rng.standard_normal(n)).cuda()
    b = torch.from_numpy(rng.standard_normal(n)).cuda()
    op = SparseSPD(cp, ri, ordering=1, grid=(nx, ny, nz), max_width=64)

    def f(g):
        v = torch.from_numpy(M @ np.exp(g)).cuda()
        return ((w * op.solve(v, b)).sum() + op.logdet(v)).item()

    v = torch.from_numpy(M @ np.exp(g0)).cuda().requires_grad_(True)
    loss = (w * op.solve(v, b)).sum() + op.logdet(v)
    (gv,) = torch.autograd.grad(loss, (v,))
    grad_g = np.exp(g0) * (M.T @ gv.cpu().numpy())
    eps = 1e-2
    scale = np.linalg.norm(grad_g) / np.sqrt(n)
    worst = 0.0
    for _ in range(32):
        d = rng.standard_normal(n)
        d /= np.linalg.norm(d)
        fd = (f(g0 + eps * d) - f(g0 - eps * d)) / (2 * eps)
        an = float(grad_g @ d)
        worst = max(worst, abs(fd - an) / max(abs(an), scale))
    assert worst <= 1e-6, worst
    op.free()
