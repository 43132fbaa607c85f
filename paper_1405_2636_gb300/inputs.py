"""Seeded synthetic workloads for the supernodal factorization.

This module only draws random numbers and assembles test matrices; it holds
none of the factorization's arithmetic.  Both the oracle-based tests and the
GPU path consume what it produces, so it lives on its own.

The paper measures on SuiteSparse matrices (Table I) that are not available
here; these seeded PDE matrices stand in for them at comparable scale
(n ~ 1e5, nnz(L) ~ 1e8, 0.1-1 TFlop).

Every generator returns a ``scipy.sparse.csc_matrix`` with sorted row indices
and the full (both triangles) pattern.  Grid node (x, y, z) has index
x + nx * (y + ny * z); with several dof per node, unknown = node * dof + d.
All random draws use NumPy's PCG64 through ``np.random.default_rng([seed,
stream])`` so that matrix values and right-hand sides are independent streams.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import numpy as np
import scipy.sparse as sp

STREAM_MATRIX = 0
STREAM_RHS = 1
STREAM_EXTRA = 2


def rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream)])


def _finish(rows, cols, vals, n) -> sp.csc_matrix:
    A = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsc()
    A.sum_duplicates()
    A.sort_indices()
    return A


def _node_index(nx, ny, nz):
    return np.arange(nx * ny * nz, dtype=np.int64).reshape(nz, ny, nx)


def laplacian_2d(nx: int, ny: int, shift: float = 1e-2) -> sp.csc_matrix:
    """Dirichlet 5-point Laplacian (4 on the diagonal, -1 to each neighbour) + shift*I."""
    return laplacian_3d(nx, ny, 1, shift=shift, two_d=True)


def laplacian_3d(nx: int, ny: int, nz: int, shift: float = 0.0, two_d: bool = False) -> sp.csc_matrix:
    """Dirichlet 7-point (or 5-point when two_d) Laplacian + shift*I."""
    idx = _node_index(nx, ny, nz)
    n = nx * ny * nz
    rows, cols, vals = [], [], []
    diag = (4.0 if two_d else 6.0) + shift
    rows.append(idx.ravel()); cols.append(idx.ravel()); vals.append(np.full(n, diag))
    for ax in ((2, 1) if two_d else (2, 1, 0)):
        a = np.take(idx, np.arange(idx.shape[ax] - 1), axis=ax).ravel()
        b = np.take(idx, np.arange(1, idx.shape[ax]), axis=ax).ravel()
        rows += [a, b]; cols += [b, a]; vals += [np.full(a.size, -1.0)] * 2
    return _finish(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), n)


def diffusion_3d(nx: int, ny: int, nz: int, seed: int, sigma: float = 1.0) -> sp.csc_matrix:
    """7-point variable-coefficient diffusion, node coefficients exp(sigma g), g ~ N(0,1).

    Face coefficient between neighbours i, j is (k_i + k_j) / 2; a missing
    neighbour (Dirichlet boundary) adds k_i to the diagonal; grid spacing 1.
    sigma > 1 gives the high-contrast variants used to exercise refinement.
    """
    n = nx * ny * nz
    kappa = np.exp(sigma * rng(seed, STREAM_MATRIX).standard_normal(n))
    idx = _node_index(nx, ny, nz)
    diag = np.zeros(n)
    rows, cols, vals = [], [], []
    for ax in (2, 1, 0):
        a = np.take(idx, np.arange(idx.shape[ax] - 1), axis=ax).ravel()
        b = np.take(idx, np.arange(1, idx.shape[ax]), axis=ax).ravel()
        c = 0.5 * (kappa[a] + kappa[b])
        rows += [a, b]; cols += [b, a]; vals += [-c, -c]
        np.add.at(diag, a, c)
        np.add.at(diag, b, c)
        lo = np.take(idx, [0], axis=ax).ravel()
        hi = np.take(idx, [idx.shape[ax] - 1], axis=ax).ravel()
        np.add.at(diag, lo, kappa[lo])
        np.add.at(diag, hi, kappa[hi])
    rows.append(np.arange(n)); cols.append(np.arange(n)); vals.append(diag)
    return _finish(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), n)


def quasi_definite_3d(nx: int, ny: int, nz: int, seed: int, shift: float = 0.1) -> sp.csc_matrix:
    """Symmetric indefinite, quasi-definite: two unknowns per grid node (u, p),
    [[K, B^T], [B, -C]] interleaved node by node (unknown 2 a is u_a, 2 a + 1
    is p_a), K the 7-point diffusion operator of this seed, C = shift x the
    diffusion operator of seed + 1, and B ~ U(-0.5, 0.5) on the 7-point
    stencil.  Every symmetric ordering of it has an LDL^T factorization
    without pivoting, with n/2 positive and n/2 negative pivots."""
    K = diffusion_3d(nx, ny, nz, seed).tocoo()
    C = diffusion_3d(nx, ny, nz, seed + 1).tocoo()
    g = rng(seed, STREAM_EXTRA)
    bvals = g.uniform(-0.5, 0.5, size=K.nnz)
    n = 2 * nx * ny * nz
    rows = np.concatenate([2 * K.row, 2 * C.row + 1, 2 * K.row + 1, 2 * K.col])
    cols = np.concatenate([2 * K.col, 2 * C.col + 1, 2 * K.col, 2 * K.row + 1])
    vals = np.concatenate([K.data, -shift * C.data, bvals, bvals])
    return _finish(rows, cols, vals, n)


def diffusion_3d_kappa(nx: int, ny: int, nz: int, seed: int, sigma: float = 1.0) -> np.ndarray:
    """The node coefficients exp(sigma g) that diffusion_3d draws for this seed."""
    return np.exp(sigma * rng(seed, STREAM_MATRIX).standard_normal(nx * ny * nz))


def diffusion_3d_coefficient_map(nx: int, ny: int, nz: int):
    """The values of diffusion_3d are linear in the node coefficients kappa:
    returns (colptr, rowind, M) with the CSC pattern of diffusion_3d and a
    sparse M (nnz x n) such that its values are M @ kappa."""
    n = nx * ny * nz
    idx = _node_index(nx, ny, nz)
    R, C, node, coef = [], [], [], []

    def add(r, c, m, v):
        R.append(r); C.append(c); node.append(m); coef.append(np.full(r.size, v))

    for ax in (2, 1, 0):
        a = np.take(idx, np.arange(idx.shape[ax] - 1), axis=ax).ravel()
        b = np.take(idx, np.arange(1, idx.shape[ax]), axis=ax).ravel()
        for (r, c) in ((a, b), (b, a)):
            add(r, c, a, -0.5); add(r, c, b, -0.5)
        for r in (a, b):
            add(r, r, a, 0.5); add(r, r, b, 0.5)
        lo = np.take(idx, [0], axis=ax).ravel()
        hi = np.take(idx, [idx.shape[ax] - 1], axis=ax).ravel()
        add(lo, lo, lo, 1.0); add(hi, hi, hi, 1.0)
    R = np.concatenate(R); C = np.concatenate(C)
    key = C * n + R
    uniq = np.unique(key)
    pos = np.searchsorted(uniq, key)
    M = sp.csr_matrix((np.concatenate(coef), (pos, np.concatenate(node))), shape=(uniq.size, n))
    M.sum_duplicates()
    rowind = (uniq % n).astype(np.int32)
    colptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(uniq // n, minlength=n), out=colptr[1:])
    return colptr, rowind, M


def _haar_rotations(g: np.random.Generator, count: int) -> np.ndarray:
    """count x 3 x 3 rotations: QR of a Gaussian, signs fixed, det +1."""
    z = g.standard_normal((count, 3, 3))
    q, r = np.linalg.qr(z)
    s = np.sign(np.diagonal(r, axis1=1, axis2=2))
    s[s == 0] = 1.0
    q = q * s[:, None, :]
    det = np.linalg.det(q)
    q[det < 0, :, 2] *= -1.0
    return q


def elasticity_27pt(nx: int, ny: int, nz: int, seed: int) -> sp.csc_matrix:
    """27-point stencil, 3 dof per node, SPD 3x3 coupling blocks.

    For every pair of 27-point neighbours (i, j), K_ij = R diag(mu) R^T with
    mu ~ logU[1, 1e3] and R a Haar rotation; the pair contributes
    [K -K; -K K].  A neighbour outside the box adds its K to the diagonal
    block of i (Dirichlet), which makes the matrix positive definite.
    """
    g = rng(seed, STREAM_MATRIX)
    nn = nx * ny * nz
    idx = _node_index(nx, ny, nz)
    coords = np.stack(np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij"), -1)
    coords = coords.reshape(-1, 3)  # (z, y, x) per node index
    offsets = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
               if (dz, dy, dx) > (0, 0, 0)]
    dims = np.array([nz, ny, nx])
    ii, jj, bnd = [], [], []
    for off in offsets:
        o = np.array(off)
        nb = coords + o
        inside = np.all((nb >= 0) & (nb < dims), axis=1)
        src = np.nonzero(inside)[0]
        dst = (nb[inside, 2] + nx * (nb[inside, 1] + ny * nb[inside, 0])).astype(np.int64)
        ii.append(src); jj.append(dst)
        # missing neighbours in direction +off and -off are Dirichlet couplings
        bnd.append(np.nonzero(~inside)[0])
        nbm = coords - o
        insm = np.all((nbm >= 0) & (nbm < dims), axis=1)
        bnd.append(np.nonzero(~insm)[0])
    ii = np.concatenate(ii); jj = np.concatenate(jj); bnd = np.concatenate(bnd)
    npair = ii.size
    nb_ = bnd.size
    mu = np.exp(g.uniform(0.0, np.log(1e3), size=(npair + nb_, 3)))
    R = _haar_rotations(g, npair + nb_)
    K = np.einsum("pik,pk,pjk->pij", R, mu, R)
    Kp, Kb = K[:npair], K[npair:]
    d3 = np.arange(3)
    rr, cc = np.meshgrid(d3, d3, indexing="ij")
    rr = rr.ravel(); cc = cc.ravel()
    rows, cols, vals = [], [], []

    def add(a, b, blocks, sign):
        rows.append((3 * a[:, None] + rr[None, :]).ravel())
        cols.append((3 * b[:, None] + cc[None, :]).ravel())
        vals.append(sign * blocks.reshape(-1, 9).ravel())

    add(ii, ii, Kp, 1.0); add(jj, jj, Kp, 1.0)
    add(ii, jj, Kp, -1.0); add(jj, ii, Kp, -1.0)
    add(bnd, bnd, Kb, 1.0)
    del idx
    return _finish(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), 3 * nn)


def convection_diffusion_2d(k: int, seed: int) -> Tuple[sp.csc_matrix, dict]:
    """-Laplace(u) + w . grad(u) on the unit square, k x k interior nodes.

    First-order upwind, h = 1/(k+1), nu = 1, Dirichlet; w = |w| (cos t, sin t)
    with t ~ U[0, 2 pi) and mesh Peclet |w| h / 2 ~ U(0, 10).  Rows are scaled
    by h^2.  Values are unsymmetric, the pattern is symmetric.
    """
    g = rng(seed, STREAM_MATRIX)
    theta = g.uniform(0.0, 2 * np.pi)
    pe = g.uniform(0.0, 10.0)
    h = 1.0 / (k + 1)
    wmag = 2.0 * pe / h
    wx, wy = wmag * np.cos(theta), wmag * np.sin(theta)
    idx = _node_index(k, k, 1)[0]
    n = k * k
    rows, cols, vals = [], [], []
    rows.append(idx.ravel()); cols.append(idx.ravel())
    vals.append(np.full(n, 4.0 + h * (abs(wx) + abs(wy))))
    for ax, w in ((1, wx), (0, wy)):
        a = np.take(idx, np.arange(k - 1), axis=ax).ravel()       # left/below
        b = np.take(idx, np.arange(1, k), axis=ax).ravel()        # right/above
        # row b couples to its lower neighbour a; row a to its upper neighbour b
        rows += [b, a]; cols += [a, b]
        vals += [np.full(a.size, -1.0 - h * max(w, 0.0)), np.full(a.size, -1.0 - h * max(-w, 0.0))]
    A = _finish(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), n)
    return A, {"theta": theta, "peclet": pe, "h": h}


def random_spd_graph(n: int, avg_degree: float, seed: int) -> sp.csc_matrix:
    """Random symmetric pattern, strictly diagonally dominant SPD values."""
    g = rng(seed, STREAM_MATRIX)
    m = int(n * avg_degree / 2)
    a = g.integers(0, n, size=m)
    b = g.integers(0, n, size=m)
    keep = a != b
    a, b = a[keep], b[keep]
    v = -g.uniform(0.1, 1.0, size=a.size)
    rows = np.concatenate([a, b]); cols = np.concatenate([b, a]); vals = np.concatenate([v, v])
    A = _finish(rows, cols, vals, n)
    d = np.asarray(abs(A).sum(axis=1)).ravel() + 1.0
    return (A + sp.diags(d)).tocsc()


def rhs(n: int, nrhs: int, seed: int) -> np.ndarray:
    """n x nrhs right-hand sides ~ U(-1, 1), Fortran order (column-major)."""
    return np.asfortranarray(rng(seed, STREAM_RHS).uniform(-1.0, 1.0, size=(nrhs, n)).T)


def csc_arrays(A: sp.csc_matrix):
    """(colptr int64, rowind int32, values float64) of a CSC matrix."""
    A = sp.csc_matrix(A)
    A.sort_indices()
    return (np.ascontiguousarray(A.indptr, dtype=np.int64),
            np.ascontiguousarray(A.indices, dtype=np.int32),
            np.ascontiguousarray(A.data, dtype=np.float64))


@dataclass(frozen=True)
class Workload:
    """A named matrix with its grid (for the geometric ordering) and RHS count."""
    name: str
    grid: Tuple[int, int, int]
    dof: int
    nrhs: int
    seed: int

    def matrix(self) -> sp.csc_matrix:
        nx, ny, nz = self.grid
        if self.name.startswith("laplace2d"):
            return laplacian_2d(nx, ny, 1e-2)
        if self.name.startswith("diffusion3d"):
            return diffusion_3d(nx, ny, nz, self.seed)
        if self.name.startswith("elasticity27"):
            return elasticity_27pt(nx, ny, nz, self.seed)
        raise KeyError(self.name)

    def rhs(self, n: int) -> np.ndarray:
        return rhs(n, self.nrhs, self.seed)


# The workloads: 2-D 5-point Laplacian 31x31 (+1e-2 I), the 64^3 7-point
# variable-coefficient diffusion with 16 right-hand sides, and the 40^3
# 27-point 3-dof elasticity-like system.
LAPLACE2D_31 = Workload("laplace2d_31x31", (31, 31, 1), 1, 1, 1)
DIFFUSION3D_64 = Workload("diffusion3d_64^3", (64, 64, 64), 1, 16, 2)
ELASTICITY27_40 = Workload("elasticity27_40^3x3", (40, 40, 40), 3, 1, 3)


def batched_sides(count: int, seed: int, k_lo: int = 12, k_hi: int = 80) -> List[int]:
    """Grid side of each system of the batched workload, k ~ U{k_lo..k_hi}."""
    return [int(k) for k in rng(seed, STREAM_EXTRA).integers(k_lo, k_hi + 1, size=count)]


def batched_convection_diffusion(count: int, seed: int, k_lo: int = 12, k_hi: int = 80,
                                 systems: Optional[Sequence[int]] = None):
    """The batched workload: ``count`` independent 2-D convection-diffusion
    systems, side k ~ U{k_lo..k_hi} per system (n = k^2), each with its own
    wind angle and mesh Peclet number and one right-hand side ~ U(-1, 1).

    System s draws from seed ``seed * 1_000_003 + s``, so a subset
    (``systems``: indices in any order; all by default) holds the same
    systems as the whole batch.  Returns (list of csc matrices, list of
    sides, concatenated right-hand sides), in the order of ``systems``.
    """
    sides = batched_sides(count, seed, k_lo, k_hi)
    idx = range(count) if systems is None else systems
    mats, rhss, ks = [], [], []
    for s in idx:
        if not 0 <= s < count:
            raise ValueError(f"system {s} outside 0..{count - 1}")
        k = sides[s]
        sseed = seed * 1_000_003 + s
        A, _ = convection_diffusion_2d(k, sseed)
        mats.append(A)
        ks.append(k)
        rhss.append(rhs(A.shape[0], 1, sseed).ravel())
    return mats, ks, (np.concatenate(rhss) if rhss else np.zeros(0))


BATCHED_CD_4096 = {"name": "batched_convdiff2d_4096x_k12-80", "count": 4096, "seed": 4}


def gapped_update_case(m: int, k: int, nb: int, seed: int, avg_block: int = 200):
    """The kernel-study input of Sec. V-B: C = C - A B^T with B the first nb rows
    of A; C is a panel twice as tall as A whose rows are cut into random blocks
    of about ``avg_block`` rows; A's rows come in blocks that each lie inside
    one block of C, without overlap.

    Returns (A m x k column-major, C hc x nc column-major, rowmap int32[m],
    colmap int32[nb]) as NumPy arrays.
    """
    g = rng(seed, STREAM_EXTRA)
    hc = 2 * m
    # C blocks: random sizes in [1, 2*avg-1] until they cover hc rows
    cuts = [0]
    while cuts[-1] < hc:
        cuts.append(min(hc, cuts[-1] + int(g.integers(1, 2 * avg_block))))
    cblocks = list(zip(cuts[:-1], cuts[1:]))
    # A blocks: walk C blocks in order, take a random sub-interval of each
    # until m rows are placed (rows stay increasing, blocks never overlap)
    rowmap = []
    while len(rowmap) < m:
        for (a, b) in cblocks:
            if len(rowmap) >= m:
                break
            if g.random() < 0.5:
                continue
            size = min(b - a, m - len(rowmap))
            take = int(g.integers(1, size + 1))
            start = a + int(g.integers(0, (b - a) - take + 1))
            rowmap.extend(range(start, start + take))
        rowmap = sorted(set(rowmap))[:m]
    rowmap = np.asarray(rowmap[:m], dtype=np.int32)
    nc = max(nb, int(np.ceil(nb * 1.5)))
    colmap = np.sort(g.choice(nc, size=nb, replace=False)).astype(np.int32)
    A = np.asfortranarray(g.standard_normal((m, k)))
    C = np.asfortranarray(g.standard_normal((hc, nc)))
    return A, C, rowmap, colmap
