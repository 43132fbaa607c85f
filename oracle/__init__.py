"""Oracle for the supernodal sparse factorization (Lacoste et al., Sec. III).

TEST INFRASTRUCTURE ONLY.  This package is imported by the tests, by the
smoke check and by the CPU-baseline leg of the benchmark -- never by the
product library or its Python binding.  It shares no code with the CUDA path.

The arithmetic lives in ``spx_oracle.c`` (plain C, FP64, column by column);
this module only marshals NumPy / SciPy CSC arrays to it and back.  The
helpers here that are not the method itself (permuting a matrix, the
backward-error formula, densifying a factor) are plain NumPy/SciPy.

Pins (see the ``tests/test_oracle_*.py`` files): dense Cholesky / LU by
brute force for n <= 200, ||A - L L^T||_F / ||A||_F <= 1e-14, the closed-form
Cholesky factor of the 1-D Laplacian, the closed-form spectrum of the 2-D
5-point Laplacian (log-determinant), column counts from two independent
algorithms, a hand-ordered nested dissection of small grids, a
hand-computed static-pivot replacement, and for the selected inverse the
dense inverse by brute force, the closed-form inverse of the 1-D Laplacian
and trace(A Z) = n; for LDL^T the reconstruction P A P^T = L D L^T by brute
force, Sylvester's law of inertia against dense eigenvalues, the Cholesky
factor as L sqrt(D) on SPD matrices, the closed-form LDL^T of the 1-D
Laplacian and a hand-computed static-pivot replacement; for the panel
update (Sec. V-B) a hand-computed gapped case and the Schur-complement
identity M22 - L21 L21^T = L22 L22^T of a dense Cholesky factor.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spx_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle's C file into ``liboracle.so`` next to it."""
    if force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.ora_nd_grid.argtypes = [ctypes.c_int] * 4 + [_i64p]
        lib.ora_nd_graph.argtypes = [ctypes.c_int64, _i64p, _i32p, _i64p]
        lib.ora_etree.argtypes = [ctypes.c_int64, _i64p, _i32p, _i64p]
        lib.ora_colcounts.argtypes = [ctypes.c_int64, _i64p, _i32p, _i64p, _i64p]
        lib.ora_symbolic.argtypes = [ctypes.c_int64, _i64p, _i32p, _i64p, _i32p, _i64p]
        lib.ora_cholesky.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, _i64p, _i32p, _f64p]
        lib.ora_lu.argtypes = [
            ctypes.c_int64, _i64p, _i32p, _f64p, _i64p, _i32p, ctypes.c_double,
            _f64p, _f64p, _i64p,
        ]
        lib.ora_solve_cholesky.argtypes = [
            ctypes.c_int64, _i64p, _i32p, _f64p, ctypes.c_int64, _f64p, ctypes.c_int64,
        ]
        lib.ora_solve_lu.argtypes = [
            ctypes.c_int64, _i64p, _i32p, _f64p, _f64p, ctypes.c_int64, _f64p, ctypes.c_int64,
        ]
        lib.ora_spmv.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, _f64p, _f64p]
        lib.ora_selinv.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, _f64p]
        lib.ora_ldlt.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, _i64p, _i32p, ctypes.c_double,
                                 _f64p, _i64p]
        lib.ora_solve_ldlt.argtypes = [
            ctypes.c_int64, _i64p, _i32p, _f64p, ctypes.c_int64, _f64p, ctypes.c_int64,
        ]
        _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _csc(A) -> sp.csc_matrix:
    A = sp.csc_matrix(A)
    A.sort_indices()
    return A


def _arrays(A: sp.csc_matrix):
    Ap = np.ascontiguousarray(A.indptr, dtype=np.int64)
    Ai = np.ascontiguousarray(A.indices, dtype=np.int32)
    Ax = np.ascontiguousarray(A.data, dtype=np.float64)
    return Ap, Ai, Ax


# --------------------------------------------------------------------------
# Ordering (Sec. III: nested dissection gives the permutation and the tree)
# --------------------------------------------------------------------------

def nd_grid(nx: int, ny: int, nz: int = 1, dof: int = 1) -> np.ndarray:
    """Geometric nested dissection of an nx*ny*nz grid (new -> old)."""
    n = nx * ny * nz * dof
    perm = np.empty(n, dtype=np.int64)
    rc = _load().ora_nd_grid(nx, ny, nz, dof, _p(perm, _i64p))
    if rc != 0:
        raise ValueError(f"ora_nd_grid failed ({rc})")
    return perm


def symmetrized_pattern(A) -> sp.csc_matrix:
    """Pattern of A + A^T (ones), the pattern the factorization works on."""
    A = _csc(A)
    P = (abs(A) + abs(A.T)).tocsc()
    P.data[:] = 1.0
    P = P.tocsc()
    P.sort_indices()
    return P


def nd_graph(A) -> np.ndarray:
    """Level-structure nested dissection of the graph of A + A^T."""
    P = symmetrized_pattern(A).tolil()
    P.setdiag(0)
    P = _csc(P)
    P.eliminate_zeros()
    Ap, Ai, _ = _arrays(P)
    n = P.shape[0]
    perm = np.empty(n, dtype=np.int64)
    rc = _load().ora_nd_graph(n, _p(Ap, _i64p), _p(Ai, _i32p), _p(perm, _i64p))
    if rc != 0:
        raise ValueError(f"ora_nd_graph failed ({rc})")
    return perm


def permute(A, perm: np.ndarray) -> sp.csc_matrix:
    """P A P^T with the new -> old permutation ``perm``."""
    A = _csc(A)
    return _csc(A[perm, :][:, perm])


# --------------------------------------------------------------------------
# Elimination tree, column counts, symbolic pattern
# --------------------------------------------------------------------------

def etree(Pperm) -> np.ndarray:
    """Liu's elimination tree of an already permuted symmetric pattern."""
    Ap, Ai, _ = _arrays(_csc(Pperm))
    n = len(Ap) - 1
    parent = np.empty(n, dtype=np.int64)
    _load().ora_etree(n, _p(Ap, _i64p), _p(Ai, _i32p), _p(parent, _i64p))
    return parent


def colcounts(Pperm, parent: np.ndarray) -> np.ndarray:
    Ap, Ai, _ = _arrays(_csc(Pperm))
    n = len(Ap) - 1
    count = np.empty(n, dtype=np.int64)
    parent = np.ascontiguousarray(parent, dtype=np.int64)
    _load().ora_colcounts(n, _p(Ap, _i64p), _p(Ai, _i32p), _p(parent, _i64p), _p(count, _i64p))
    return count


@dataclass
class Symbolic:
    n: int
    parent: np.ndarray      # elimination tree from Liu's algorithm
    counts: np.ndarray      # column counts from row subtrees
    Lp: np.ndarray          # column pointers of the pattern of L
    Li: np.ndarray          # sorted row indices (diagonal first)
    parent_sym: np.ndarray  # elimination tree from the pattern itself


def symbolic(Pperm) -> Symbolic:
    Pperm = _csc(Pperm)
    Ap, Ai, _ = _arrays(Pperm)
    n = Pperm.shape[0]
    parent = etree(Pperm)
    counts = colcounts(Pperm, parent)
    Lp = np.zeros(n + 1, dtype=np.int64)
    Lp[1:] = np.cumsum(counts)
    Li = np.empty(int(Lp[-1]), dtype=np.int32)
    parent_sym = np.empty(n, dtype=np.int64)
    rc = _load().ora_symbolic(
        n, _p(Ap, _i64p), _p(Ai, _i32p), _p(Lp, _i64p), _p(Li, _i32p), _p(parent_sym, _i64p)
    )
    if rc != 0:
        raise RuntimeError(f"symbolic pattern does not match column counts at column {-rc - 1}")
    return Symbolic(n, parent, counts, Lp, Li, parent_sym)


# --------------------------------------------------------------------------
# Numerical factorization and solves
# --------------------------------------------------------------------------

class NotPositiveDefinite(ArithmeticError):
    def __init__(self, col):
        super().__init__(f"non-positive pivot at permuted column {col}")
        self.col = col


@dataclass
class Factor:
    method: str              # "llt", "lu" or "ldlt"
    perm: np.ndarray         # new -> old
    sym: Symbolic
    Lx: np.ndarray           # L values in the pattern (LU: unit diagonal stored as 1; LDL^T: D on the diagonal)
    Ut: Optional[np.ndarray] = None   # LU: U transposed in L's pattern
    nrepl: int = 0           # LU: static pivot replacements
    tau: float = 0.0

    @property
    def n(self) -> int:
        return self.sym.n

    def L(self) -> sp.csc_matrix:
        s = self.sym
        return sp.csc_matrix((self.Lx, s.Li, s.Lp), shape=(s.n, s.n))

    def U(self) -> sp.csc_matrix:
        s = self.sym
        return sp.csc_matrix((self.Ut, s.Li, s.Lp), shape=(s.n, s.n)).T.tocsc()


def cholesky(A, perm: np.ndarray) -> Factor:
    """L with P A P^T = L L^T, on the given ordering."""
    A = _csc(A)
    perm = np.ascontiguousarray(perm, dtype=np.int64)
    Pa = permute(A, perm)
    s = symbolic(symmetrized_pattern(Pa))
    Ap, Ai, Ax = _arrays(Pa)
    Lx = np.zeros(int(s.Lp[-1]), dtype=np.float64)
    rc = _load().ora_cholesky(
        s.n, _p(Ap, _i64p), _p(Ai, _i32p), _p(Ax, _f64p), _p(s.Lp, _i64p), _p(s.Li, _i32p),
        _p(Lx, _f64p),
    )
    if rc != 0:
        raise NotPositiveDefinite(-rc - 1)
    return Factor("llt", perm, s, Lx)


def static_pivot_threshold(A) -> float:
    """tau = sqrt(eps) * ||A||_inf with eps = 2^-52 (reading of Sec. III)."""
    A = _csc(A)
    norm_inf = float(np.max(np.asarray(abs(A).sum(axis=1)).ravel())) if A.nnz else 0.0
    return float(np.sqrt(2.0 ** -52) * norm_inf)


def lu(A, perm: np.ndarray, tau: Optional[float] = None) -> Factor:
    """Static-pivot LU with P A P^T = L U on the pattern of A + A^T."""
    A = _csc(A)
    perm = np.ascontiguousarray(perm, dtype=np.int64)
    if tau is None:
        tau = static_pivot_threshold(A)
    Pa = permute(A, perm)
    s = symbolic(symmetrized_pattern(Pa))
    Ap, Ai, Ax = _arrays(Pa)
    nnz = int(s.Lp[-1])
    Lx = np.zeros(nnz, dtype=np.float64)
    Ut = np.zeros(nnz, dtype=np.float64)
    nrepl = np.zeros(1, dtype=np.int64)
    _load().ora_lu(
        s.n, _p(Ap, _i64p), _p(Ai, _i32p), _p(Ax, _f64p), _p(s.Lp, _i64p), _p(s.Li, _i32p),
        float(tau), _p(Lx, _f64p), _p(Ut, _f64p), _p(nrepl, _i64p),
    )
    return Factor("lu", perm, s, Lx, Ut, int(nrepl[0]), float(tau))


def ldlt(A, perm: np.ndarray, tau: Optional[float] = None) -> Factor:
    """P A P^T = L D L^T with static pivoting, unit L; Lx holds D on its diagonal."""
    A = _csc(A)
    perm = np.ascontiguousarray(perm, dtype=np.int64)
    if tau is None:
        tau = static_pivot_threshold(A)
    Pa = permute(A, perm)
    s = symbolic(symmetrized_pattern(Pa))
    Ap, Ai, Ax = _arrays(Pa)
    Lx = np.zeros(int(s.Lp[-1]), dtype=np.float64)
    nrepl = np.zeros(1, dtype=np.int64)
    rc = _load().ora_ldlt(s.n, _p(Ap, _i64p), _p(Ai, _i32p), _p(Ax, _f64p), _p(s.Lp, _i64p),
                          _p(s.Li, _i32p), float(tau), _p(Lx, _f64p), _p(nrepl, _i64p))
    if rc != 0:
        raise ZeroDivisionError(f"zero pivot in column {-rc - 1}")
    return Factor("ldlt", perm, s, Lx, None, int(nrepl[0]), float(tau))


def inertia(F: Factor) -> tuple:
    """(positive, negative) pivots of an LDL^T factor."""
    d = F.Lx[F.sym.Lp[:-1]]
    return int(np.sum(d > 0)), int(np.sum(d < 0))


def solve(F: Factor, B: np.ndarray) -> np.ndarray:
    """x with A x = b, in the original numbering (B: n or n x nrhs)."""
    B = np.asarray(B, dtype=np.float64)
    one = B.ndim == 1
    B2 = B.reshape(F.n, -1)
    X = np.asfortranarray(B2[F.perm, :])
    s = F.sym
    nrhs = X.shape[1]
    lib = _load()
    if F.method == "llt":
        lib.ora_solve_cholesky(
            s.n, _p(s.Lp, _i64p), _p(s.Li, _i32p), _p(F.Lx, _f64p), nrhs, _p(X, _f64p), s.n
        )
    elif F.method == "ldlt":
        lib.ora_solve_ldlt(
            s.n, _p(s.Lp, _i64p), _p(s.Li, _i32p), _p(F.Lx, _f64p), nrhs, _p(X, _f64p), s.n
        )
    else:
        lib.ora_solve_lu(
            s.n, _p(s.Lp, _i64p), _p(s.Li, _i32p), _p(F.Lx, _f64p), _p(F.Ut, _f64p), nrhs,
            _p(X, _f64p), s.n,
        )
    out = np.empty_like(X)
    out[F.perm, :] = X
    return out.ravel() if one else out


def logdet(F: Factor) -> float:
    """log det A = 2 sum_j log L(j, j) for a Cholesky factor."""
    if F.method != "llt":
        raise ValueError("logdet of a Cholesky factor only")
    return float(2.0 * np.sum(np.log(F.Lx[F.sym.Lp[:-1]])))


def selected_inverse(F: Factor) -> np.ndarray:
    """Entries of (P A P^T)^{-1} on the pattern of L (Takahashi recurrence)."""
    if F.method != "llt":
        raise ValueError("selected inverse of a Cholesky factor only")
    s = F.sym
    Zx = np.zeros(len(F.Lx), dtype=np.float64)
    rc = _load().ora_selinv(s.n, _p(s.Lp, _i64p), _p(s.Li, _i32p), _p(F.Lx, _f64p), _p(Zx, _f64p))
    if rc != 0:
        raise RuntimeError("pattern of L is not closed under the recurrence")
    return Zx


def logdet_gradient(A, F: Factor) -> np.ndarray:
    """d log det A / d A_ij = (A^{-1})_ji for every stored entry of A, in
    A's CSC order (entries treated as independent)."""
    A = _csc(A)
    Zx = selected_inverse(F)
    s = F.sym
    Z = sp.csc_matrix((Zx, s.Li, s.Lp), shape=(s.n, s.n))
    iperm = np.empty_like(F.perm)
    iperm[F.perm] = np.arange(len(F.perm))
    coo = A.tocoo()
    pi, pj = iperm[coo.row], iperm[coo.col]
    r, c = np.maximum(pi, pj), np.minimum(pi, pj)
    vals = np.asarray(Z[r, c]).ravel()
    out = np.empty(A.nnz)
    # tocoo of a canonical CSC keeps the CSC order
    out[:] = vals
    return out


def panel_update(A: np.ndarray, B: np.ndarray, C: np.ndarray, rowmap: np.ndarray,
                 colmap: np.ndarray, lower: bool) -> np.ndarray:
    """The supernodal update of Sec. V-B: C - A B^T subtracted at the target
    positions the block structure gives (row i of A to row rowmap[i] of C,
    row j of B to column colmap[j]); with ``lower`` only the entries with
    source row i >= facing row j (the diagonal-block region of a Cholesky
    target).  FP64: the product W = A B^T, then the scatter.  Returns a new C.
    Pinned (tests/test_oracle_update.py) by a hand-computed case and by the
    Schur-complement identity of a dense Cholesky factor."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    out = np.array(C, dtype=np.float64, copy=True)
    W = A @ B.T
    for j in range(B.shape[0]):
        i0 = j if lower else 0
        out[rowmap[i0:], colmap[j]] -= W[i0:, j]
    return out


def spmv(A, x: np.ndarray) -> np.ndarray:
    A = _csc(A)
    Ap, Ai, Ax = _arrays(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(A.shape[0], dtype=np.float64)
    _load().ora_spmv(A.shape[0], _p(Ap, _i64p), _p(Ai, _i32p), _p(Ax, _f64p), _p(x, _f64p),
                     _p(y, _f64p))
    return y


# --------------------------------------------------------------------------
# Metrics (readings stated in the design notes; not printed in the paper)
# --------------------------------------------------------------------------

def flops(counts: np.ndarray, method: str = "llt") -> float:
    """Factorization flops counted from the exact symbolic structure.

    Cholesky: sum_j c_j^2; LU: sum_j 2 (c_j - 1)^2 + (c_j - 1), with c_j the
    column count including the diagonal (Table I reports flops this way).
    """
    c = np.asarray(counts, dtype=np.float64)
    if method == "llt":
        return float(np.sum(c * c))
    return float(np.sum(2.0 * (c - 1.0) ** 2 + (c - 1.0)))


def backward_error(A, X: np.ndarray, B: np.ndarray) -> float:
    """max over right-hand sides of ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)."""
    A = _csc(A)
    X = np.asarray(X, dtype=np.float64).reshape(A.shape[0], -1)
    B = np.asarray(B, dtype=np.float64).reshape(A.shape[0], -1)
    norm_a = float(np.max(np.asarray(abs(A).sum(axis=1)).ravel()))
    worst = 0.0
    for c in range(X.shape[1]):
        r = B[:, c] - spmv(A, X[:, c])
        den = norm_a * np.max(np.abs(X[:, c])) + np.max(np.abs(B[:, c]))
        worst = max(worst, float(np.max(np.abs(r)) / den) if den > 0 else 0.0)
    return worst
