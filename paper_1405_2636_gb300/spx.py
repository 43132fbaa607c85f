"""Thin ctypes binding of libspx (include/spx.h).

Argument marshalling only: every step of the factorization and the solves
runs in the library's CUDA kernels.  Device arrays are passed as PyTorch CUDA
tensors (their data pointers); host arrays as NumPy arrays.  There is no CPU
fallback: if ``libspx.so`` is missing or no sm_103 GPU is present, calls fail
loudly.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspx.so")

SPX_OK, SPX_ERR_ARG, SPX_ERR_ALLOC, SPX_ERR_CUDA, SPX_ERR_NOT_SPD = 0, 1, 2, 3, 4
SPX_ERR_ZERO_PIVOT, SPX_ERR_TIMEOUT, SPX_ERR_NOT_CONVERGED, SPX_ERR_STATE = 5, 6, 7, 8
SPX_LLT, SPX_LU, SPX_LDLT = 0, 1, 2
METHODS = {"llt": SPX_LLT, "lu": SPX_LU, "ldlt": SPX_LDLT}
SPX_FP64, SPX_FP32, SPX_TF32, SPX_BF16 = 0, 1, 2, 3
SPX_ORDER_AUTO, SPX_ORDER_GRID, SPX_ORDER_GRAPH, SPX_ORDER_GIVEN, SPX_ORDER_NATURAL = 0, 1, 2, 3, 4

PRECISIONS = {"fp64": SPX_FP64, "fp32": SPX_FP32, "tf32": SPX_TF32, "bf16": SPX_BF16}
STATUS_NAMES = {0: "SPX_OK", 1: "SPX_ERR_ARG", 2: "SPX_ERR_ALLOC", 3: "SPX_ERR_CUDA",
                4: "SPX_ERR_NOT_SPD", 5: "SPX_ERR_ZERO_PIVOT", 6: "SPX_ERR_TIMEOUT",
                7: "SPX_ERR_NOT_CONVERGED", 8: "SPX_ERR_STATE"}

# Every symbol include/spx.h declares.
EXPORTED = ["spx_default_options", "spx_default_refine", "spx_analyze", "spx_factorize",
            "spx_solve", "spx_get_info", "spx_get_perm", "spx_get_factor", "spx_last_error",
            "spx_free", "spx_set_profiling", "spx_get_kernel_stats",
            "spx_get_panels", "spx_solve_noalloc", "spx_set_wait_limit", "spx_roofline_model",
            "spx_update_create", "spx_update_stage", "spx_update_run", "spx_update_get_info",
            "spx_update_last_error", "spx_update_free",
            "spx_partition", "spx_factorize_part", "spx_part_get", "spx_part_set",
            "spx_batch_analyze", "spx_batch_run", "spx_batch_tune", "spx_batch_set_config",
            "spx_batch_get_info", "spx_batch_system_info", "spx_batch_get_perm",
            "spx_batch_get_factor", "spx_batch_last_error", "spx_batch_free",
            "spx_logdet", "spx_selected_inverse", "spx_get_selected_inverse", "spx_logdet_grad",
            "spx_solve_grad"]


class spx_options(ctypes.Structure):
    _fields_ = [("ordering", ctypes.c_int32), ("grid", ctypes.c_int32 * 3),
                ("dof", ctypes.c_int32), ("max_width", ctypes.c_int32),
                ("amalg_ratio", ctypes.c_double), ("perm", ctypes.POINTER(ctypes.c_int64)),
                ("lower_only", ctypes.c_int32), ("queue_panels", ctypes.c_int32),
                ("pivot_tau", ctypes.c_double), ("deterministic", ctypes.c_int32),
                ("reserved1", ctypes.c_int32)]


class spx_refine(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("gmres_restart", ctypes.c_int32),
                ("gmres_max_iter", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("tol", ctypes.c_double)]


class spx_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("gmres_iters", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("backward_error", ctypes.c_double)]


class spx_info(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "n", "nnz_a", "nnz_l", "nnz_stored", "factor_bytes", "nsupernodes", "npanels",
        "nlevels", "nupdates", "bad_col", "npivot_repl")] + [
        ("method", ctypes.c_int32), ("precision", ctypes.c_int32)] + [
        (name, ctypes.c_double) for name in ("flops", "flops_stored", "update_flops")] + [
        ("launches_factor", ctypes.c_int64), ("launches_solve", ctypes.c_int64)] + [
        (name, ctypes.c_double) for name in ("analyze_ms", "factor_ms", "solve_ms")] + [
        ("npivot_neg", ctypes.c_int64), ("noalloc_timeout", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


KERNEL_CLASSES = ["assemble", "diag", "trsm", "update", "update_tc", "queue"]
_NK = len(KERNEL_CLASSES)


class spx_kernel_stats(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * _NK), ("launches", ctypes.c_int64 * _NK),
                ("flops", ctypes.c_double * _NK), ("bytes", ctypes.c_double * _NK)]

    def as_dict(self) -> dict:
        return {c: {"ms": self.ms[i], "launches": self.launches[i], "flops": self.flops[i],
                    "bytes": self.bytes[i]} for i, c in enumerate(KERNEL_CLASSES)}


class spx_batch_info(ctypes.Structure):
    _fields_ = [("nsys", ctypes.c_int32), ("nclasses", ctypes.c_int32)] + [
        (name, ctypes.c_int64) for name in ("n_total", "n_max", "nnz_total", "nnz_l_total",
                                            "factor_elems")] + [
        ("flops", ctypes.c_double)] + [
        (name, ctypes.c_int32) for name in ("precision", "ctas_per_sm", "leaf_width",
                                            "rows_per_thread")] + [
        (name, ctypes.c_double) for name in ("tuned_ms", "analyze_ms", "run_ms")] + [
        ("max_pivot_repl", ctypes.c_int64), ("not_converged", ctypes.c_int32),
        ("max_iters", ctypes.c_int32), ("max_backward_error", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64


def load():
    """Load libspx.so (built in-tree by ``build.build()``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run paper_1405_2636_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    lib.spx_default_options.argtypes = [ctypes.POINTER(spx_options)]
    lib.spx_default_options.restype = None
    lib.spx_default_refine.argtypes = [ctypes.POINTER(spx_refine)]
    lib.spx_default_refine.restype = None
    lib.spx_analyze.argtypes = [_i64, _vp, _vp, ctypes.c_int, ctypes.POINTER(spx_options),
                                ctypes.POINTER(_vp)]
    lib.spx_factorize.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp]
    lib.spx_solve.argtypes = [_vp, ctypes.c_int32, _vp, _i64, _vp, _i64, ctypes.c_int,
                              ctypes.POINTER(spx_refine), ctypes.POINTER(spx_solve_info), _vp]
    lib.spx_get_info.argtypes = [_vp, ctypes.POINTER(spx_info)]
    lib.spx_get_perm.argtypes = [_vp, _vp]
    lib.spx_get_factor.argtypes = [_vp, _vp, _vp, _vp, _vp]
    lib.spx_last_error.argtypes = [_vp]
    lib.spx_last_error.restype = ctypes.c_char_p
    lib.spx_set_profiling.argtypes = [_vp, ctypes.c_int]
    lib.spx_get_kernel_stats.argtypes = [_vp, ctypes.POINTER(spx_kernel_stats)]
    lib.spx_get_panels.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
    lib.spx_solve_noalloc.argtypes = [_vp, ctypes.c_int32, _vp, _i64, _vp, _i64, _vp]
    lib.spx_free.argtypes = [_vp]
    lib.spx_free.restype = None
    lib.spx_set_wait_limit.argtypes = [_vp, _i64]
    lib.spx_partition.argtypes = [_vp, ctypes.c_int32, _vp, _vp, _vp]
    lib.spx_factorize_part.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int32, _vp]
    lib.spx_part_get.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp]
    lib.spx_part_set.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp]
    lib.spx_roofline_model.argtypes = [_vp, ctypes.c_int, _vp, _vp]
    lib.spx_update_create.argtypes = [_i64, _i64, _i64, _i64, _i64, _vp, _vp, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)]
    lib.spx_update_stage.argtypes = [_vp, _vp, _vp, _i64, _vp]
    lib.spx_update_run.argtypes = [_vp, _vp, ctypes.c_int, _vp]
    lib.spx_update_get_info.argtypes = [_vp, _vp, _vp]
    lib.spx_update_last_error.argtypes = [_vp]
    lib.spx_update_last_error.restype = ctypes.c_char_p
    lib.spx_update_free.argtypes = [_vp]
    lib.spx_update_free.restype = None
    lib.spx_batch_analyze.argtypes = [ctypes.c_int32, _vp, _vp, _vp, _vp, ctypes.POINTER(spx_options),
                                      ctypes.POINTER(_vp)]
    lib.spx_batch_run.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int,
                                  ctypes.POINTER(spx_refine), _vp]
    lib.spx_batch_tune.argtypes = lib.spx_batch_run.argtypes
    lib.spx_batch_set_config.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    lib.spx_batch_get_info.argtypes = [_vp, ctypes.POINTER(spx_batch_info)]
    lib.spx_batch_system_info.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
    lib.spx_batch_get_perm.argtypes = [_vp, ctypes.c_int32, _vp]
    lib.spx_batch_get_factor.argtypes = [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp]
    lib.spx_batch_last_error.argtypes = [_vp]
    lib.spx_batch_last_error.restype = ctypes.c_char_p
    lib.spx_logdet.argtypes = [_vp, ctypes.POINTER(ctypes.c_double)]
    lib.spx_selected_inverse.argtypes = [_vp, _vp]
    lib.spx_get_selected_inverse.argtypes = [_vp, _vp, _vp, _vp]
    lib.spx_logdet_grad.argtypes = [_vp, _vp, ctypes.c_int, _vp]
    lib.spx_solve_grad.argtypes = [_vp, ctypes.c_int32, _vp, _i64, _vp, _i64, _vp, ctypes.c_int, _vp]
    lib.spx_batch_free.argtypes = [_vp]
    lib.spx_batch_free.restype = None
    for name in ("spx_analyze", "spx_factorize", "spx_solve", "spx_get_info", "spx_get_perm",
                 "spx_get_factor", "spx_set_profiling", "spx_get_kernel_stats",
                 "spx_get_panels", "spx_solve_noalloc", "spx_set_wait_limit", "spx_roofline_model",
                 "spx_update_create",
                 "spx_update_stage", "spx_update_run", "spx_update_get_info",
                 "spx_partition", "spx_factorize_part", "spx_part_get", "spx_part_set",
                 "spx_batch_analyze", "spx_batch_run",
                 "spx_batch_tune", "spx_batch_set_config", "spx_batch_get_info",
                 "spx_batch_system_info", "spx_batch_get_perm", "spx_batch_get_factor",
                 "spx_logdet", "spx_selected_inverse", "spx_get_selected_inverse",
                 "spx_logdet_grad", "spx_solve_grad"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class SpxError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _check(status: int, handle=None):
    if status != SPX_OK:
        msg = load().spx_last_error(handle)
        raise SpxError(status, msg.decode() if msg else "")


def _ptr(a) -> int:
    """Data pointer of a NumPy array or a torch tensor."""
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _is_device(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


def default_options(**kw) -> spx_options:
    o = spx_options()
    load().spx_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if k == "grid":
            for i, g in enumerate(list(v) + [1] * (3 - len(v))):
                o.grid[i] = int(g)
        elif k == "perm":
            continue
        else:
            setattr(o, k, v)
    return o


def default_refine(**kw) -> spx_refine:
    r = spx_refine()
    load().spx_default_refine(ctypes.byref(r))
    for k, v in kw.items():
        setattr(r, k, v)
    return r


class Handle:
    """An analysed pattern and (after ``factorize``) its device-resident factor."""

    def __init__(self, raw: int, n: int, nnz: int):
        self._h = raw
        self.n = n
        self.nnz = nnz

    # -- lifecycle -----------------------------------------------------------
    def free(self):
        if self._h:
            load().spx_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    # -- calls -----------------------------------------------------------------
    def factorize(self, values, precision="fp64", stream=None):
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        if not _is_device(values):
            values = np.ascontiguousarray(values, dtype=np.float64)
        st = load().spx_factorize(self._h, _ptr(values), 1 if _is_device(values) else 0, prec,
                                  _stream_ptr(stream))
        _check(st, self._h)

    def solve(self, B, X=None, refine=None, stream=None) -> tuple:
        """Solve A X = B.  B: (n,) or (n, nrhs), column-major host array or a
        CUDA tensor laid out column-major (i.e. ``B.t().contiguous().t()``)."""
        dev = _is_device(B)
        if dev:
            one = B.dim() == 1
            nrhs = 1 if one else B.shape[1]
            ldb = self.n if one else B.stride(1)
            if X is None:
                import torch
                X = torch.empty((nrhs, self.n), dtype=torch.float64, device=B.device).t() \
                    if not one else torch.empty(self.n, dtype=torch.float64, device=B.device)
            ldx = self.n if one else X.stride(1)
        else:
            B = np.asfortranarray(B, dtype=np.float64)
            one = B.ndim == 1
            nrhs = 1 if one else B.shape[1]
            ldb = self.n
            if X is None:
                X = np.empty_like(B, order="F")
            ldx = self.n
        info = spx_solve_info()
        rptr = ctypes.byref(refine) if refine is not None else None
        st = load().spx_solve(self._h, nrhs, _ptr(B), ldb, _ptr(X), ldx, 1 if dev else 0, rptr,
                              ctypes.byref(info), _stream_ptr(stream))
        if st not in (SPX_OK, SPX_ERR_NOT_CONVERGED):
            _check(st, self._h)
        return X, {"iters": info.iters, "gmres_iters": info.gmres_iters,
                   "converged": bool(info.converged), "backward_error": info.backward_error,
                   "status": STATUS_NAMES[st]}

    def info(self) -> dict:
        i = spx_info()
        _check(load().spx_get_info(self._h, ctypes.byref(i)), self._h)
        return i.as_dict()

    def roofline_model(self, precision: str, hbm_gbs: float, fp64_gflops: float, fp32_gflops: float,
                       tensor_gflops: float) -> dict:
        """Per kernel class, the summed per-task roofline time (ms) of the
        factorization in ``precision`` (spx_roofline_model)."""
        peaks = np.array([hbm_gbs, fp64_gflops, fp32_gflops, tensor_gflops], dtype=np.float64)
        out = np.zeros(len(KERNEL_CLASSES), dtype=np.float64)
        _check(load().spx_roofline_model(self._h, PRECISIONS[precision], _ptr(peaks), _ptr(out)), self._h)
        return {c: float(out[i]) for i, c in enumerate(KERNEL_CLASSES)}

    # -- subtree-to-rank distribution with fan-in --------------------------------
    def partition(self, nranks: int) -> dict:
        """spx_partition: owner rank of every panel (-1: the top, factored by
        rank 0 after the fan-in) and the packed sizes of every part (index
        nranks: the top)."""
        npn = self.info()["npanels"]
        owner = np.empty(npn, np.int32)
        vals = np.empty(nranks + 1, np.int64)
        invs = np.empty(nranks + 1, np.int64)
        _check(load().spx_partition(self._h, nranks, _ptr(owner), _ptr(vals), _ptr(invs)), self._h)
        self._part = {"nranks": nranks, "owner": owner, "values": vals, "inverses": invs}
        return self._part

    def factorize_part(self, values, precision="fp64", part=0, stream=None):
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        if values is not None and not _is_device(values):
            values = np.ascontiguousarray(values, dtype=np.float64)
        on_dev = 1 if (values is not None and _is_device(values)) else 0
        _check(load().spx_factorize_part(self._h, _ptr(values), on_dev, prec, int(part), _stream_ptr(stream)),
               self._h)

    def part_get(self, part: int, with_inverses: bool = False, out=None, stream=None):
        """Packed panel values (then inverse blocks) of a part as a CUDA tensor
        of the factor's type."""
        import torch
        k = part if part >= 0 else self._part["nranks"]
        n = int(self._part["values"][k] + (self._part["inverses"][k] if with_inverses else 0))
        if out is None:
            dt = torch.float64 if self.info()["precision"] == SPX_FP64 else torch.float32
            out = torch.empty(max(n, 1), dtype=dt, device="cuda")
        _check(load().spx_part_get(self._h, int(part), 1 if with_inverses else 0, _ptr(out), _stream_ptr(stream)),
               self._h)
        return out

    def part_set(self, part: int, buf, with_inverses: bool = False, stream=None):
        _check(load().spx_part_set(self._h, int(part), 1 if with_inverses else 0, _ptr(buf), _stream_ptr(stream)),
               self._h)

    def set_wait_limit(self, polls: int = 0):
        """Polls (~256 ns each) before a sweep wait gives up; 0 = default."""
        _check(load().spx_set_wait_limit(self._h, int(polls)), self._h)

    def set_profiling(self, on: bool = True):
        _check(load().spx_set_profiling(self._h, 1 if on else 0), self._h)

    def kernel_stats(self) -> dict:
        k = spx_kernel_stats()
        _check(load().spx_get_kernel_stats(self._h, ctypes.byref(k)), self._h)
        return k.as_dict()

    def panels(self) -> dict:
        """Panel structure: first column, width, height, level, parent."""
        npn = self.info()["npanels"]
        out = {"first_col": np.empty(npn, np.int64), "width": np.empty(npn, np.int32),
               "height": np.empty(npn, np.int32), "level": np.empty(npn, np.int32),
               "parent": np.empty(npn, np.int32)}
        _check(load().spx_get_panels(self._h, *[_ptr(out[k]) for k in
                                                 ("first_col", "width", "height", "level", "parent")]),
               self._h)
        return out

    def perm(self) -> np.ndarray:
        p = np.empty(self.n, dtype=np.int64)
        _check(load().spx_get_perm(self._h, _ptr(p)), self._h)
        return p

    # -- differentiation -------------------------------------------------------
    def logdet(self) -> float:
        v = ctypes.c_double()
        _check(load().spx_logdet(self._h, ctypes.byref(v)), self._h)
        return v.value

    def selected_inverse(self, stream=None):
        _check(load().spx_selected_inverse(self._h, _stream_ptr(stream)), self._h)

    def selected_inverse_on_pattern(self, Lp: np.ndarray, Li: np.ndarray) -> np.ndarray:
        Lp = np.ascontiguousarray(Lp, dtype=np.int64)
        Li = np.ascontiguousarray(Li, dtype=np.int32)
        Zx = np.empty(len(Li), dtype=np.float64)
        _check(load().spx_get_selected_inverse(self._h, _ptr(Lp), _ptr(Li), _ptr(Zx)), self._h)
        return Zx

    def logdet_grad(self, out=None, stream=None):
        """(A^{-1})_{ji} for every stored entry (i, j), in CSC order."""
        if out is None:
            out = np.empty(self.nnz, dtype=np.float64)
        _check(load().spx_logdet_grad(self._h, _ptr(out), 1 if _is_device(out) else 0,
                                      _stream_ptr(stream)), self._h)
        return out

    def solve_grad(self, Lam, X, out=None, stream=None):
        """-sum_r Lam(i, r) X(j, r) for every stored entry (i, j).  Lam, X:
        (n,) or column-major (n, nrhs), both host or both CUDA tensors."""
        dev = _is_device(Lam)
        if dev:
            nrhs = 1 if Lam.dim() == 1 else Lam.shape[1]
            ldl = self.n if Lam.dim() == 1 else Lam.stride(1)
            ldx = self.n if X.dim() == 1 else X.stride(1)
            if out is None:
                import torch
                out = torch.empty(self.nnz, dtype=torch.float64, device=Lam.device)
        else:
            Lam = np.asfortranarray(Lam, dtype=np.float64)
            X = np.asfortranarray(X, dtype=np.float64)
            nrhs = 1 if Lam.ndim == 1 else Lam.shape[1]
            ldl = ldx = self.n
            if out is None:
                out = np.empty(self.nnz, dtype=np.float64)
        _check(load().spx_solve_grad(self._h, nrhs, _ptr(Lam), ldl, _ptr(X), ldx, _ptr(out),
                                     1 if dev else 0, _stream_ptr(stream)), self._h)
        return out

    def factor_on_pattern(self, Lp: np.ndarray, Li: np.ndarray, lu: bool = False):
        Lp = np.ascontiguousarray(Lp, dtype=np.int64)
        Li = np.ascontiguousarray(Li, dtype=np.int32)
        Lx = np.empty(len(Li), dtype=np.float64)
        Ut = np.empty(len(Li), dtype=np.float64) if lu else None
        _check(load().spx_get_factor(self._h, _ptr(Lp), _ptr(Li), _ptr(Lx), _ptr(Ut)), self._h)
        return (Lx, Ut) if lu else Lx


def analyze(colptr: np.ndarray, rowind: np.ndarray, method: str = "llt", perm=None,
            **opts) -> Handle:
    """spx_analyze on host CSC arrays (int64 colptr, int32 rowind)."""
    colptr = np.ascontiguousarray(colptr, dtype=np.int64)
    rowind = np.ascontiguousarray(rowind, dtype=np.int32)
    n = len(colptr) - 1
    o = default_options(**opts)
    keep = None
    if perm is not None:
        keep = np.ascontiguousarray(perm, dtype=np.int64)
        o.perm = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        o.ordering = SPX_ORDER_GIVEN
    raw = _vp()
    m = METHODS[method]
    st = load().spx_analyze(n, _ptr(colptr), _ptr(rowind), m, ctypes.byref(o), ctypes.byref(raw))
    _check(st, None)
    del keep
    return Handle(raw.value, n, int(colptr[-1]))


ENGINES = {"auto": 0, "cuda_cores": 1, "tensor_cores": 2}


def _ucheck(status: int, plan=None):
    if status != SPX_OK:
        msg = load().spx_update_last_error(plan)
        raise SpxError(status, msg.decode() if msg else "")


class UpdatePlan:
    """One (source, target) update task run through the factorization's own
    update kernels (spx_update_*): C -= A B^T, B the first nb_rows rows of A
    (of W for LDL^T), row i of A to row rowmap[i] of C, row j of B to column
    colmap[j]."""

    def __init__(self, m, nb_rows, k, ldc, nc, rowmap, colmap, lower=True, precision="fp64",
                 engine="auto", ldlt=False):
        rowmap = np.ascontiguousarray(rowmap, dtype=np.int32)
        colmap = np.ascontiguousarray(colmap, dtype=np.int32)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        eng = ENGINES[engine] if isinstance(engine, str) else int(engine)
        raw = _vp()
        _ucheck(load().spx_update_create(m, nb_rows, k, ldc, nc, _ptr(rowmap), _ptr(colmap),
                                         1 if lower else 0, prec, eng, 1 if ldlt else 0,
                                         ctypes.byref(raw)), None)
        self._u = raw.value
        self.m, self.k = m, k

    def free(self):
        if self._u:
            load().spx_update_free(self._u)
            self._u = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def stage(self, A, W=None, lda=None, stream=None):
        """A (and W): CUDA tensors, column-major m x k (``X.t().contiguous().t()``)."""
        if lda is None:   # a size-1 dimension may carry any stride
            lda = A.stride(1) if A.dim() == 2 and A.shape[1] > 1 else self.m
        _ucheck(load().spx_update_stage(self._u, _ptr(A), _ptr(W), lda, _stream_ptr(stream)), self._u)

    def run(self, C, wait=True, stream=None):
        _ucheck(load().spx_update_run(self._u, _ptr(C), 1 if wait else 0, _stream_ptr(stream)), self._u)

    def info(self) -> dict:
        e = ctypes.c_int32()
        t = ctypes.c_int64()
        _ucheck(load().spx_update_get_info(self._u, ctypes.byref(e), ctypes.byref(t)), self._u)
        return {"engine": {1: "cuda_cores", 2: "tensor_cores"}[e.value], "tiles": t.value}


def update(A, C, rowmap, colmap, nb_rows, lower=True, precision="fp64", engine="auto", W=None,
           stream=None):
    """C -= A B^T once through the factorization's update kernels (creates,
    stages, runs and frees an UpdatePlan).  A, W, C: column-major CUDA tensors."""
    m, k = A.shape
    nc = C.shape[1]
    ldc = C.stride(1) if nc > 1 else C.shape[0]
    plan = UpdatePlan(m, nb_rows, k, ldc, nc, rowmap, colmap, lower=lower,
                      precision=precision, engine=engine, ldlt=W is not None)
    try:
        plan.stage(A, W, stream=stream)
        plan.run(C, wait=True, stream=stream)
    finally:
        plan.free()


# ---------------------------------------------------------------------------
# Batched static-pivot LU (spx_batch_*)
# ---------------------------------------------------------------------------
def _bcheck(status: int, handle=None):
    if status != SPX_OK:
        msg = load().spx_batch_last_error(handle)
        raise SpxError(status, msg.decode() if msg else "")


class Batch:
    """Many small independent systems, factorized and solved in one launch."""

    def __init__(self, raw: int, ns: np.ndarray, nnzs: np.ndarray):
        self._h = raw
        self.ns = ns
        self.nnzs = nnzs
        self.nsys = len(ns)
        self.n_total = int(ns.sum())
        self.nnz_total = int(nnzs.sum())

    def free(self):
        if self._h:
            load().spx_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def _args(self, values, B, X):
        dev = _is_device(values)
        if not dev:
            values = np.ascontiguousarray(values, dtype=np.float64)
            if B is not None:
                B = np.ascontiguousarray(B, dtype=np.float64)
                if X is None:
                    X = np.empty(self.n_total, dtype=np.float64)
        elif B is not None and X is None:
            import torch
            X = torch.empty(self.n_total, dtype=torch.float64, device=values.device)
        return dev, values, B, X

    def run(self, values, B=None, X=None, precision="fp32", refine=None, stream=None):
        """Factorize all systems and (B given) solve each; returns (X, status name)."""
        dev, values, B, X = self._args(values, B, X)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        rptr = ctypes.byref(refine) if refine is not None else None
        st = load().spx_batch_run(self._h, _ptr(values), _ptr(B), _ptr(X), 1 if dev else 0, prec,
                                  rptr, _stream_ptr(stream))
        if st not in (SPX_OK, SPX_ERR_NOT_CONVERGED):
            _bcheck(st, self._h)
        return X, STATUS_NAMES[st]

    def tune(self, values, B, X=None, precision="fp32", refine=None, stream=None):
        dev, values, B, X = self._args(values, B, X)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        rptr = ctypes.byref(refine) if refine is not None else None
        st = load().spx_batch_tune(self._h, _ptr(values), _ptr(B), _ptr(X), 1 if dev else 0, prec,
                                   rptr, _stream_ptr(stream))
        if st not in (SPX_OK, SPX_ERR_NOT_CONVERGED):
            _bcheck(st, self._h)
        return X, STATUS_NAMES[st]

    def set_config(self, ctas_per_sm=0, leaf_width=8, rows_per_thread=0):
        _bcheck(load().spx_batch_set_config(self._h, ctas_per_sm, leaf_width, rows_per_thread),
                self._h)

    def info(self) -> dict:
        i = spx_batch_info()
        _bcheck(load().spx_batch_get_info(self._h, ctypes.byref(i)), self._h)
        return i.as_dict()

    def system_info(self) -> dict:
        out = {"iters": np.empty(self.nsys, np.int32), "berr": np.empty(self.nsys, np.float64),
               "converged": np.empty(self.nsys, np.int32),
               "npivot_repl": np.empty(self.nsys, np.int32), "bad_col": np.empty(self.nsys, np.int64)}
        _bcheck(load().spx_batch_system_info(self._h, *[_ptr(out[k]) for k in
                                                        ("iters", "berr", "converged",
                                                         "npivot_repl", "bad_col")]), self._h)
        return out

    def perm(self, s: int) -> np.ndarray:
        p = np.empty(int(self.ns[s]), dtype=np.int64)
        _bcheck(load().spx_batch_get_perm(self._h, s, _ptr(p)), self._h)
        return p

    def factor_on_pattern(self, s: int, Lp: np.ndarray, Li: np.ndarray):
        Lp = np.ascontiguousarray(Lp, dtype=np.int64)
        Li = np.ascontiguousarray(Li, dtype=np.int32)
        Lx = np.empty(len(Li), dtype=np.float64)
        Ut = np.empty(len(Li), dtype=np.float64)
        _bcheck(load().spx_batch_get_factor(self._h, s, _ptr(Lp), _ptr(Li), _ptr(Lx), _ptr(Ut)),
                self._h)
        return Lx, Ut


def batch_analyze(systems, grids=None, **opts) -> Batch:
    """spx_batch_analyze on a list of (colptr, rowind) host CSC patterns.
    grids: None or a list of (nx, ny, nz) per system (grid ordering rule)."""
    ns = np.array([len(cp) - 1 for cp, _ in systems], dtype=np.int64)
    nnzs = np.array([int(cp[-1]) for cp, _ in systems], dtype=np.int64)
    colptr = np.ascontiguousarray(np.concatenate([np.asarray(cp, np.int64) for cp, _ in systems])
                                  if systems else np.zeros(0, np.int64))
    rowind = np.ascontiguousarray(np.concatenate([np.asarray(ri, np.int32) for _, ri in systems])
                                  if systems else np.zeros(0, np.int32))
    g = None
    if grids is not None:
        g = np.ascontiguousarray(np.array([list(x) + [1] * (3 - len(x)) for x in grids],
                                          dtype=np.int32).ravel())
    o = default_options(**opts)
    raw = _vp()
    st = load().spx_batch_analyze(len(ns), _ptr(ns), _ptr(colptr), _ptr(rowind), _ptr(g),
                                  ctypes.byref(o), ctypes.byref(raw))
    _bcheck(st, None)
    return Batch(raw.value, ns, nnzs)
