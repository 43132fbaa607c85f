"""Element-wise parity of the factorization's own update kernels (Sec. V-B:
C = C - A B^T with B the first rows of A, subtracted straight into a gapped
target panel through the row map) against the oracle's panel update.

Every engine the factorization uses runs here through spx_update_* on the
paper's kernel-study generator (C twice as tall as A, random blocks of about
200 rows, A's blocks inside C's blocks): update_kernel<double> and
update_kernel<float> on the CUDA cores (64 x 64 and 256 x 16 tiles), and
update_tc_kernel on the tensor cores with TF32, BF16 and split-TF32 operands
and the two LDL^T forms (B from the D L^T rows).  The expected values are the
oracle's FP64 update on the operands the kernel multiplies: the panel values,
rounded to TF32 (to nearest, ties away) or BF16 (to nearest even) for the
tensor-core kinds.  Each entry must lie within the FP32 (or FP64) dot-product
error bound of its own magnitude sum sum_k |a_ik b_jk|, which a dropped K
term, a mis-mapped row or column, or a wrong lower/upper mask exceeds by
orders of magnitude; entries the task does not touch must come back bit-equal.
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


def tf32_rna(x: np.ndarray) -> np.ndarray:
    """FP32 -> TF32 (10 mantissa bits), round to nearest, ties away from zero."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    sign = b & np.uint32(0x80000000)
    mag = ((b & np.uint32(0x7FFFFFFF)) + np.uint32(0x1000)) & np.uint32(0xFFFFE000)
    return (sign | mag).view(np.float32)


def bf16_rne(x: np.ndarray) -> np.ndarray:
    """FP32 -> BF16 (7 mantissa bits), round to nearest even."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


CASES = [  # m, k (source width), nb (facing rows), lower, seed
    (301, 33, 97, True, 1),      # odd sizes, K not a multiple of 8
    (257, 1, 65, False, 2),      # K = 1
    (1000, 64, 130, True, 3),    # several 128-row tiles, ragged facing block
    (777, 45, 16, False, 4),     # facing block of 16 rows: narrow CUDA-core tiles
    (2048, 256, 511, True, 5),   # wide source panel, K = 256
    (8192, 64, 400, False, 6),   # more tiles than one wave of the GPU
    (8192, 160, 300, False, 7),  # more tiles than SMs, K spanning several operand-ring turns per tile
]

COMBOS = [  # precision, engine, ldlt
    ("fp64", "cuda_cores", False), ("fp32", "cuda_cores", False), ("tf32", "cuda_cores", False),
    ("fp32", "tensor_cores", False), ("tf32", "tensor_cores", False),
    ("bf16", "tensor_cores", False),
    ("fp64", "cuda_cores", True), ("fp32", "cuda_cores", True),
    ("tf32", "tensor_cores", True), ("bf16", "tensor_cores", True),
]


def _operand(x32: np.ndarray, prec: str, engine: str) -> np.ndarray:
    """The values the kernel multiplies, as FP64."""
    if engine == "tensor_cores" and prec == "tf32":
        return tf32_rna(x32).astype(np.float64)
    if engine == "tensor_cores" and prec == "bf16":
        return bf16_rne(x32).astype(np.float64)
    return x32.astype(np.float64)


def _colmajor(torch, M, dtype):
    return torch.from_numpy(np.ascontiguousarray(M.T, dtype=dtype)).cuda().t()


def _run_case(torch, m, k, nb, lower, seed, prec, engine, ldlt):
    A, C, rowmap, colmap = inputs.gapped_update_case(m, k, nb, seed)
    Wd = np.random.default_rng([seed, 99]).standard_normal((m, k)) if ldlt else None
    fp64 = prec == "fp64"
    dt = np.float64 if fp64 else np.float32
    As, Cs = A.astype(dt), C.astype(dt)
    Ws = Wd.astype(dt) if ldlt else None
    plan = spx.UpdatePlan(m, nb, k, C.shape[0], C.shape[1], rowmap, colmap, lower=lower,
                          precision=prec, engine=engine, ldlt=ldlt)
    assert plan.info()["engine"] == engine
    tC = _colmajor(torch, Cs, dt)
    plan.stage(_colmajor(torch, As, dt), _colmajor(torch, Ws, dt) if ldlt else None)
    plan.run(tC, wait=True)
    got = tC.cpu().numpy().astype(np.float64)
    plan.free()

    a = As.astype(np.float64) if fp64 else _operand(As, prec, engine)
    bsrc = Ws if ldlt else As
    b = (bsrc.astype(np.float64) if fp64 else _operand(bsrc, prec, engine))[:nb]
    expect = oracle.panel_update(a, b, Cs.astype(np.float64), rowmap, colmap, lower)
    mag = -oracle.panel_update(np.abs(a), np.abs(b), np.zeros_like(expect), rowmap, colmap, lower)
    touched = oracle.panel_update(np.ones((m, 1)), np.ones((nb, 1)), np.zeros_like(expect), rowmap,
                                  colmap, lower) != 0
    u = 2.0 ** -53 if fp64 else 2.0 ** -24
    c = 4.0 if engine == "tensor_cores" else 2.0
    tol = c * (k + 2) * u * (mag + np.abs(expect))
    if engine == "tensor_cores" and prec == "fp32":
        tol += 2.0 ** -19 * mag          # split TF32 drops lo*lo and rounds lo to TF32
    err = np.abs(got - expect)
    bad = err > tol
    assert not bad.any(), (f"{int(bad.sum())} entries outside the bound; worst excess "
                           f"{float(np.max(err - tol)):.3e} at {np.argwhere(bad)[0]}")
    assert np.array_equal(got[~touched], Cs.astype(np.float64)[~touched])


@pytest.mark.parametrize("prec,engine,ldlt", COMBOS)
@pytest.mark.parametrize("m,k,nb,lower,seed", CASES)
def test_update_kernels_elementwise(torch, m, k, nb, lower, seed, prec, engine, ldlt):
    _run_case(torch, m, k, nb, lower, seed, prec, engine, ldlt)


def test_engine_choice_follows_the_factorization(torch):
    """Tensor cores for the single-precision modes when the source is at
    least 32 wide (LDL^T in FP32 stays on the CUDA cores); CUDA cores for
    FP64 and for narrow sources."""
    rowmap = np.arange(300, dtype=np.int32)
    colmap = np.arange(40, dtype=np.int32)
    for prec, k, ldlt, want in [("fp64", 64, False, "cuda_cores"), ("tf32", 64, False, "tensor_cores"),
                                ("bf16", 32, False, "tensor_cores"), ("tf32", 31, False, "cuda_cores"),
                                ("fp32", 64, False, "tensor_cores"), ("fp32", 64, True, "cuda_cores"),
                                ("bf16", 64, True, "tensor_cores")]:
        p = spx.UpdatePlan(300, 40, k, 300, 40, rowmap, colmap, precision=prec, ldlt=ldlt)
        assert p.info()["engine"] == want, (prec, k, ldlt)
        p.free()
    with pytest.raises(spx.SpxError) as e:
        spx.UpdatePlan(300, 40, 64, 300, 40, rowmap, colmap, precision="fp64", engine="tensor_cores")
    assert e.value.status == spx.SPX_ERR_ARG


def test_repeated_runs_accumulate(torch):
    """Runs enqueued without waiting subtract the product once each."""
    m, k, nb = 600, 64, 70
    A, C, rowmap, colmap = inputs.gapped_update_case(m, k, nb, 17)
    A32 = bf16_rne(A.astype(np.float32))          # exact in BF16 and TF32
    plan = spx.UpdatePlan(m, nb, k, C.shape[0], C.shape[1], rowmap, colmap, lower=True,
                          precision="tf32")
    tC = _colmajor(torch, C.astype(np.float32), np.float32)
    plan.stage(_colmajor(torch, A32, np.float32))
    for _ in range(3):
        plan.run(tC, wait=False)
    plan.run(tC, wait=True)
    got = tC.cpu().numpy().astype(np.float64)
    a = A32.astype(np.float64)
    expect = C.astype(np.float32).astype(np.float64)
    for _ in range(4):
        expect = oracle.panel_update(a, a[:nb], expect, rowmap, colmap, True)
    mag = -oracle.panel_update(np.abs(a), np.abs(a[:nb]), np.zeros_like(expect), rowmap, colmap, True)
    assert np.all(np.abs(got - expect) <= 16 * (k + 2) * 2.0 ** -24 * (4 * mag + np.abs(expect)))
    plan.free()
