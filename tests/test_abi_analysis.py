"""Host-side checks of libspx through its C ABI (no GPU needed).

The library must load and export every function include/spx.h declares;
spx_analyze (host-only) must order exactly like the oracle's nested
dissection and count exactly the oracle's nnz(L) and flops; bad input must
come back as SPX_ERR_ARG with a message, never as a crash.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1405_2636_gb300 import build as spx_build
from paper_1405_2636_gb300 import inputs, spx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    spx_build.build()
    spx.load()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "spx.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(spx_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    names = _declared_functions()
    assert set(names) == set(spx.EXPORTED)
    lib = ctypes.CDLL(spx.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name


def _postorder(parent):
    n = len(parent)
    kids = [[] for _ in range(n)]
    for j in range(n):
        if parent[j] >= 0:
            kids[parent[j]].append(j)
    out = []
    for r in range(n):
        if parent[r] >= 0:
            continue
        stack = [(r, 0)]
        while stack:
            v, i = stack.pop()
            if i < len(kids[v]):
                stack.append((v, i + 1))
                stack.append((kids[v][i], 0))
            else:
                out.append(v)
    return np.asarray(out, dtype=np.int64)


def _oracle_counts(A, perm):
    Pa = oracle.permute(A, perm)
    s = oracle.symbolic(oracle.symmetrized_pattern(Pa))
    return s


@pytest.mark.parametrize("grid,dof,maker", [
    ((31, 31, 1), 1, lambda: inputs.laplacian_2d(31, 31)),
    ((13, 11, 9), 1, lambda: inputs.diffusion_3d(13, 11, 9, 3)),
    ((5, 4, 6), 3, lambda: inputs.elasticity_27pt(5, 4, 6, 4)),
    ((2, 2, 2), 1, lambda: inputs.laplacian_3d(2, 2, 2, 1.0)),
    ((1, 1, 1), 1, lambda: inputs.laplacian_3d(1, 1, 1, 1.0)),
])
def test_grid_analysis_matches_oracle(grid, dof, maker):
    A = maker()
    cp, ri, _ = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "llt", ordering=spx.SPX_ORDER_GRID, grid=grid, dof=dof, max_width=24)
    perm = h.perm()
    assert np.array_equal(perm, oracle.nd_grid(*grid, dof))
    s = _oracle_counts(A, perm)
    info = h.info()
    assert info["nnz_l"] == int(s.Lp[-1])
    assert info["flops"] == oracle.flops(s.counts, "llt")
    assert info["nnz_l"] <= info["nnz_stored"] <= 1.12 * info["nnz_l"] + 1
    h.free()


@pytest.mark.parametrize("n,seed", [(50, 1), (300, 2), (1500, 3)])
def test_graph_analysis_matches_oracle(n, seed):
    A = inputs.random_spd_graph(n, 5.0, seed)
    cp, ri, _ = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "lu", ordering=spx.SPX_ORDER_GRAPH, max_width=16)
    perm = h.perm()
    # the oracle's nested dissection, then a postorder of its elimination tree
    # (roots and children in ascending order), which makes supernodes contiguous
    nd = oracle.nd_graph(A)
    parent = oracle.etree(oracle.symmetrized_pattern(oracle.permute(A, nd)))
    assert np.array_equal(perm, nd[_postorder(parent)])
    s = _oracle_counts(A, perm)
    info = h.info()
    assert info["nnz_l"] == int(s.Lp[-1])
    assert info["flops"] == pytest.approx(oracle.flops(s.counts, "lu"), rel=0, abs=0.5)
    h.free()


def test_given_and_natural_orderings():
    A = inputs.diffusion_3d(6, 5, 4, 1)
    cp, ri, _ = inputs.csc_arrays(A)
    rng = np.random.default_rng(0)
    p = rng.permutation(A.shape[0])
    h = spx.analyze(cp, ri, "llt", perm=p)
    q = h.perm()
    # the library may append an elimination-tree postorder; the factor's
    # fill must then equal the oracle's on the final order
    assert sorted(q.tolist()) == list(range(A.shape[0]))
    s = _oracle_counts(A, q)
    assert h.info()["nnz_l"] == int(s.Lp[-1])
    h2 = spx.analyze(cp, ri, "llt", ordering=spx.SPX_ORDER_NATURAL)
    s2 = _oracle_counts(A, h2.perm())
    assert h2.info()["nnz_l"] == int(s2.Lp[-1])


def test_lower_only_input_has_same_structure():
    A = inputs.laplacian_2d(9, 7)
    cp, ri, _ = inputs.csc_arrays(A)
    import scipy.sparse as sp
    Lo = sp.tril(A).tocsc()
    cpl, ril, _ = inputs.csc_arrays(Lo)
    h1 = spx.analyze(cp, ri, "llt", ordering=spx.SPX_ORDER_GRID, grid=(9, 7, 1))
    h2 = spx.analyze(cpl, ril, "llt", ordering=spx.SPX_ORDER_GRID, grid=(9, 7, 1), lower_only=1)
    assert h1.info()["nnz_l"] == h2.info()["nnz_l"]
    assert np.array_equal(h1.perm(), h2.perm())


def test_bad_input_is_rejected():
    cp = np.array([0, 2, 1], dtype=np.int64)      # decreasing
    ri = np.array([0, 1], dtype=np.int32)
    with pytest.raises(spx.SpxError) as e:
        spx.analyze(cp, ri)
    assert e.value.status == spx.SPX_ERR_ARG
    cp = np.array([0, 1, 2], dtype=np.int64)
    ri = np.array([0, 5], dtype=np.int32)         # row out of range
    with pytest.raises(spx.SpxError):
        spx.analyze(cp, ri)
    A = inputs.laplacian_2d(4, 4)
    cp, ri, _ = inputs.csc_arrays(A)
    with pytest.raises(spx.SpxError) as e:        # grid does not match n
        spx.analyze(cp, ri, ordering=spx.SPX_ORDER_GRID, grid=(5, 4, 1))
    assert "grid" in str(e.value)
    with pytest.raises(spx.SpxError):             # not a permutation
        spx.analyze(cp, ri, perm=np.zeros(16, dtype=np.int64))
    with pytest.raises(spx.SpxError):             # too wide for the diagonal kernels
        spx.analyze(cp, ri, max_width=4096)
    ri2 = ri.copy()
    ri2[1] = ri2[0]                               # duplicate entry in column 0
    with pytest.raises(spx.SpxError) as e:
        spx.analyze(cp, ri2)
    assert "duplicate" in str(e.value)


def test_calls_on_null_or_unfactored_handles_fail_cleanly():
    lib = spx.load()
    assert lib.spx_factorize(None, None, 0, 0, None) == spx.SPX_ERR_ARG
    assert lib.spx_get_info(None, None) == spx.SPX_ERR_ARG
    lib.spx_free(None)
    A = inputs.laplacian_2d(4, 4)
    cp, ri, _ = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri)
    b = np.ones(16)
    x = np.zeros(16)
    st = lib.spx_solve(h._h, 1, b.ctypes.data, 16, x.ctypes.data, 16, 0, None, None, None)
    assert st == spx.SPX_ERR_STATE
    assert b"factorize" in lib.spx_last_error(h._h)


def test_wait_limit_on_an_analysed_handle():
    """spx_set_wait_limit needs no GPU: it checks its argument and keeps the
    value for the next sweeps."""
    A = inputs.laplacian_2d(9, 9)
    cp, ri, _ = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "llt")
    for bad in (-1, 2 ** 32):
        with pytest.raises(spx.SpxError) as e:
            h.set_wait_limit(bad)
        assert e.value.status == spx.SPX_ERR_ARG
    h.set_wait_limit(2 ** 32 - 1)
    h.set_wait_limit(0)
    assert spx.load().spx_set_wait_limit(None, 0) == spx.SPX_ERR_ARG
    h.free()


def test_update_plan_rejects_bad_arguments():
    """The kernel-study plan checks sizes, maps and the engine before it
    touches the device."""
    rm = np.arange(10, dtype=np.int32)
    cm = np.arange(4, dtype=np.int32)
    bad = [dict(m=10, nb_rows=11, k=8, ldc=10, nc=4),              # nb_rows > m
           dict(m=10, nb_rows=4, k=0, ldc=10, nc=4),               # k = 0
           dict(m=10, nb_rows=4, k=8, ldc=9, nc=4),                # rowmap reaches ldc
           dict(m=10, nb_rows=4, k=8, ldc=10, nc=3)]               # colmap reaches nc
    for b in bad:
        with pytest.raises(spx.SpxError) as e:
            spx.UpdatePlan(b["m"], b["nb_rows"], b["k"], b["ldc"], b["nc"], rm, cm)
        assert e.value.status == spx.SPX_ERR_ARG
    for prec, ldlt in (("fp64", False), ("fp32", True)):
        with pytest.raises(spx.SpxError) as e:   # no tensor-core form of these
            spx.UpdatePlan(10, 4, 8, 10, 4, rm, cm, precision=prec, engine="tensor_cores", ldlt=ldlt)
        assert e.value.status == spx.SPX_ERR_ARG
    lib = spx.load()
    assert lib.spx_update_run(None, None, 1, None) == spx.SPX_ERR_ARG
    lib.spx_update_free(None)


def test_update_task_structure_invariants():
    """Every source row below a facing block lies in its target (Sec. V-B:
    each block of the source lies inside one block of the facing panel)."""
    A = inputs.diffusion_3d(10, 9, 8, 7)
    cp, ri, _ = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "llt", ordering=spx.SPX_ORDER_GRID, grid=(10, 9, 8), max_width=8)
    info = h.info()
    assert info["npanels"] >= info["nsupernodes"] * 0 + 1
    assert info["update_flops"] <= info["flops_stored"]
    assert info["flops_stored"] >= info["flops"]


def _edge_patterns():
    import scipy.sparse as sp
    n = 40
    diag = sp.identity(n, format="csc") * 2.0                       # no update at all
    dense = sp.csc_matrix(np.ones((70, 70)) + 70 * np.eye(70))      # one supernode, split into panels
    m = 60
    arrow = sp.lil_matrix((m, m))                                   # dense last row and column
    for i in range(m):
        arrow[i, i] = 4.0
        arrow[i, m - 1] = arrow[m - 1, i] = 1.0
    arrow[m - 1, m - 1] = 100.0
    blocks = sp.block_diag([inputs.random_spd_graph(80, 4.0, 1),   # two components
                            inputs.random_spd_graph(50, 4.0, 2)]).tocsc()
    unsym = (sp.random(90, 90, density=0.04, random_state=5, format="csc")
             + sp.identity(90) * 5).tocsc()                          # LU on A + A^T
    nodiag = inputs.laplacian_2d(6, 6).tolil()                      # a column without its diagonal
    nodiag[7, 7] = 0
    nodiag = nodiag.tocsc()
    nodiag.eliminate_zeros()
    return [("diagonal", diag, "llt"), ("dense", dense, "llt"), ("dense", dense, "lu"),
            ("arrow", arrow.tocsc(), "llt"), ("components", blocks, "llt"),
            ("unsymmetric", unsym, "lu"), ("no-diagonal", nodiag, "lu")]


@pytest.mark.parametrize("name,A,method", _edge_patterns(), ids=lambda v: v if isinstance(v, str) else "")
@pytest.mark.parametrize("ordering", [spx.SPX_ORDER_NATURAL, spx.SPX_ORDER_GRAPH])
def test_edge_patterns_match_oracle(name, A, method, ordering):
    """Fill and flop count of the library's analysis equal the oracle's
    symbolic factorization on the library's final order, for patterns at the
    edges of the supernode partition."""
    cp, ri, _ = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, method, ordering=ordering, max_width=16)
    perm = h.perm()
    assert sorted(perm.tolist()) == list(range(A.shape[0]))
    s = _oracle_counts(A, perm)
    info = h.info()
    assert info["nnz_l"] == int(s.Lp[-1])
    assert info["flops"] == pytest.approx(oracle.flops(s.counts, method), rel=0, abs=0.5)
    assert info["nnz_l"] <= info["nnz_stored"]
    if name == "diagonal":
        assert info["nupdates"] == 0 and info["npanels"] == A.shape[0]
    if name == "dense":
        assert info["npanels"] == (A.shape[0] + 15) // 16
    h.free()


@pytest.mark.parametrize("method,maker,opts", [
    ("llt", lambda: inputs.diffusion_3d(10, 9, 8, 7), dict(ordering=1, grid=(10, 9, 8), max_width=8)),
    ("llt", lambda: inputs.random_spd_graph(700, 5.0, 3), dict(ordering=2, max_width=24)),
    ("lu", lambda: inputs.convection_diffusion_2d(25, 1)[0], dict(ordering=1, grid=(25, 25, 1), max_width=16)),
], ids=["grid-llt", "graph-llt", "grid-lu"])
def test_panel_tree_invariants(method, maker, opts):
    """The panel structure (Sec. III: supernodes split into panels of at most
    max_width columns, each a dense trapezoid of its rows) accounts exactly
    for the stored entries and the stored flop count, and its tree is a
    level structure: parents later and higher, leaves at level 0."""
    A = maker()
    cp, ri, _ = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, method, **opts)
    P, info = h.panels(), h.info()
    w, hh = P["width"].astype(np.int64), P["height"].astype(np.int64)
    par, lev = P["parent"], P["level"]
    assert w.sum() == A.shape[0] and np.all(w >= 1) and np.all(w <= opts["max_width"])
    assert P["first_col"][0] == 0 and np.array_equal(np.diff(P["first_col"]), w[:-1])
    assert np.all(hh >= w) and np.all(hh <= A.shape[0] - P["first_col"])
    assert info["nnz_stored"] == int(np.sum(w * (hh - w) + w * (w + 1) // 2))
    c = np.concatenate([hh[p] - np.arange(w[p]) for p in range(len(w))]).astype(np.float64)
    stored = np.sum(c * c) if method == "llt" else np.sum(2 * (c - 1) ** 2 + (c - 1))
    assert info["flops_stored"] == pytest.approx(stored, rel=1e-15)
    for p in range(len(par)):
        assert par[p] == -1 or (par[p] > p and lev[par[p]] > lev[p])
    has_child = np.zeros(len(par), bool)
    has_child[par[par >= 0]] = True
    assert np.all(lev[~has_child] == 0) and info["nlevels"] == lev.max() + 1
    h.free()


def test_binding_structs_match_the_header(tmp_path):
    """Every struct the ctypes binding mirrors has the size the C compiler
    gives the declaration in include/spx.h (a field added on one side only
    would make the library write past the binding's buffer)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "sizes.c"
    names = ["spx_options", "spx_refine", "spx_solve_info", "spx_info", "spx_kernel_stats",
             "spx_batch_info"]
    src.write_text('#include <stdio.h>\n#include "spx.h"\nint main(void){\n' +
                   "".join(f'printf("%zu\\n", sizeof({n}));\n' for n in names) + "return 0;}\n")
    exe = tmp_path / "sizes"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    sizes = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                            text=True).stdout.split()]
    import ctypes
    assert sizes == [ctypes.sizeof(getattr(spx, n)) for n in names]
    assert spx.spx_kernel_stats.as_dict  # one entry per kernel class of the header
    assert len(spx.KERNEL_CLASSES) == 6
