"""Subtree-to-rank distribution with fan-in (the paper's future-work
section): the partition of the panel tree and the one exchange of the
distributed factorization -- the sum of the ranks' top-panel contributions
onto rank 0 -- checked on the CPU with 2 and 4 gloo ranks.

The library's partition (spx_partition, host only) maps whole subtrees to
ranks and keeps the separators above them (the top) on rank 0.  Here each
rank computes the contribution of its subtrees to the top block densely,
A_TS A_SS^-1 A_ST on its own columns S (test arithmetic, standing in for the
GPU factorization of the subtrees); the fan-in module sums them onto rank 0,
whose Cholesky factor of A_TT minus that sum must equal the top block of the
oracle's factor of the whole matrix: the subtrees are independent, which is
exactly what the partition must guarantee.
"""
import datetime
import os
import socket

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_1405_2636_gb300 import fanin, inputs, spx

GRID = (12, 11, 10)


def _system():
    A = inputs.diffusion_3d(*GRID, 23)
    cp, ri, vals = inputs.csc_arrays(A)
    h = spx.analyze(cp, ri, "llt", ordering=spx.SPX_ORDER_GRID, grid=GRID, max_width=32)
    return A, h


@pytest.mark.parametrize("nranks", [1, 2, 3, 4, 8])
def test_partition_keeps_subtrees_independent(nranks):
    A, h = _system()
    part = h.partition(nranks)
    owner = part["owner"]
    P = h.panels()
    assert owner.shape == (h.info()["npanels"],)
    assert set(np.unique(owner)) <= set(range(-1, nranks))
    # the top is closed upwards: a top panel's parent is a top panel
    for q in range(len(owner)):
        if owner[q] < 0 and P["parent"][q] >= 0:
            assert owner[P["parent"][q]] < 0
        if owner[q] >= 0 and P["parent"][q] >= 0:
            assert owner[P["parent"][q]] in (owner[q], -1)
    # no entry of L couples two ranks' subtrees (oracle's symbolic pattern)
    F = oracle.cholesky(A, h.perm())
    cols = fanin.subtree_columns(h, owner)
    col_owner = np.empty(A.shape[0], np.int64)
    for k, c in cols.items():
        col_owner[c] = k
    Lp, Li = F.sym.Lp, F.sym.Li
    for j in range(A.shape[0]):
        oj = col_owner[j]
        if oj >= 0:
            oi = col_owner[Li[Lp[j]:Lp[j + 1]]]
            assert np.all((oi == oj) | (oi < 0))
    # packed sizes: every panel's values and inverse block in exactly one part
    assert part["values"].sum() == sum((P["height"] * P["width"]).tolist())
    assert part["inverses"].sum() == sum((P["width"] ** 2).tolist())
    if nranks > 1:
        work = [len(cols.get(r, [])) for r in range(nranks)]
        assert min(work) > 0


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, queue):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    try:
        A, h = _system()
        part = h.partition(world)
        cols = fanin.subtree_columns(h, part["owner"])
        PA = oracle.permute(A, h.perm()).toarray()
        T = np.sort(cols.get(-1, np.zeros(0, np.int64)))
        S = np.sort(cols.get(rank, np.zeros(0, np.int64)))
        # this rank's contribution to the top block (its subtrees eliminated)
        contrib = np.zeros((len(T), len(T)))
        if len(S):
            ASS, ATS = PA[np.ix_(S, S)], PA[np.ix_(T, S)]
            contrib = ATS @ sla.solve(ASS, ATS.T, assume_a="pos")
        buf = torch.from_numpy(np.ascontiguousarray(contrib))
        fanin.fan_in(buf, world, rank, dist)
        res = {"owner": part["owner"]}
        if rank == 0:
            schur = PA[np.ix_(T, T)] - buf.numpy()
            res["LTT"] = np.linalg.cholesky(schur)
            res["T"] = T
        queue.put((rank, res))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_gloo_ranks_fan_in_to_the_top_factor(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, queue)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        got = dict(queue.get(timeout=240) for _ in range(world))
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    for r in range(1, world):   # every rank computed the same partition
        assert np.array_equal(got[r]["owner"], got[0]["owner"])
    A, h = _system()
    F = oracle.cholesky(A, h.perm())
    T = got[0]["T"]
    assert len(T) > 0
    L = F.L().toarray()
    ref = L[np.ix_(T, T)]
    assert np.linalg.norm(got[0]["LTT"] - ref) <= 1e-12 * np.linalg.norm(ref)
