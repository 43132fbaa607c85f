"""Distributed factorization by subtrees with fan-in of the top panels.

The library partitions the panel tree (spx_partition): whole bottom subtrees
go to ranks with their flops balanced, and the panels above them -- the top
separators -- belong to rank 0.  Every update then stays inside one rank's
subtrees or goes from them into the top panels (the fan-in of the paper's
future-work section), so the only exchange of the factorization is one sum
of the ranks' top panels onto rank 0 before rank 0 factors the top.  This
module drives that sequence over torch.distributed (NCCL with CUDA tensors,
gloo with CPU tensors); each rank holds its own handle on the same pattern.
"""
from __future__ import annotations

from typing import Optional

import numpy as np


def fan_in(buf, world: int, rank: int, dist=None):
    """Sum the ranks' packed top panels onto rank 0 (the fan-in): one
    reduce of one contiguous buffer.  Returns the buffer (the sum on rank 0)."""
    if world <= 1:
        return buf
    if dist is None:
        import torch.distributed as dist
    dist.reduce(buf, dst=0, op=dist.ReduceOp.SUM)
    return buf


def gather_parts(h, world: int, rank: int, dist=None):
    """Copy every other rank's factored subtrees (values and inverse blocks)
    into rank 0's handle, so that rank 0 holds the whole factor and can solve."""
    if world <= 1:
        return
    if dist is None:
        import torch.distributed as dist
    import torch
    part = h._part
    dt = torch.float64 if h.info()["precision"] == 0 else torch.float32
    for r in range(1, world):
        n = int(part["values"][r] + part["inverses"][r])
        if rank == r:
            dist.send(h.part_get(r, with_inverses=True), dst=0)
        elif rank == 0:
            buf = torch.empty(max(n, 1), dtype=dt, device="cuda")
            dist.recv(buf, src=r)
            h.part_set(r, buf, with_inverses=True)


def factorize_distributed(h, values, precision: str, world: int, rank: int, dist=None,
                          gather: bool = True) -> dict:
    """The distributed factorization of the module docstring on this rank's
    handle `h`; rank 0 ends with the top factored (and, with `gather`, the
    whole factor).  Returns the partition (owners, part sizes)."""
    part = h.partition(world)
    h.factorize_part(values, precision, rank)
    top = h.part_get(-1, with_inverses=False)
    fan_in(top, world, rank, dist)
    if rank == 0:
        h.part_set(-1, top, with_inverses=False)
        h.factorize_part(None, precision, -1)
    if gather:
        gather_parts(h, world, rank, dist)
    return part


def subtree_columns(h, owner: np.ndarray) -> dict:
    """Permuted columns of each part (rank r, and -1 for the top), from the
    panel structure: {part: array of columns}."""
    P = h.panels()
    out = {}
    for q in range(len(owner)):
        cols = np.arange(P["first_col"][q], P["first_col"][q] + P["width"][q])
        out.setdefault(int(owner[q]), []).append(cols)
    return {k: np.concatenate(v) for k, v in out.items()}
