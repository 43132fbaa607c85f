"""Host logic for runs on several GPUs of one node (one process per GPU).

The factorization of one sparse system does not split across GPUs with a
single exchange step: the top separators of the elimination tree receive
updates from every subtree, and the paper leaves the fan-in distribution of
subtrees over GPUs to future work (Sec. VI).  So every rank factors its own
replica of the workload, and the ranks meet only around the timed region
(a barrier before it, the maximum of the step times after it).

A batch of independent systems does split: each rank takes a bin of
systems of about equal work (longest job first onto the least-loaded rank)
and runs it on its own GPU; the ranks combine their statistics once, after
the timed runs.  No collective touches the data path in either case.
"""
from __future__ import annotations

import heapq
import os
from typing import Dict, List, Sequence, Tuple


def env_ranks() -> Tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def lu_work_estimate(side: int) -> float:
    """Relative factorization work of a 2-D grid system of the given side:
    nested dissection factors n = side^2 unknowns in O(n^1.5) = O(side^3)
    operations, the root separator's dense block dominating."""
    return float(side) ** 3


def shard_by_work(work: Sequence[float], world: int) -> List[List[int]]:
    """Split items 0..len(work)-1 over ``world`` ranks: items by decreasing
    work (ties by index), each onto the rank with the least work so far
    (ties by rank).  Every item lands on exactly one rank; each rank's list
    is ascending.  The heaviest rank exceeds the lightest by at most the
    largest single item."""
    if world < 1:
        raise ValueError("world must be >= 1")
    bins: List[List[int]] = [[] for _ in range(world)]
    heap = [(0.0, r) for r in range(world)]
    for s in sorted(range(len(work)), key=lambda i: (-float(work[i]), i)):
        load, r = heapq.heappop(heap)
        bins[r].append(s)
        heapq.heappush(heap, (load + float(work[s]), r))
    return [sorted(b) for b in bins]


class RankGroup:
    """Barrier and scalar reductions over the ranks of the default process
    group; with one rank every call is the identity.  ``device`` holds the
    reduction tensors ("cuda:i" for NCCL, "cpu" for gloo)."""

    def __init__(self, world: int, device):
        self.world = world
        self.device = device

    def _reduce(self, x: float, op: str) -> float:
        if self.world == 1:
            return float(x)
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op={"max": dist.ReduceOp.MAX, "min": dist.ReduceOp.MIN,
                               "sum": dist.ReduceOp.SUM}[op])
        return float(t.item())

    def barrier(self) -> None:
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max(self, x: float) -> float:
        return self._reduce(x, "max")

    def min(self, x: float) -> float:
        return self._reduce(x, "min")

    def sum(self, x: float) -> float:
        return self._reduce(x, "sum")


# How each statistic of a rank's share of a batch combines over the ranks.
BATCH_COMBINE: Dict[str, str] = {
    "ms": "max",                  # the batch is done when the slowest rank is
    "flops": "sum",
    "systems": "sum",
    "n_total": "sum",
    "nnz_l_total": "sum",
    "all_converged": "min",       # 1 only if every rank's systems converged
    "max_backward_error": "max",
    "max_refine_iters": "max",
    "pivot_replacements": "sum",
}


def combine_batch_stats(group: RankGroup, stats: Dict[str, float]) -> Dict[str, float]:
    """Combine per-rank batch statistics (keys of BATCH_COMBINE) over the
    ranks, in a fixed key order so that every rank issues the same
    collectives; ``gflops`` is the whole job's flops over the slowest
    rank's time."""
    out = {k: getattr(group, how)(stats[k]) for k, how in BATCH_COMBINE.items()}
    out["gflops"] = out["flops"] / (out["ms"] / 1e3) / 1e9 if out["ms"] > 0 else float("nan")
    return out


def whole_job_rate(units_per_rank: float, world: int, max_ms: float) -> float:
    """Throughput of ``world`` replicas that each processed ``units_per_rank``
    units, the step ending when the slowest rank ends (units per second)."""
    return world * units_per_rank / (max_ms / 1e3)
