"""Multi-rank host logic: replicas of one system and shards of a batch of
independent systems (the batched LU), checked on the CPU, including two
ranks over a gloo process group."""
import datetime
import os
import socket

import numpy as np
import pytest

from paper_1405_2636_gb300 import inputs, replicas


def test_shard_by_work_covers_each_item_once_and_balances():
    rng = np.random.default_rng(0)
    work = rng.uniform(1.0, 100.0, size=1000)
    for world in (1, 2, 3, 8):
        bins = replicas.shard_by_work(work, world)
        assert len(bins) == world
        assert sorted(s for b in bins for s in b) == list(range(1000))
        assert all(b == sorted(b) for b in bins)
        loads = [work[b].sum() for b in bins]
        # longest job first onto the least-loaded rank: the spread is at
        # most one item
        assert max(loads) - min(loads) <= work.max() + 1e-9


def test_shard_of_the_batched_workload():
    sides = inputs.batched_sides(4096, 4)
    work = [replicas.lu_work_estimate(k) for k in sides]
    b2 = replicas.shard_by_work(work, 2)
    assert b2 == replicas.shard_by_work(work, 2)          # deterministic
    l0, l1 = (sum(work[s] for s in b) for b in b2)
    assert abs(l0 - l1) / (l0 + l1) < 1e-3
    # a rank's subset is the same systems as in the whole batch
    mats, ks, _ = inputs.batched_convection_diffusion(16, 4, systems=[5, 2])
    allm, allk, _ = inputs.batched_convection_diffusion(16, 4)
    assert ks == [allk[5], allk[2]]
    assert (mats[0] != allm[5]).nnz == 0 and (mats[1] != allm[2]).nnz == 0
    with pytest.raises(ValueError):
        inputs.batched_convection_diffusion(16, 4, systems=[16])


def test_shard_edge_cases():
    assert replicas.shard_by_work([], 3) == [[], [], []]
    assert replicas.shard_by_work([5.0], 2) == [[0], []]
    assert replicas.shard_by_work([1.0] * 4, 2) == [[0, 2], [1, 3]]   # ties by index, then rank
    with pytest.raises(ValueError):
        replicas.shard_by_work([1.0], 0)


def test_whole_job_rate_counts_every_replica():
    assert replicas.whole_job_rate(4e11, 1, 50.0) == pytest.approx(8e12)
    assert replicas.whole_job_rate(4e11, 2, 50.0) == pytest.approx(1.6e13)


def test_one_rank_group_is_the_identity():
    g = replicas.RankGroup(1, "cpu")
    g.barrier()
    assert (g.max(3.5), g.min(-1.0), g.sum(2.0)) == (3.5, -1.0, 2.0)
    stats = {k: float(i + 1) for i, k in enumerate(replicas.BATCH_COMBINE)}
    c = replicas.combine_batch_stats(g, stats)
    assert all(c[k] == stats[k] for k in replicas.BATCH_COMBINE)
    assert c["gflops"] == pytest.approx(stats["flops"] / (stats["ms"] / 1e3) / 1e9)


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, queue):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=60))
    try:
        w, r, loc = replicas.env_ranks()
        g = replicas.RankGroup(w, "cpu")
        g.barrier()
        res = {"env": (w, r, loc), "max": g.max(10.0 + r), "min": g.min(10.0 + r), "sum": g.sum(1.5)}
        sides = inputs.batched_sides(64, 4)
        mine = replicas.shard_by_work([replicas.lu_work_estimate(k) for k in sides], w)[r]
        local = {"ms": 20.0 + 5.0 * r, "flops": 1e9 * len(mine), "systems": float(len(mine)),
                 "n_total": float(sum(sides[s] ** 2 for s in mine)), "nnz_l_total": 100.0,
                 "all_converged": 1.0 if r == 0 else 0.0, "max_backward_error": 1e-12 * (r + 1),
                 "max_refine_iters": float(r + 1), "pivot_replacements": float(r)}
        res["combined"] = replicas.combine_batch_stats(g, local)
        res["mine"] = mine
        queue.put((r, res))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_combine():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = dict(queue.get(timeout=180) for _ in range(2))
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    sides = inputs.batched_sides(64, 4)
    for r in range(2):
        res = got[r]
        assert res["env"] == (2, r, r)
        assert (res["max"], res["min"], res["sum"]) == (11.0, 10.0, 3.0)
        c = res["combined"]
        assert c == got[0]["combined"]                    # every rank holds the same result
        assert c["ms"] == 25.0 and c["systems"] == 64.0 and c["flops"] == 64e9
        assert c["n_total"] == float(sum(k * k for k in sides))
        assert c["all_converged"] == 0.0 and c["max_backward_error"] == 2e-12
        assert c["max_refine_iters"] == 2.0 and c["pivot_replacements"] == 1.0
        assert c["gflops"] == pytest.approx(64e9 / 0.025 / 1e9)
    assert sorted(got[0]["mine"] + got[1]["mine"]) == list(range(64))
