"""Host-side logic of the multi-GPU benchmark, on CPU with gloo (world size 2).

Each rank runs an independent replica (weak scaling): the ranks draw
different point sets of the same recipe, and the reported time is the
maximum over ranks.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 10.0 + 5.0 * rank
        out[rank] = bench.max_over_ranks(mine, world)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == out[1] == 15.0


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5


def test_replicas_are_independent_draws_of_the_same_recipe():
    import bench
    from paper_1102_2878_gb300 import datagen

    x = datagen.isotropic_mixture(5000, 3, 6, 0.05, seed=1)
    a, b, c = bench.replica_points(x, 0), bench.replica_points(x, 1), bench.replica_points(x, 2)
    assert a is x
    assert b.shape == x.shape and b.dtype == np.float32 and not np.array_equal(b, x)
    assert not np.array_equal(b, c)
    assert np.array_equal(b, bench.replica_points(x, 1))  # deterministic per rank
    assert (b >= 0).all() and (b <= 1).all()
    # same distribution: means agree closely
    assert np.allclose(b.mean(0), x.mean(0), atol=2e-3)


def test_dist_env_defaults(monkeypatch):
    import bench

    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (0, 1, 0)
    monkeypatch.setenv("RANK", "3")
    monkeypatch.setenv("WORLD_SIZE", "4")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.dist_env() == (3, 4, 1)


def test_query_groups_spans():
    import bench

    # consecutive batches up to the limit; a batch above it stands alone
    assert bench.query_groups([5, 3, 10, 2, 2], 8) == [(0, 8), (8, 18), (18, 22)]
    assert bench.query_groups([20], 8) == [(0, 20)]
    assert bench.query_groups([1] * 5, 2) == [(0, 2), (2, 4), (4, 5)]
    spans = bench.query_groups([7, 1, 9, 4, 4, 30, 2], 12)
    assert spans[0][0] == 0 and spans[-1][1] == 57
    assert all(a < b for a, b in spans) and all(spans[k][1] == spans[k + 1][0] for k in range(len(spans) - 1))


def test_load_problem_shapes():
    import bench

    x, r, hs, eps, sizes = bench.load_problem("kde2d_n1e4", 500)
    assert x.shape == (500, 2) and r is None and sizes is None and eps == 1e-2
    q, r, hs, eps, sizes = bench.load_problem("kde32d_r1e6_q64batches", 2000)
    assert r.shape == (2000, 32) and q.shape == (sum(sizes), 32) and len(sizes) == 64 and len(hs) == 16
    assert eps == 1e-2 and q.dtype == np.float32 and q.flags["C_CONTIGUOUS"]
