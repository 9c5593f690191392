"""The benchmark's multi-rank plumbing on CPU: two gloo ranks, no GPU.

Each rank solves an independent subgame (weak scaling, no data-path collective); the only
cross-rank operations are the barrier and the max-over-ranks of the timed seconds, which
decide the whole-job throughput."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    r, w, _ = bench.dist_env()
    dist = bench.dist_init(w, use_cuda=False)
    bench.barrier(dist)
    # rank r pretends to have spent 1 + r seconds on 100 iterations
    value, t = bench.aggregate(100, 1.0 + r, w, dist)
    seeds = bench.workload_spec(r).seeds
    q.put((r, value, t, seeds))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_contract():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for r, value, t, _ in out:
        assert t == pytest.approx(2.0)            # slowest rank's time
        assert value == pytest.approx(200 / 2.0)  # all ranks' iterations / that time
    assert out[0][3] != out[1][3]                 # each rank solves its own subgame


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.dist_init(1, use_cuda=False) is None
    value, t = bench.aggregate(50, 2.0, 1, None)
    assert (value, t) == (25.0, 2.0)
